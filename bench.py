#!/usr/bin/env python
"""TTN-TDVP throughput benchmark on GB300.

Workload: the two-state x 24-mode vibronic model on its 4-layer ML tree
(bonds 24/16/12/8 from the root down, local dimensions 10..30, dt = 0.1), as
a batch of seeded instances (seed s draws frequencies, couplings and local
dimensions).  One step = one projector-splitting TDVP step (forward and
reverse sweep) of every instance in the batch, one kernel launch.

Metric: TDVP steps/s summed over instances, batched mixed precision
(complex64 bulk, FP64 state / Krylov scalars / QR); the plain FP64 path on
the same batch, the population error between the two, and p50/p99 per-step
latency (device time stamps between consecutive step completions of an
instance) are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
    python bench.py --impl reference ...     # the CPU oracle on the same workload
    python bench.py --serve                  # serving stream through ttn_server (own JSON line)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "TTN-TDVP steps/s: batched mixed-precision vs FP64 at <=1e-6 pop. error; p50/p99"
UNIT = "steps/s"
DT = 0.1
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2          # 1/64 of the FP32 rate on GB300
N_SM = 152
SM_MAX_MHZ = 2070.0
PEAK_FP32 = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # TFLOP/s
PEAK_FP64 = N_SM * FP64_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


# the sources of the sweep kernel: a traffic figure counts only while they
# are the ones it was measured on
KERNEL_SOURCES = ("ttn_device.cuh", "ttn_tc.cuh", "ttn_variant.cuh", "ttn_var_mix_solo.cu", "ttn_program.h")


def kernel_source_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2503_15460_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(batch):
    """DRAM bytes of one launch (batch instance-steps) from the committed ncu
    summary, if it was measured on the current kernel source; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_program_kernel_vibronic2x24_mixed.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2503_15460_gb300", "csrc", f), "rb").read())
    if h.hexdigest() != rec.get("kernel_source_sha256"):
        return None
    return rec["dram_bytes_per_instance_step"] * batch


def workload_name(batch, workload="vibronic"):
    if workload == "heom":
        return (f"HEOM spin-boson as a TTN: 16 exponentials (Drude-Lorentz + 15 Matsubara), depth 10 "
                f"(32 modes of dim 11), system leaf dim 4, balanced binary tree (65 nodes), chi 24, Arnoldi; "
                f"batch of {batch} instances sweeping the reorganisation energy lambda, dt={WORKLOAD_DT[workload]}")
    if workload == "multiset":
        return (f"multi-set linear vibronic model (the sets are {MULTISET_SHAPE['n_states']} electronic states, "
                f"one TTN each): {MULTISET_SHAPE['n_modes']} modes of dim {MULTISET_SHAPE['d']}, balanced binary "
                f"tree, bonds {MULTISET_SHAPE['chi']}, every set occupied at t = 0 (amplitudes {MULTISET_AMPS}, "
                f"normalised); batch of {batch} seeded instances, "
                f"dt={WORKLOAD_DT[workload]}")
    if workload == "spinboson300":
        return (f"spin-boson, 1 spin + 300 Ohmic modes (wc 5, orthogonal-polynomial bath on [0, 50]), d 20, "
                f"balanced binary tree (601 nodes), fixed chi 8; batch of {batch} instances sweeping alpha "
                f"in [0.1, 0.5], dt={WORKLOAD_DT[workload]}")
    return (f"vibronic 2 states x 24 modes, ML tree depth 4 (46 nodes, bonds 24/16/12/8, "
            f"local dims 10..30), batch of {batch} seeded instances, dt={DT}")


WORKLOAD_DT = {"vibronic": DT, "heom": 0.015, "spinboson300": 0.01, "multiset": 0.1}
MULTISET_SHAPE = {"n_states": 4, "n_modes": 16, "d": 8, "chi": 8}
# every set occupied at t = 0 (a superposition): a start with empty sets is
# ill-conditioned at truncated bonds, so the mixed-vs-complex128 check would
# measure the conditioning, not the arithmetic
MULTISET_AMPS = (0.85, 0.3, 0.3, 0.3)


def rank_seed0(batch, rank):
    """First seed of a rank's instances: ranks draw disjoint seed ranges
    (weak scaling: every rank holds `batch` independent instances)."""
    return 2 + rank * batch


def max_over_ranks(x, world, device):
    """The slowest rank's value (no-op for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(batch, world, steps, seconds):
    """Whole-job instance-steps per second."""
    return batch * world * steps / seconds


def make_problems(batch, seed0, workload="vibronic"):
    """Instances of a workload; instance index i = seed0 + i - 2 picks the
    seed (vibronic) or the swept parameter (heom: lambda, spinboson300:
    alpha)."""
    import workloads as W
    if workload == "heom":
        return [W.config_c4(lam=0.05 + 0.0005 * (seed0 - 2 + i)) for i in range(batch)]
    if workload == "multiset":
        return [W.multiset_vibronic_problem(seed=seed0 + i, dt=WORKLOAD_DT["multiset"], amps=MULTISET_AMPS,
                                            **MULTISET_SHAPE)
                for i in range(batch)]
    if workload == "spinboson300":
        # alpha only scales the couplings (g ~ sqrt(alpha)): discretise once
        import dataclasses
        base = W.config_c3(alpha=0.1)
        out = []
        for i in range(batch):
            a = 0.1 + 0.4 * (((seed0 - 2 + i) * 0.618034) % 1.0)
            sc = np.sqrt(a / 0.1)
            H = dataclasses.replace(base.H, coeffs=[c * sc if len(f) == 2 else c
                                                    for c, f in zip(base.H.coeffs, base.H.factors)])
            out.append(dataclasses.replace(base, H=H, name=f"c3_alpha{a:.4f}"))
        return out
    return [W.config_c2(seed=seed0 + i) for i in range(batch)]


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def observed_populations(ctx, p):
    """Site populations of the observed leaves, or the set populations of a
    multi-set state."""
    import workloads as W
    if isinstance(p, W.MultiSetProblem):
        return ctx.set_populations()
    return np.concatenate(ctx.populations(p.obs_leaves))


def run_ours(args, rank, world, local_rank):
    import torch
    import workloads as W
    torch.cuda.set_device(local_rank)
    from paper_2503_15460_gb300 import ttn
    ttn.ttn_set_device(local_rank)
    stream = torch.cuda.Stream()
    batch = args.batch
    DT = WORKLOAD_DT[args.workload]
    probs = make_problems(batch, rank_seed0(batch, rank), args.workload)

    def make_ctxs(precision, subset=None):
        out = []
        for p in (probs if subset is None else subset):
            c = ttn.Context(p.tree, precision)
            ttn.ttn_set_stream(c.h, stream.cuda_stream)
            if isinstance(p, W.MultiSetProblem):
                c.set_multiset_hamiltonian(p.H)
                c.set_multiset_state(p.tensors)
            else:
                c.set_state(p.tensors)
                c.set_hamiltonian(p.H)
            out.append(c)
        return out

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # measured pipe peaks of this device (roofline denominators)
    peaks = ttn.ttn_pipe_peaks(stream.cuda_stream, 0.5)

    # ---- mixed precision, batched: the headline ------------------------------
    ctxs = make_ctxs(ttn.TTN_MIXED)
    handles = [c.h for c in ctxs]
    batch_bytes = sum(ttn.ttn_device_bytes(h) for h in handles)
    for _ in range(args.warmup):
        ttn.ttn_step_batch(handles, DT, 1)
    fl0 = np.sum([ttn.ttn_flop_counts(h) for h in handles], axis=0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                ttn.ttn_step_batch(handles, DT, 1)
            ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
    clocks = clk.summary()
    fl1 = np.sum([ttn.ttn_flop_counts(h) for h in handles], axis=0)
    flops_per_step, flops64_per_step = (fl1 - fl0) / args.steps
    lat = []
    for h in handles:
        _, _, st = ttn.ttn_step_stats(h, args.steps + 1)
        if len(st) >= 2:
            lat.extend(np.diff(st.astype(np.float64)) / 1e6)
    value = aggregate_rate(batch, world, args.steps, ms / 1e3)

    # ---- plain FP64 on the same batch ----------------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        c64 = make_ctxs(ttn.TTN_FP64)
        h64 = [c.h for c in c64]
        ttn.ttn_step_batch(h64, DT, 1)                      # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.fp64_steps):
                ttn.ttn_step_batch(h64, DT, 1)
            e1.record(stream)
        e1.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        for c in c64:
            c.close()
        fp64 = {"value": aggregate_rate(batch, world, args.fp64_steps, ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps}
        # accuracy over the whole benchmarked horizon: the first instances of
        # the timed mixed batch (warm-up + timed steps) against the same
        # instances propagated in complex128 (each on a 16-block cluster)
        nchk = min(args.check_instances, batch)
        horizon = args.warmup + args.steps
        cref = make_ctxs(ttn.TTN_FP64, probs[:nchk])
        for c in cref:
            ttn.ttn_set_cluster(c.h, 16)
        ttn.ttn_step_batch([c.h for c in cref], DT, horizon)
        err = 0.0
        for a, b, p in zip(ctxs[:nchk], cref, probs[:nchk]):
            pa, pb = observed_populations(a, p), observed_populations(b, p)
            err = max(err, float(np.abs(pa - pb).max()))
        for c in cref:
            c.close()
        fp64["pop_err_mixed_vs_fp64"] = err
        fp64["pop_err_steps"] = horizon
        fp64["pop_err_instances"] = nchk
        fp64["pop_err_note"] = ("max |population| difference over all leaves (multi-set: over the sets) after the "
                                "warm-up and timed steps of "
                                "the benchmarked mixed batch, against complex128 from the same initial states")

    # ---- end to end through the public API (host buffers) --------------------
    e2e = None
    if args.e2e:
        t0 = time.perf_counter()
        torch.cuda.synchronize()
        ce = []
        h2d = 0
        for p in probs:
            c = ttn.Context(p.tree, ttn.TTN_MIXED)
            ttn.ttn_set_stream(c.h, stream.cuda_stream)
            c.set_state(p.tensors)
            c.set_hamiltonian(p.H)
            coeff, tp, lf, mats, off = p.H.to_csr()
            h2d += sum(a.nbytes for a in p.tensors) + coeff.nbytes + tp.nbytes + lf.nbytes + mats.nbytes + off.nbytes
            ce.append(c)
        ttn.ttn_step_batch([c.h for c in ce], DT, args.steps)
        d2h = 0
        for c, p in zip(ce, probs):
            pops = c.populations(p.obs_leaves)
            d2h += sum(x.nbytes for x in pops) * 2      # complex d x d read back per leaf
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        el = max_over_ranks(t1 - t0, world, "cuda")
        e2e = {"value": aggregate_rate(batch, world, args.steps, el), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "includes": "context creation, state and Hamiltonian upload, K steps, population read-back"}
        for c in ce:
            c.close()

    for c in ctxs:
        c.close()
    return dict(ms=ms, value=value, flops_per_step=float(flops_per_step), flops64_per_step=float(flops64_per_step),
                lat=lat, clocks=clocks, fp64=fp64, e2e=e2e, batch_bytes=batch_bytes, peaks=peaks)


def alu_roofline(flops, flops64, seconds, traffic, peaks=None):
    """Per-pipe utilisation of one step: FP32 work against the FP32 pipe,
    FP64 work against the FP64 pipe; the pipe with the larger lower bound
    on time is the one that binds.  peaks = (fp32, fp64) TFLOP/s measured in
    this run by the FMA-throughput kernels (ttn_pipe_peaks); else the unit
    counts at the maximum clock."""
    f32 = flops - flops64
    a32, a64 = f32 / seconds / 1e12, flops64 / seconds / 1e12
    p32, p64 = peaks if peaks else (PEAK_FP32, PEAK_FP64)
    pipes = {"fp32": {"achieved": a32, "peak": p32, "frac": a32 / p32, "flops_per_step": f32,
                      "nominal_peak": PEAK_FP32},
             "fp64": {"achieved": a64, "peak": p64, "frac": a64 / p64, "flops_per_step": flops64,
                      "nominal_peak": PEAK_FP64}}
    bind = max(pipes, key=lambda k: pipes[k]["frac"])
    b = pipes[bind]
    src = ("measured in this run: FP32 / FP64 fused multiply-add throughput of a kernel filling every SM with "
           "independent FMA chains (ttn_pipe_peaks, CUDA events), fractions are of measured") if peaks else (
           f"derived: {N_SM} SMs x {FP32_LANES_PER_SM} FP32 / {FP64_LANES_PER_SM} FP64 lanes x 2 flop x "
           f"{SM_MAX_MHZ:.0f} MHz")
    return {"bound": "alu", "pipe": bind, "achieved": b["achieved"], "peak": b["peak"], "unit": "TFLOP/s",
            "frac": b["frac"], "traffic": traffic, "peak_source": src,
            "pipes": pipes, "flops_per_step": flops}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_leg(args, steps, one_core):
    """Time `steps` oracle steps of instance seed 2 in a child process: on one
    core with one BLAS thread, or on every core with one BLAS thread per core."""
    cores = len(os.sched_getaffinity(0))
    threads = 1 if one_core else cores
    code = (
        "import os, sys, time; sys.path.insert(0, %r)\n"
        "%s"
        "import workloads as W\n"
        "from oracle.ttn import TTN\n"
        "p = W.config_c2(seed=2)\n"
        "s = TTN(p.tree, p.H, p.tensors)\n"
        "t0 = time.perf_counter(); s.step(p.dt, %d); t1 = time.perf_counter()\n"
        "print(t1 - t0)\n" % (ROOT, ("os.sched_setaffinity(0, {min(os.sched_getaffinity(0))})\n" if one_core else ""),
                                steps))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1 if one_core else cores, "kind": "oracle",
                "error": r.stderr[-300:]}
    el = float(r.stdout.strip().splitlines()[-1])
    return {"value": steps / el, "unit": UNIT, "cores": 1 if one_core else cores, "kind": "oracle",
            "blas_threads": threads, "seconds": el,
            "sample": f"{steps} TDVP step(s) of 1 instance (seed 2) of the workload, NumPy complex128 oracle"}


def cpu_baseline(args):
    """The oracle, as it stands, on one instance of the same workload for a
    bounded number of steps: one leg pinned to one core (BLAS threads 1),
    one on all host cores (BLAS threads = cores); the all-core leg is the
    reported value."""
    allc = _oracle_leg(args, args.cpu_steps, one_core=False)
    one = _oracle_leg(args, args.cpu_steps, one_core=True)
    out = dict(allc)
    out["cpu_model"] = cpu_model()
    out["single_core"] = one
    return out


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed on the same workload."""
    if rank != 0:
        return 0
    import workloads as W
    from oracle.ttn import TTN
    p = W.config_c2(seed=2)
    s = TTN(p.tree, p.H, p.tensors)
    for _ in range(args.warmup):
        s.step(p.dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(p.dt, 1)
    el = time.perf_counter() - t0
    value = args.steps / el
    cores = len(os.sched_getaffinity(0))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "impl": "reference",
            # the same workload as our arm; each timed step is a bounded
            # sample of it: one step of one of its instances (instance-steps/s)
            "config": {"workload": workload_name(args.batch), "global_batch": args.batch * world,
                       "instances_per_gpu": args.batch, "precision": "fp64 (oracle)",
                       "sample": "each step: one TDVP step of instance 0 (seed 2) of the batch"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed TDVP steps of 1 instance (seed 2) of the "
                                       f"{args.batch}-instance workload, NumPy complex128"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# accuracy of the mixed form over long horizons (separate JSON line)
# ---------------------------------------------------------------------------
ACCURACY_WORKLOADS = ("vibronic", "heom", "spinboson300")


def accuracy_problems(workload, n):
    import workloads as W
    if workload == "heom":
        return [W.config_c4(lam=0.1 * (1.0 + 0.25 * i)) for i in range(n)]
    if workload == "spinboson300":
        return [W.config_c3(alpha=a) for a in (0.1, 0.5)[:n]]
    return [W.config_c2(seed=2 + i) for i in range(n)]


def accuracy_observables(ctx, p, workload):
    """Vibronic / spin-boson: every leaf's populations; HEOM: the reduced
    density matrix of the system (all four elements of vec rho_S)."""
    if workload == "heom":
        return np.asarray(ctx.vacuum_projection(p.meta["sys"]))
    return np.concatenate(ctx.populations(p.obs_leaves))


def run_accuracy(args):
    """Mixed against complex128 on the GPU over a configuration's horizon:
    both arms batched (one launch per interval and precision), each instance
    on a 16-block cluster; the largest observable difference is recorded
    every `--acc-every` steps."""
    import torch
    torch.cuda.set_device(0)
    from paper_2503_15460_gb300 import ttn
    ttn.ttn_set_device(0)
    wl = args.workload
    probs = accuracy_problems(wl, args.acc_instances)
    dt = probs[0].dt
    steps = args.acc_steps or probs[0].nsteps

    def ctxs(precision):
        out = []
        for p in probs:
            c = ttn.Context(p.tree, precision)
            c.set_cluster(args.acc_cluster)
            c.set_state(p.tensors)
            c.set_hamiltonian(p.H)
            out.append(c)
        return out

    c64, cmx = ctxs(ttn.TTN_FP64), ctxs(ttn.TTN_MIXED)
    curve, done, t64, tmx = [], 0, 0.0, 0.0
    while done < steps:
        k = min(args.acc_every, steps - done)
        t0 = time.perf_counter()
        ttn.ttn_step_batch([c.h for c in c64], dt, k)
        t1 = time.perf_counter()
        ttn.ttn_step_batch([c.h for c in cmx], dt, k)
        t2 = time.perf_counter()
        t64 += t1 - t0
        tmx += t2 - t1
        done += k
        err = max(float(np.abs(accuracy_observables(a, p, wl) - accuracy_observables(b, p, wl)).max())
                  for a, b, p in zip(cmx, c64, probs))
        curve.append([done, err])
        print(f"[accuracy] {wl} step {done}: max |mixed - fp64| = {err:.3e}", file=sys.stderr, flush=True)
    norms = [float(c.norm_energy()[0]) for c in c64]
    for c in c64 + cmx:
        c.close()
    line = {"metric": "max |observable(mixed) - observable(complex128)| over the horizon, GPU",
            "workload": wl, "instances": [p.name for p in probs], "dt": dt, "steps": steps,
            "observable": "vec rho_S of the system" if wl == "heom" else "populations of every leaf",
            "max_err": max(e for _, e in curve), "curve": curve, "cluster_blocks": args.acc_cluster,
            "seconds_fp64": t64, "seconds_mixed": tmx, "fp64_norm_end": norms}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# serving stream (continuous batching through ttn_server)
# ---------------------------------------------------------------------------
SERVE_RANGES = dict(n_modes_range=(8, 64), d_range=(8, 20), chi_range=(4, 12), steps_range=(10, 40))
# the serving leg of the default run: the same recipe, fewer requests and steps
SERVE_RANGES_DEFAULT = dict(n_modes_range=(8, 48), d_range=(8, 20), chi_range=(4, 12), steps_range=(6, 20))


def serve_workload_name(n, ranges):
    r = ranges
    return (f"{n} seeded requests, half spin-boson (dt 0.05, alpha U[0.05,1], beta in {{inf,5,1}}) and half "
            f"two-state vibronic (dt 0.1), balanced binary trees, modes {r['n_modes_range']}, local dims "
            f"{r['d_range']}, bond dims {r['chi_range']}, steps {r['steps_range']}")


def serve_stream(ttn, W, n_requests, ranges, slice_ms, burst=True, sample=8, sample_steps=3, log=None):
    """Continuous batching of a seeded request stream through ttn_server:
    optionally all requests at t0 (burst), then Poisson arrivals at 80 % of
    the measured capacity; the reference runs a sample of the requests one
    at a time in FP64 (ttn_step)."""
    reqs = W.config_c5_requests(n_requests, seed=5, **ranges)
    probs = [W.c5_problem(r) for r in reqs]
    total_steps = sum(p.nsteps for p in probs)
    log = log or (lambda m: None)

    def contexts(precision):
        cs = []
        for p in probs:
            c = ttn.Context(p.tree, precision, on_host=True)
            c.set_state(p.tensors)
            c.set_hamiltonian(p.H)
            cs.append(c)
        return cs

    def run(arrivals):
        ctxs = contexts(ttn.TTN_MIXED)
        srv = ttn.Server(ttn.TTN_MIXED, slice_ms=slice_ms)
        order = np.argsort(arrivals, kind="stable")
        t_arr, t_done, tick = {}, {}, {}
        nxt = 0
        t0 = time.perf_counter()
        while len(t_done) < len(probs):
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals[order[nxt]] <= now:
                i = int(order[nxt])
                tick[srv.submit(ctxs[i], probs[i].dt, probs[i].nsteps)] = i
                t_arr[i] = now
                nxt += 1
            running, queued = srv.pump()
            if running == 0 and queued == 0 and nxt < len(order):
                time.sleep(max(0.0, arrivals[order[nxt]] - (time.perf_counter() - t0)))
            for t, st in srv.poll():
                if st != ttn.TTN_OK:
                    raise RuntimeError(f"request {tick[t]} failed with status {st}")
                t_done[tick[t]] = time.perf_counter() - t0
        makespan = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        for c in ctxs:
            c.close()
        resp = np.array([t_done[i] - t_arr[i] for i in range(len(probs))])
        return {"steps_per_s": total_steps / makespan, "makespan_s": makespan,
                "p50_step_ms": st["p50_step_ms"], "p99_step_ms": st["p99_step_ms"],
                "p50_request_s": float(np.percentile(resp, 50)), "p99_request_s": float(np.percentile(resp, 99)),
                "launches": st["launches"], "peak_running": st["peak_running"],
                "peak_bytes": st["peak_bytes"]}

    log(f"{len(probs)} requests, {total_steps} steps")
    out = {"requests": len(probs), "steps": total_steps}
    if burst:
        b = run(np.zeros(len(probs)))
        log(f"burst: {b['makespan_s']:.1f} s, {b['steps_per_s']:.1f} steps/s")
        capacity = b["steps_per_s"]
        out["burst"] = b
    else:
        # capacity from a burst of the first quarter of the stream
        sub = min(len(probs), max(8, len(probs) // 4))
        saved = probs
        probs = probs[:sub]
        total_sub = sum(p.nsteps for p in probs)
        b = run(np.zeros(len(probs)))
        probs = saved
        capacity = b["steps_per_s"]
        out["capacity_probe"] = {"requests": sub, "steps": total_sub, "steps_per_s": capacity}
    rate = 0.8 * capacity / (total_steps / len(probs))        # requests per second
    rng = np.random.default_rng(55)
    arr = np.cumsum(rng.exponential(1.0 / rate, len(probs)))
    pois = run(arr)
    pois["arrival_rate_per_s"] = rate
    log(f"poisson: {pois['makespan_s']:.1f} s, {pois['steps_per_s']:.1f} steps/s")
    out["poisson"] = pois
    # reference: one request at a time, complex128, on a sample of requests and steps
    t, sample_steps_done = 0.0, 0
    for i in range(min(sample, len(probs))):
        p = probs[i]
        n = min(p.nsteps, sample_steps)
        c = ttn.Context(p.tree, ttn.TTN_FP64)
        c.set_state(p.tensors)
        c.set_hamiltonian(p.H)
        t0 = time.perf_counter()
        c.step(p.dt, n)
        t += time.perf_counter() - t0
        sample_steps_done += n
        c.close()
    alone = sample_steps_done / t
    log(f"one at a time FP64: {alone:.2f} steps/s over {sample_steps_done} steps")
    out["one_at_a_time_fp64"] = {"value": alone, "unit": UNIT,
                                 "sample": f"first {min(sample, len(probs))} requests run alone with ttn_step, at "
                                           f"most {sample_steps} steps each ({sample_steps_done} steps)"}
    out["speedup_vs_one_at_a_time_fp64"] = pois["steps_per_s"] / alone
    return out


def run_serving(args):
    """--serve: the serving stream (all requests at t0, then Poisson
    arrivals at 80 % of the burst's capacity) as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    from paper_2503_15460_gb300 import ttn
    import workloads as W
    ttn.ttn_set_device(0)
    ranges = dict(SERVE_RANGES)
    if args.serve_full:
        ranges = dict(n_modes_range=(8, 128), d_range=(8, 20), chi_range=(8, 48), steps_range=(100, 400))
    if args.serve_steps_range:
        ranges["steps_range"] = tuple(args.serve_steps_range)
    res = serve_stream(ttn, W, args.serve_requests, ranges, args.slice_ms, burst=True,
                       sample=args.serve_sample, sample_steps=args.serve_sample_steps,
                       log=lambda m: print(f"[serve] {m}", file=sys.stderr, flush=True))
    line = {
        "metric": "serving: aggregate TTN-TDVP steps/s, continuous batching (mixed) vs one request at a time (FP64)",
        "value": res["poisson"]["steps_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
        "dtype": "c64 bulk / f64 state", "data": "synthetic",
        "config": {"workload": serve_workload_name(args.serve_requests, ranges),
                   "arrivals": "Poisson at 80% of the burst capacity (seed 55)", "slice_ms": args.slice_ms},
        **res,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=2 * N_SM, help="instances per GPU (two thread blocks per SM)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--check-instances", type=int, default=4)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu", action="store_false")
    ap.add_argument("--workload", default="vibronic", choices=sorted(WORKLOAD_DT),
                    help="vibronic (the headline), heom, spinboson300 or multiset (batched parameter sweeps)")
    ap.add_argument("--serve", action="store_true", help="run the serving stream instead (separate JSON line)")
    ap.add_argument("--accuracy", action="store_true",
                    help="mixed against complex128 over the workload's horizon instead (separate JSON line)")
    ap.add_argument("--acc-steps", type=int, default=0, help="horizon (0: the configuration's step count)")
    ap.add_argument("--acc-every", type=int, default=50)
    ap.add_argument("--acc-instances", type=int, default=2)
    ap.add_argument("--acc-cluster", type=int, default=16)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-steps-range", type=int, nargs=2, default=None, metavar=("LO", "HI"),
                    help="override the requests' step counts (a bounded sample of the same size ranges)")
    ap.add_argument("--serve-full", action="store_true",
                    help="--serve with the paper-shaped ranges (8-128 modes, bond dims 8-48, 100-400 steps)")
    ap.add_argument("--default-serve-requests", type=int, default=160,
                    help="requests of the serving leg of the default run (0: skip it)")
    ap.add_argument("--serve-sample", type=int, default=8)
    ap.add_argument("--serve-sample-steps", type=int, default=3)
    ap.add_argument("--slice-ms", type=float, default=20.0)
    args = ap.parse_args()
    if args.serve:
        return run_serving(args)
    if args.accuracy:
        return run_accuracy(args)
    if args.workload != "vibronic":
        args.e2e = args.cpu = False      # those legs are defined on the headline workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    r = run_ours(args, rank, world, local_rank)
    if rank == 0:
        lat = sorted(r["lat"])
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 bulk / f64 state", "data": "synthetic",
            "config": {"workload": workload_name(args.batch, args.workload), "global_batch": args.batch * world,
                       "instances_per_gpu": args.batch, "precision": "mixed",
                       "l2": f"inputs larger than L2: the batch holds {r['batch_bytes'] / 1e9:.1f} GB on the device",
                       "parallelism": f"replicas x{world}, one thread block per instance"},
            "batch_step_interval_p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "batch_step_interval_p99_ms": float(np.percentile(lat, 99)) if lat else None,
            "batch_step_interval_note": ("interval between consecutive step completions of one instance in the "
                                         "lock-step batch (every instance steps together); serving latency is "
                                         "under 'serving'"),
            "fp64": r["fp64"],
            "speedup_vs_fp64": (r["value"] / r["fp64"]["value"]) if r["fp64"] else None,
            "gpu_launches": args.steps,
            "roofline": alu_roofline(r["flops_per_step"], r["flops64_per_step"], r["ms"] / args.steps / 1e3,
                                     measured_traffic(args.batch) if args.workload == "vibronic" else None,
                                     r["peaks"]),
            "clocks": r["clocks"],
            "e2e": r["e2e"],
        }
        if args.default_serve_requests > 0 and args.workload == "vibronic" and world == 1:
            from paper_2503_15460_gb300 import ttn as _ttn
            import workloads as _W
            sv = serve_stream(_ttn, _W, args.default_serve_requests, SERVE_RANGES_DEFAULT, args.slice_ms,
                              burst=False, sample=args.serve_sample, sample_steps=args.serve_sample_steps)
            line["serving"] = {
                "workload": serve_workload_name(args.default_serve_requests, SERVE_RANGES_DEFAULT),
                "arrivals": "Poisson at 80% of the capacity measured on a burst of the first quarter (seed 55)",
                "steps_per_s": sv["poisson"]["steps_per_s"], "unit": UNIT,
                "p50_step_ms": sv["poisson"]["p50_step_ms"], "p99_step_ms": sv["poisson"]["p99_step_ms"],
                "p50_request_s": sv["poisson"]["p50_request_s"], "p99_request_s": sv["poisson"]["p99_request_s"],
                "one_at_a_time_fp64": sv["one_at_a_time_fp64"],
                "speedup_vs_one_at_a_time_fp64": sv["speedup_vs_one_at_a_time_fp64"],
                "detail": sv,
            }
        if args.cpu:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
