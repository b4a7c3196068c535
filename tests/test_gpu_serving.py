"""Serving: continuous batching of independent propagations through
ttn_server (include/ttn.h).  Requests of different trees, bond dimensions,
local dimensions, Hamiltonians and time steps arrive while others run; each
result must equal the same propagation run alone with ttn_step."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


def request_problems(n, seed=5):
    rs = W.config_c5_requests(n, seed=seed, n_modes_range=(3, 10), d_range=(4, 8), chi_range=(2, 6),
                              steps_range=(4, 12))
    return [W.c5_problem(r) for r in rs]


def host_ctx(lib, p, precision):
    c = lib.Context(p.tree, precision, on_host=True)
    c.set_state(p.tensors)
    c.set_hamiltonian(p.H)
    return c


def run_alone(lib, p, precision):
    c = lib.Context(p.tree, precision)
    c.set_state(p.tensors)
    c.set_hamiltonian(p.H)
    c.step(p.dt, p.nsteps)
    st = c.get_state()
    pops = np.concatenate(c.populations(p.obs_leaves))
    c.close()
    return st, pops


def serve(lib, probs, precision, arrivals=(4, 2), **srv_kw):
    """Submit probs in waves (arrivals[0] first, then arrivals[1] per pump)
    and pump until every request has finished."""
    srv = lib.Server(precision, **srv_kw)
    ctxs, tickets, done = [], {}, {}
    nxt, first = 0, True
    while len(done) < len(probs):
        k = arrivals[0] if first else arrivals[1]
        first = False
        for _ in range(k):
            if nxt < len(probs):
                p = probs[nxt]
                c = host_ctx(lib, p, precision)
                assert c.device_bytes() == 0
                tickets[srv.submit(c, p.dt, p.nsteps)] = nxt
                ctxs.append(c)
                nxt += 1
        srv.pump()
        for t, st in srv.poll():
            done[tickets[t]] = st
    return srv, ctxs, done


def test_serving_alone_equals_mix(gpu_lib):
    probs = request_problems(12)
    srv, ctxs, done = serve(gpu_lib, probs, gpu_lib.TTN_MIXED, slice_ms=0.5)
    assert all(st == gpu_lib.TTN_OK for st in done.values())
    stats = srv.stats()
    assert stats["completed"] == len(probs)
    assert stats["steps"] == sum(p.nsteps for p in probs)
    assert stats["peak_running"] >= 2           # requests overlapped on the device
    assert stats["launches"] > 1
    assert stats["n_latencies"] == sum(p.nsteps - 1 for p in probs)
    assert 0 < stats["p50_step_ms"] <= stats["p99_step_ms"]
    for p, c in zip(probs, ctxs):
        assert c.device_bytes() == 0            # retired to the host
        want_state, want_pops = run_alone(gpu_lib, p, gpu_lib.TTN_MIXED)
        for x, y in zip(want_state, c.get_state()):
            assert np.array_equal(x, y)
        got_pops = np.concatenate(c.populations(p.obs_leaves))
        assert np.abs(got_pops - want_pops).max() <= MIXED_TOL
        c.close()
    srv.close()


def test_serving_fp64_matches_alone(gpu_lib):
    probs = request_problems(5, seed=7)
    srv, ctxs, done = serve(gpu_lib, probs, gpu_lib.TTN_FP64, arrivals=(2, 1), slice_ms=0.5)
    assert all(st == gpu_lib.TTN_OK for st in done.values())
    for p, c in zip(probs, ctxs):
        want_state, _ = run_alone(gpu_lib, p, gpu_lib.TTN_FP64)
        for x, y in zip(want_state, c.get_state()):
            assert np.array_equal(x, y)
        c.close()
    srv.close()


def test_admission_by_footprint(gpu_lib):
    probs = request_problems(8, seed=9)
    fps = sorted(host_ctx(gpu_lib, p, gpu_lib.TTN_MIXED).footprint() for p in probs)
    budget = fps[-1] + fps[-2]                  # the two largest fit side by side
    assert budget < sum(fps)                    # but not everything at once
    srv = gpu_lib.Server(gpu_lib.TTN_MIXED, hbm_budget=budget, slice_ms=0.5, use_graph=False)
    ctxs = []
    for p in probs:
        c = host_ctx(gpu_lib, p, gpu_lib.TTN_MIXED)
        srv.submit(c, p.dt, p.nsteps)
        ctxs.append(c)
    while True:
        running, queued = srv.pump()
        st = srv.stats()
        assert st["bytes_in_use"] <= budget
        if running == 0 and queued == 0:
            break
    st = srv.stats()
    assert st["completed"] == len(probs) and st["failed"] == 0
    assert st["peak_bytes"] <= budget
    assert st["peak_running"] < len(probs)      # the budget held requests back
    for p, c in zip(probs, ctxs):
        want_state, _ = run_alone(gpu_lib, p, gpu_lib.TTN_MIXED)
        for x, y in zip(want_state, c.get_state()):
            assert np.array_equal(x, y)
        c.close()
    srv.close()


def test_oversized_request_rejected(gpu_lib):
    probs = request_problems(3, seed=11)
    ctxs = [host_ctx(gpu_lib, p, gpu_lib.TTN_MIXED) for p in probs]
    fps = [c.footprint() for c in ctxs]
    big = int(np.argmax(fps))
    budget = max(f for i, f in enumerate(fps) if i != big)
    if budget >= fps[big]:
        pytest.skip("no request is larger than the others")
    srv = gpu_lib.Server(gpu_lib.TTN_MIXED, hbm_budget=budget, slice_ms=0.5)
    tickets = {srv.submit(c, p.dt, p.nsteps): i for i, (c, p) in enumerate(zip(ctxs, probs))}
    srv.drain()
    status = {tickets[t]: s for t, s in srv.poll()}
    assert status[big] == gpu_lib.TTN_E_OOM
    assert all(status[i] == gpu_lib.TTN_OK for i in range(len(probs)) if i != big)
    srv.close()
    for c in ctxs:
        c.close()


def test_materialize_evict_round_trip(gpu_lib):
    p = W.config_c1()
    c = host_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    fp = c.footprint()
    c.materialize()
    assert c.device_bytes() == fp
    c.step(p.dt, 3)
    mid = c.get_state()
    c.evict()
    assert c.device_bytes() == 0
    for x, y in zip(mid, c.get_state()):
        assert np.array_equal(x, y)
    c.step(p.dt, 3)                             # materialises again
    ref = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    ref.set_state(p.tensors)
    ref.set_hamiltonian(p.H)
    ref.step(p.dt, 6)
    for x, y in zip(ref.get_state(), c.get_state()):
        assert np.array_equal(x, y)
    assert gpu_lib.ttn_step_stats(c.h)[0] == 6
    ref.close()
    c.close()


def test_serving_cluster_lanes_alone_equals_mix(gpu_lib):
    """Requests on one block and on 4-block clusters in one stream: the
    server runs them in two lanes whose launches overlap; every result
    equals ttn_step alone with the same block count, bit for bit."""
    probs = request_problems(8, seed=9)
    blocks = [4 if i % 2 else 1 for i in range(len(probs))]
    precision = gpu_lib.TTN_MIXED
    srv = gpu_lib.Server(precision, slice_ms=0.5)
    ctxs, tickets, done = [], {}, {}
    for i, p in enumerate(probs):
        c = host_ctx(gpu_lib, p, precision)
        c.set_cluster(blocks[i])
        tickets[srv.submit(c, p.dt, p.nsteps)] = i
        ctxs.append(c)
        if i % 3 == 2:
            srv.pump()
    while len(done) < len(probs):
        srv.pump()
        for t, st in srv.poll():
            done[tickets[t]] = st
    assert all(st == gpu_lib.TTN_OK for st in done.values())
    stats = srv.stats()
    assert stats["completed"] == len(probs)
    assert stats["steps"] == sum(p.nsteps for p in probs)
    for i, (p, c) in enumerate(zip(probs, ctxs)):
        a = gpu_lib.Context(p.tree, precision)
        a.set_cluster(blocks[i])
        a.set_state(p.tensors)
        a.set_hamiltonian(p.H)
        a.step(p.dt, p.nsteps)
        for x, y in zip(a.get_state(), c.get_state()):
            assert np.array_equal(x, y)
        a.close()
        c.close()
    srv.close()
