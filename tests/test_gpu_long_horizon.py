"""Accuracy of the mixed-precision form over many steps of the full-size
configurations: the complex64-bulk propagation against complex128 on the
GPU (itself checked against the oracle at these sizes in
test_gpu_full_size.py), observables compared every 20 steps.  The bar is
the mixed form's 1e-6 on populations (and on the reduced density matrix of
the HEOM system).  The configurations' full horizons (1000 and 2000 steps)
are measured by `bench.py --accuracy`; these tests cover the first 200
(vibronic) and 60 (HEOM) steps."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


def pair(lib, probs, blocks=16):
    out = []
    for precision in (lib.TTN_FP64, lib.TTN_MIXED):
        cs = []
        for p in probs:
            c = lib.Context(p.tree, precision)
            c.set_cluster(blocks)
            c.set_state(p.tensors)
            c.set_hamiltonian(p.H)
            cs.append(c)
        out.append(cs)
    return out


def curve(lib, probs, nsteps, every, observe):
    c64, cmx = pair(lib, probs)
    errs = []
    for _ in range(nsteps // every):
        lib.ttn_step_batch([c.h for c in c64], probs[0].dt, every)
        lib.ttn_step_batch([c.h for c in cmx], probs[0].dt, every)
        errs.append(max(float(np.abs(observe(a, p) - observe(b, p)).max()) for a, b, p in zip(cmx, c64, probs)))
    for c in c64 + cmx:
        c.close()
    return errs


def test_vibronic_2x24_mixed_200_steps(gpu_lib):
    probs = [W.config_c2(seed=s) for s in (2, 3)]
    errs = curve(gpu_lib, probs, 200, 20, lambda c, p: np.concatenate(c.populations(p.obs_leaves)))
    assert max(errs) <= MIXED_TOL, errs


def test_heom_k16_mixed_60_steps(gpu_lib):
    probs = [W.config_c4()]
    errs = curve(gpu_lib, probs, 60, 20, lambda c, p: np.asarray(c.vacuum_projection(p.meta["sys"])))
    assert max(errs) <= MIXED_TOL, errs
