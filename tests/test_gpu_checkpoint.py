"""Checkpoint / resume (ttn_save, ttn_load): a propagation stopped, saved,
loaded into a fresh context and continued gives bit-identical tensors to
the uninterrupted one, in both precisions and after subspace expansion."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["TTN_FP64", "TTN_MIXED"])
def test_resume_is_bit_identical(gpu_lib, precision):
    prec = getattr(gpu_lib, precision)
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    a = gpu_lib.Context(p.tree, prec)
    a.set_state(p.tensors)
    a.set_hamiltonian(p.H)
    a.step(p.dt, 3)
    blob = a.save()
    b = gpu_lib.Context(W.config_c1().tree, prec)      # any tree: load replaces it
    b.load(blob)
    a.step(p.dt, 3)
    b.step(p.dt, 3)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert gpu_lib.ttn_step_stats(b.h)[0] == 6
    a.close(); b.close()


def test_resume_after_expansion(gpu_lib):
    p = W.config_c1(chi=2, d=4)
    opts = gpu_lib.ttn_step_opts(expand=1, eps_spawn=1e-6, chi_max=6)
    a = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    a.set_state(p.tensors)
    a.set_hamiltonian(p.H)
    a.step(p.dt, 6, opts)
    grown = a.bond_dims()
    assert np.any(grown[1:] > p.tree.bond_dim[1:])
    b = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    b.load(a.save())
    assert np.array_equal(b.bond_dims(), grown)
    a.step(p.dt, 2)
    b.step(p.dt, 2)
    pa = np.concatenate(a.populations(p.obs_leaves))
    pb = np.concatenate(b.populations(p.obs_leaves))
    assert np.array_equal(pa, pb)
    a.close(); b.close()
