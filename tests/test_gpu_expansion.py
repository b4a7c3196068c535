"""GPU subspace expansion (paper Sec. II.D) against the oracle's dense
two-site implementation: same bond-dimension trajectory, same populations."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import ExpandingTTN, full_state

pytestmark = pytest.mark.gpu


def run_pair(gpu_lib, p, nsteps, eps, chi_max, precision):
    ctx = gpu_lib.Context(p.tree, precision)
    ctx.set_state(p.tensors)
    ctx.set_hamiltonian(p.H)
    ref = ExpandingTTN(p.tree, p.H, p.tensors)
    opts = gpu_lib.ttn_step_opts(expand=1, eps_spawn=eps, chi_max=chi_max)
    worst, grew = 0.0, False
    for _ in range(nsteps):
        ref.step_adaptive(p.dt, eps, chi_max, 1)
        ctx.step(p.dt, 1, opts)
        bd = ctx.bond_dims()
        assert np.array_equal(bd[1:], ref.t.bond_dim[1:]), (bd, ref.t.bond_dim)
        grew |= bool(np.any(bd[1:] > p.tree.bond_dim[1:]))
        a = np.concatenate(ctx.populations(p.obs_leaves))
        b = np.concatenate(ref.populations(p.obs_leaves))
        worst = max(worst, float(np.abs(a - b).max()))
    psi_gpu = full_state(ref.t, ctx.get_state()) if p.tree.n < 12 else None
    psi_ref = full_state(ref.t, ref.A) if p.tree.n < 12 else None
    ctx.close()
    return worst, grew, psi_gpu, psi_ref


def test_expansion_spin_boson_fp64(gpu_lib):
    p = W.config_c1(chi=2, d=4)
    worst, grew, a, b = run_pair(gpu_lib, p, 12, 1e-6, 6, gpu_lib.TTN_FP64)
    assert grew
    assert worst <= 1e-10
    assert abs(abs(np.vdot(a, b)) - np.linalg.norm(a) * np.linalg.norm(b)) <= 1e-10


def test_expansion_vibronic_reduced_fp64(gpu_lib):
    p = W.config_c2(bonds=(4, 3, 3, 2), d_range=(4, 6))
    worst, grew, _, _ = run_pair(gpu_lib, p, 4, 1e-5, 6, gpu_lib.TTN_FP64)
    assert grew
    assert worst <= 1e-10


def test_expansion_spin_boson_mixed(gpu_lib):
    p = W.config_c1(chi=2, d=4)
    worst, grew, _, _ = run_pair(gpu_lib, p, 12, 1e-6, 6, gpu_lib.TTN_MIXED)
    assert grew
    assert worst <= 1e-6
