"""Parity at the full sizes of the benchmark configurations, on outputs the
oracle computes in about a minute: one or two steps of the complete problem
(not a reduced tree).  The 601-node spin-boson problem, whose oracle step
takes minutes, is checked by properties that hold at any size (norm and
energy conservation in complex128; mixed against complex128 on the GPU) and
against the oracle at a reduced mode count."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


def gpu_ctx(lib, p, precision):
    c = lib.Context(p.tree, precision)
    c.set_state(p.tensors)
    c.set_hamiltonian(p.H)
    return c


@pytest.fixture(scope="module")
def c4_oracle():
    p = W.config_c4()
    ref = TTN(p.tree, p.H, p.tensors)
    ref.step(p.dt, 1)
    return p, ref.vacuum_projection(p.meta["sys"])


def test_vibronic_2x24_full_size_two_steps(gpu_lib):
    """The benchmark's 46-node vibronic model (bonds 24/16/12/8, d 10..30)."""
    p = W.config_c2()
    ref = TTN(p.tree, p.H, p.tensors)
    ref.step(p.dt, 2)
    want = np.concatenate(ref.populations(p.obs_leaves))
    for precision, tol in ((gpu_lib.TTN_FP64, FP64_TOL), (gpu_lib.TTN_MIXED, MIXED_TOL)):
        c = gpu_ctx(gpu_lib, p, precision)
        c.step(p.dt, 2)
        got = np.concatenate(c.populations(p.obs_leaves))
        c.close()
        assert np.abs(got - want).max() <= tol


def test_heom_k16_depth10_full_size_fp64(gpu_lib, c4_oracle):
    """HEOM generator (16 exponentials, depth 10, chi 24, Arnoldi)."""
    p, want = c4_oracle
    c = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    c.step(p.dt, 1)
    got = c.vacuum_projection(p.meta["sys"])
    c.close()
    assert np.abs(got - want).max() <= FP64_TOL


def test_heom_k16_depth10_full_size_mixed(gpu_lib, c4_oracle):
    p, want = c4_oracle
    c = gpu_ctx(gpu_lib, p, gpu_lib.TTN_MIXED)
    c.step(p.dt, 1)
    got = c.vacuum_projection(p.meta["sys"])
    c.close()
    assert np.abs(got - want).max() <= MIXED_TOL


def test_spin_boson_reduced_modes_vs_oracle(gpu_lib):
    """The 300-mode problem's construction (orthogonal-polynomial bath,
    d = 20, chi = 8) at 24 modes, where the oracle is quick."""
    p = W.spin_boson_star_problem(24, 20, 8, 0.1, dt=0.01)
    ref = TTN(p.tree, p.H, p.tensors)
    ref.step(p.dt, 3)
    want = np.concatenate(ref.populations(p.obs_leaves))
    c = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    c.step(p.dt, 3)
    got = np.concatenate(c.populations(p.obs_leaves))
    c.close()
    assert np.abs(got - want).max() <= FP64_TOL


def test_spin_boson_300_modes_invariants_and_mixed(gpu_lib):
    """Full size (601 nodes): complex128 conserves norm and energy, and the
    mixed form follows <sigma_z(t)> of the complex128 GPU path."""
    p = W.config_c3()
    spin = p.meta["spin"]
    sz = np.diag([1.0, -1.0]).astype(np.complex128)
    c64 = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    cmx = gpu_ctx(gpu_lib, p, gpu_lib.TTN_MIXED)
    n0, e0 = c64.norm_energy()
    worst = 0.0
    for _ in range(4):
        c64.step(p.dt, 5)
        cmx.step(p.dt, 5)
        a = np.real(np.trace(c64.rdm(spin) @ sz))
        b = np.real(np.trace(cmx.rdm(spin) @ sz))
        worst = max(worst, abs(a - b))
    n1, e1 = c64.norm_energy()
    c64.close()
    cmx.close()
    assert abs(n1 - n0) <= 1e-10 and abs(e1 - e0) <= 1e-9 * max(1.0, abs(e0))
    assert worst <= MIXED_TOL
