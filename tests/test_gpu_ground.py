"""GPU one-site ground-state sweeps (ttn_ground_state) against the oracle's
sweep with dense / ARPACK eigen-solves.  Starting states are random
canonical tensors (seeded), whose effective Hamiltonians have
non-degenerate lowest eigenvalues, so the eigenvectors are unique up to
phase and populations can be compared.

Tolerances: complex128 eigen-solves stop at a relative residual of 1e-12,
so energies agree to 1e-10 and eigenvectors to ~1e-12 / gap.  The mixed
form stops at 1e-7 (complex64 Krylov basis), so its eigenvectors carry
~1e-7 / gap.  Before convergence the root energy depends to first order on
the isometries chosen below it, so early sweeps agree to ~1e-6 relative
(asserted at 1e-5); at convergence the energy is stationary and the error
is second order (asserted at 1e-6 relative); populations ~1e-7 / gap
(asserted at 1e-5)."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN
from oracle import exact
from tests.test_oracle_pins import random_canonical

pytestmark = pytest.mark.gpu


def run_pair(lib, p, A0, precision, nsweeps):
    ref = TTN(p.tree, p.H, A0)
    e_ref = np.array(ref.ground_state(nsweeps))
    ctx = lib.Context(p.tree, precision)
    ctx.set_state(A0)
    ctx.set_hamiltonian(p.H)
    e_gpu = ctx.ground_state(nsweeps)
    pops_gpu = np.concatenate(ctx.populations(p.obs_leaves))
    pops_ref = np.concatenate(ref.populations(p.obs_leaves))
    n2, en = ctx.norm_energy()
    ctx.close()
    return e_ref, e_gpu, pops_ref, pops_gpu, n2, en


def test_ground_state_spin_boson_fp64(gpu_lib):
    p = W.config_c1()
    A0 = random_canonical(p.tree, np.random.default_rng(3))
    e_ref, e_gpu, pr, pg, n2, en = run_pair(gpu_lib, p, A0, gpu_lib.TTN_FP64, 3)
    assert np.abs(e_gpu - e_ref).max() <= 1e-10
    assert np.abs(pg - pr).max() <= 1e-9
    assert abs(n2 - 1.0) <= 1e-12 and abs(en.real - e_gpu[-1]) <= 1e-10


def test_ground_state_full_bonds_exact_fp64(gpu_lib):
    p = W.config_c1(full_bonds=True, d=4)
    e0 = np.linalg.eigvalsh(exact.full_hamiltonian(p.tree, p.H).toarray())[0]
    ctx = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    ctx.set_state(p.tensors)
    ctx.set_hamiltonian(p.H)
    es = ctx.ground_state(2)
    ctx.close()
    assert abs(es[-1] - e0) <= 1e-10 * max(1.0, abs(e0))


def test_ground_state_vibronic_reduced_fp64(gpu_lib):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    A0 = random_canonical(p.tree, np.random.default_rng(4))
    e_ref, e_gpu, pr, pg, _, _ = run_pair(gpu_lib, p, A0, gpu_lib.TTN_FP64, 2)
    assert np.abs(e_gpu - e_ref).max() <= 1e-10
    assert np.abs(pg - pr).max() <= 1e-9


def test_ground_state_spin_boson_mixed(gpu_lib):
    p = W.config_c1()
    A0 = random_canonical(p.tree, np.random.default_rng(3))
    e_ref, e_gpu, pr, pg, _, _ = run_pair(gpu_lib, p, A0, gpu_lib.TTN_MIXED, 4)
    scale = np.abs(e_ref).max()
    assert np.abs(e_gpu - e_ref).max() <= 1e-5 * scale
    assert abs(e_gpu[-1] - e_ref[-1]) <= 1e-6 * scale
    assert np.abs(pg - pr).max() <= 1e-5


def test_ground_state_rejects_non_hermitian(gpu_lib):
    p = W.config_c4(K_matsubara=1, depth=3, chi=6, dt=0.02)
    ctx = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    ctx.set_state(p.tensors)
    ctx.set_hamiltonian(p.H)
    with pytest.raises(gpu_lib.TTNError) as e:
        ctx.ground_state(1)
    assert e.value.status == gpu_lib.TTN_E_INVALID
    ctx.close()
