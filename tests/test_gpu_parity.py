"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

FP64 mode: populations (diagonals of every leaf's reduced density matrix)
agree to 1e-10; full states agree up to the gauge, so they are compared after
contraction.  Mixed mode: populations agree to 1e-6."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN, full_state
from oracle import exact

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


def gpu_ctx(ttn, p, precision, tensors=None):
    ctx = ttn.Context(p.tree, precision)
    ctx.set_state(p.tensors if tensors is None else tensors)
    ctx.set_hamiltonian(p.H)
    return ctx


def pops(obj, leaves):
    return np.concatenate(obj.populations(leaves))


def compare_trajectory(ttn, p, nsteps, every, precision, tol, tensors=None):
    ctx = gpu_ctx(ttn, p, precision, tensors)
    ref = TTN(p.tree, p.H, p.tensors if tensors is None else tensors)
    worst = 0.0
    for _ in range(0, nsteps, every):
        ctx.step(p.dt, every)
        ref.step(p.dt, every)
        worst = max(worst, float(np.abs(pops(ctx, p.obs_leaves) - pops(ref, p.obs_leaves)).max()))
    ctx.close()
    assert worst <= tol, f"max population error {worst:.3e} > {tol:.1e}"
    return worst


def test_c1_spin_boson_fp64_200_steps(gpu_lib):
    """Spin + 4 modes, chi = 4, 200 steps at dt = 0.05 (the full run)."""
    compare_trajectory(gpu_lib, W.config_c1(), 200, 20, gpu_lib.TTN_FP64, FP64_TOL)


def test_c1_full_bond_matches_exact_propagation(gpu_lib):
    p = W.config_c1(full_bonds=True, d=4)
    ctx = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    psi0 = full_state(p.tree, p.tensors)
    Hd = exact.full_hamiltonian(p.tree, p.H, dense=True)
    times = [p.dt * 5 * (i + 1) for i in range(8)]
    ref = exact.propagate_eigh(Hd, psi0, times)
    for i in range(8):
        ctx.step(p.dt, 5)
        want = np.concatenate(exact.leaf_populations(p.tree, ref[i], p.obs_leaves))
        assert np.abs(pops(ctx, p.obs_leaves) - want).max() <= 1e-10
        psi = full_state(p.tree, ctx.get_state())
        assert abs(abs(np.vdot(psi, ref[i])) - 1.0) <= 1e-10
    ctx.close()


def test_c2_vibronic_reduced_fp64(gpu_lib):
    """The 2 x 24 vibronic model on its ML tree with reduced bond and local
    dimensions so the oracle finishes in seconds."""
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    compare_trajectory(gpu_lib, p, 6, 2, gpu_lib.TTN_FP64, FP64_TOL)


def test_random_tree_non_hermitian_fp64(gpu_lib):
    """Arnoldi path: random complex SOP on an irregular tree; full states
    compared (gauge-invariant)."""
    from tests.test_oracle_pins import small_tree, random_sop, random_canonical
    rng = np.random.default_rng(11)
    t = small_tree()
    H = random_sop(t, rng, n_terms=9)
    A = random_canonical(t, rng)
    ctx = gpu_lib.Context(t, gpu_lib.TTN_FP64)
    ctx.set_state(A)
    ctx.set_hamiltonian(H)
    ref = TTN(t, H, A)
    for _ in range(4):
        ctx.step(0.02, 1)
        ref.step(0.02, 1)
        a, b = full_state(t, ctx.get_state()), full_state(t, ref.A)
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
    ctx.close()


def test_heom_vacuum_projection_fp64(gpu_lib):
    p = W.config_c4(K_matsubara=1, depth=3, chi=6, dt=0.02)
    ctx = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    ref = TTN(p.tree, p.H, p.tensors)
    for _ in range(5):
        ctx.step(p.dt, 2)
        ref.step(p.dt, 2)
        a = ctx.vacuum_projection(p.meta["sys"])
        b = ref.vacuum_projection(p.meta["sys"])
        assert np.abs(a - b).max() <= 1e-10
    ctx.close()


def test_norm_energy_conserved_fp64(gpu_lib):
    p = W.config_c1()
    ctx = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
    n0, e0 = ctx.norm_energy()
    ctx.step(p.dt, 100)
    n1, e1 = ctx.norm_energy()
    assert abs(n1 - n0) <= 1e-11 and abs(e1 - e0) <= 1e-11
    ctx.close()


def test_c1_mixed_precision_200_steps(gpu_lib):
    compare_trajectory(gpu_lib, W.config_c1(), 200, 20, gpu_lib.TTN_MIXED, MIXED_TOL)


def test_c2_reduced_mixed_precision(gpu_lib):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    compare_trajectory(gpu_lib, p, 10, 5, gpu_lib.TTN_MIXED, MIXED_TOL)


def test_batch_equals_individual(gpu_lib):
    """Instances with different trees and Hamiltonians in one launch give
    bit-identical results to running them one at a time."""
    probs = [W.config_c1(alpha=a) for a in (0.1, 0.3)] + [W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))]
    alone, batch = [], []
    for p in probs:
        c = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64)
        c.step(p.dt, 3)
        alone.append(c.get_state()); c.close()
    ctxs = [gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64) for p in probs]
    gpu_lib.ttn_step_batch([c.h for c in ctxs], 0.05, 3)
    for c in ctxs:
        batch.append(c.get_state()); c.close()
    # the vibronic instance used dt = 0.1 alone; rerun it alone at 0.05
    c = gpu_ctx(gpu_lib, probs[2], gpu_lib.TTN_FP64)
    c.step(0.05, 3)
    alone[2] = c.get_state(); c.close()
    for a, b in zip(alone, batch):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_invalid_hamiltonian_rejected(gpu_lib):
    p = W.config_c1()
    ctx = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    H = W.SOP()
    H.add(1.0, (0, np.eye(2)))          # node 0 is not a leaf
    with pytest.raises(gpu_lib.TTNError) as e:
        ctx.set_hamiltonian(H)
    assert e.value.status == gpu_lib.TTN_E_INVALID
    with pytest.raises(gpu_lib.TTNError) as e:
        ctx.step(0.1, 1)                # no Hamiltonian yet
    assert e.value.status == gpu_lib.TTN_E_STATE
    ctx.close()
