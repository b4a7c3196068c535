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


def many_channel_problem(seed=7):
    """A random Hermitian sum of products on root(L(l1, l2), R(r1, r2), s)
    whose bond to L carries ten distinct coupling channels: starting from
    bond dimension 2 the first growths of that bond accept more than 16
    single-particle functions at once (the cap is only chi_max, Sec. II.D)."""
    spec = ("node", 1, [("node", 2, [("leaf", 6, 6, "l1"), ("leaf", 6, 6, "l2")]),
                        ("node", 8, [("leaf", 6, 6, "r1"), ("leaf", 6, 6, "r2")]),
                        ("leaf", 4, 4, "s")])
    t = W.build_tree(spec)
    rng = np.random.default_rng(seed)

    def herm(d):
        X = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        return (X + X.conj().T) / 2

    z = {lab: t.leaf_of_label(lab) for lab in ("l1", "l2", "r1", "r2", "s")}
    H = W.SOP()
    for lab in z:
        H.add(1.0, (z[lab], herm(int(t.phys_dim[z[lab]]))))
    for a in range(10):
        H.add(0.3, (z["l1" if a % 2 == 0 else "l2"], herm(6)), (z["s"], herm(4)))
    for a in range(4):
        H.add(0.2, (z["r1"], herm(6)), (z["l2"], herm(6)))
    vecs = {}
    for lab in z:
        d = int(t.phys_dim[z[lab]])
        v = rng.normal(size=d) + 1j * rng.normal(size=d)
        vecs[z[lab]] = v / np.linalg.norm(v)
    return W.Problem("many_channels", t, H, W.product_state(t, vecs), 0.05, 3, sorted(z.values()), {})


def _largest_growth(gpu_lib, p, nsteps, eps, chi_max, precision):
    ctx = gpu_lib.Context(p.tree, precision)
    ctx.set_state(p.tensors)
    ctx.set_hamiltonian(p.H)
    ref = ExpandingTTN(p.tree, p.H, p.tensors)
    opts = gpu_lib.ttn_step_opts(expand=1, eps_spawn=eps, chi_max=chi_max)
    prev, jump, worst = np.array(p.tree.bond_dim), 0, 0.0
    for _ in range(nsteps):
        ref.step_adaptive(p.dt, eps, chi_max, 1)
        ctx.step(p.dt, 1, opts)
        bd = ctx.bond_dims()
        assert np.array_equal(bd[1:], ref.t.bond_dim[1:]), (bd, ref.t.bond_dim)
        jump = max(jump, int((bd - prev).max()))
        prev = bd
        a = np.concatenate(ctx.populations(p.obs_leaves))
        b = np.concatenate(ref.populations(p.obs_leaves))
        worst = max(worst, float(np.abs(a - b).max()))
    ctx.close()
    return jump, worst


def _oracle_floor(p, nsteps, eps, chi_max):
    """The oracle's own response to 1e-15 perturbations of the initial
    tensors (two seeds): with many functions entering unoccupied at once, the
    one-site dynamics of the unoccupied directions is set by rounding, so no
    implementation can agree with the oracle better than this."""
    def run(pert, seed):
        rng = np.random.default_rng(seed)
        A = [a + pert * (rng.normal(size=a.shape) + 1j * rng.normal(size=a.shape)) for a in p.tensors]
        r = ExpandingTTN(p.tree, p.H, A)
        out = []
        for _ in range(nsteps):
            r.step_adaptive(p.dt, eps, chi_max, 1)
            out.append(np.concatenate(r.populations(p.obs_leaves)))
        return out
    base = run(0.0, 0)
    return max(float(np.abs(x - y).max()) for s in (0, 1) for x, y in zip(base, run(1e-15, s)))


@pytest.fixture(scope="module")
def many_channel_floor():
    return _oracle_floor(many_channel_problem(), 3, 1e-6, 32)


@pytest.fixture(scope="module")
def many_channel_floor_mixed():
    return _oracle_floor(many_channel_problem(), 3, 3e-5, 32)


def test_expansion_growth_above_16_fp64(gpu_lib, many_channel_floor):
    """Identical bond trajectories (one growth adds more than 16 functions);
    populations within 20 x the oracle's rounding floor on this case
    (measured 6e-9 .. 5e-8), never looser than needed elsewhere (1e-10)."""
    jump, worst = _largest_growth(gpu_lib, many_channel_problem(), 3, 1e-6, 32, gpu_lib.TTN_FP64)
    assert jump > 16
    assert worst <= max(1e-10, 20.0 * many_channel_floor)


def test_expansion_growth_above_16_mixed(gpu_lib, many_channel_floor_mixed):
    """Complex64 contractions resolve eigenvalues of the spawning operator
    down to about 1e-6 of the largest; at eps 3e-5 the growth of 17 functions
    has its smallest accepted eigenvalue at 3.2e-6 of the largest and its
    first rejected one 8 % below the threshold in sigma, so the decisions
    are clear of both the threshold and the complex64 floor and the bond
    trajectory is the oracle's.  Populations: the new functions enter
    unoccupied, so (as for complex128) the bar is 20 x the oracle's own
    response to 1e-15 perturbations (3e-8 .. 1.3e-7 here), never below the
    mixed form's 1e-6."""
    jump, worst = _largest_growth(gpu_lib, many_channel_problem(), 3, 3e-5, 32, gpu_lib.TTN_MIXED)
    assert jump > 16
    assert worst <= max(1e-6, 20.0 * many_channel_floor_mixed)
