"""GPU parity of multi-set states (paper Sec. II.A, multi-set ansatz): the
CUDA path through the C ABI against the multi-set oracle on the same seeded
inputs.  States are compared after contraction (the full multi-set vector,
which the gauge does not change) and by set populations; FP64 to 1e-10, the
complex64 bulk to 1e-6.  Also: exact propagation at full bond dimension,
the closed-form Rabi oscillation, the conversion of a single-set state, the
batched launch, and the calls a multi-set state refuses.

Element-wise parity runs from states where every set is occupied.  A start
with empty sets (zero top tensors) is ill-conditioned at truncated bond
dimension: the empty sets' single-particle functions come from QR of zero
or nearly zero matrices, and a 1e-15 perturbation of those top tensors
moves the oracle's own populations by ~7e-6 after 5 steps (1e-15 -> 6e-15
with every set occupied; tests/test_multiset_oracle.py pins both).  From
empty sets the tests check what is unique -- exact propagation at full bond
dimension, norm and energy conservation -- and that the state stays valid."""
import numpy as np
import pytest

import workloads as W
from oracle import exact
from oracle.multiset import MultiSetTTN
from oracle.ttn import full_state
from tests.test_multiset_oracle import coupled_sop, random_vecs, small_tree

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


def ctx_for(lib, tree, H, A, precision):
    c = lib.Context(tree, precision)
    c.set_multiset_hamiltonian(H)
    c.set_multiset_state(A)
    return c


def gpu_full(c, tree, S):
    return np.concatenate([full_state(tree, c.get_multiset_state(a)) for a in range(S)])


OCCUPIED = [0.6, 0.48j, 0.64]


def problems():
    """Every set occupied (well-conditioned, see the module docstring)."""
    rng = np.random.default_rng(3)
    t = small_tree(False)
    H = coupled_sop(t, rng)
    yield "random_3sets", t, H, W.multiset_product_state(t, OCCUPIED, [random_vecs(t, rng) for _ in range(3)]), 0.05
    p = W.multiset_vibronic_problem(n_states=3, n_modes=6, d=6, chi=4)
    yield p.name, p.tree, p.H, W.multiset_product_state(p.tree, OCCUPIED), p.dt


@pytest.mark.parametrize("case", [0, 1])
def test_multiset_fp64_matches_oracle(gpu_lib, case):
    name, t, H, A, dt = list(problems())[case]
    ref = MultiSetTTN(t, H, A)
    c = ctx_for(gpu_lib, t, H, A, gpu_lib.TTN_FP64)
    assert c.n_sets() == H.n_sets
    for _ in range(4):
        ref.step(dt, 5)
        c.step(dt, 5)
        np.testing.assert_allclose(c.set_populations(), ref.set_populations(), atol=FP64_TOL, err_msg=name)
        np.testing.assert_allclose(gpu_full(c, t, H.n_sets), ref.full_state(), atol=FP64_TOL, err_msg=name)
    n2, e = c.norm_energy()
    assert abs(n2 - ref.norm2()) <= 1e-11
    assert abs(e - ref.energy()) <= 1e-10 * max(1.0, abs(ref.energy()))
    c.close()


def test_multiset_mixed_matches_oracle(gpu_lib):
    name, t, H, A, dt = list(problems())[1]
    ref = MultiSetTTN(t, H, A)
    c = ctx_for(gpu_lib, t, H, A, gpu_lib.TTN_MIXED)
    for _ in range(4):
        ref.step(dt, 5)
        c.step(dt, 5)
        err = float(np.abs(c.set_populations() - ref.set_populations()).max())
        assert err <= MIXED_TOL, (name, err)
    c.close()


@pytest.mark.parametrize("amps", [OCCUPIED, [1.0, 0.0, 0.0]])
def test_multiset_full_bonds_match_exact_propagation(gpu_lib, amps):
    rng = np.random.default_rng(3)
    t = small_tree(True)
    H = coupled_sop(t, rng)
    A = W.multiset_product_state(t, amps, [random_vecs(t, rng) for _ in range(3)])
    psi0 = MultiSetTTN(t, H, A).full_state()
    Hd = exact.full_multiset_hamiltonian(t, H, dense=True)
    c = ctx_for(gpu_lib, t, H, A, gpu_lib.TTN_FP64)
    c.step(0.05, 12)
    want = exact.propagate_eigh(Hd, psi0, [0.6])[0]
    np.testing.assert_allclose(gpu_full(c, t, 3), want, atol=FP64_TOL)
    c.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_multiset_rabi_closed_form(gpu_lib, precision, tol):
    rng = np.random.default_rng(21)
    t = W.build_tree(("node", 1, [("leaf", 4, 2, "l0"), ("node", 2, [("leaf", 3, 2, "l1"), ("leaf", 5, 2, "l2")])]))
    J = 0.7
    H = W.MultiSetSOP(hermitian=True, n_sets=2)
    H.add_set(0, 1, J); H.add_set(1, 0, J)
    for l in t.leaves():
        d = int(t.phys_dim[l]); X = rng.normal(size=(d, d)); X = X + X.T
        for a in range(2):
            H.add_set(a, a, 0.3, (l, X))
    v = random_vecs(t, rng)
    c = ctx_for(gpu_lib, t, H, W.multiset_product_state(t, [1.0, 0.0], [v, v]), precision)
    for i in range(8):
        c.step(0.05, 5)
        tt = 0.25 * (i + 1)
        p = c.set_populations()
        assert abs(p[0] - np.cos(J * tt) ** 2) <= tol and abs(p[1] - np.sin(J * tt) ** 2) <= tol, (tt, p)
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_empty_sets_start_conserves_and_stays_valid(gpu_lib, precision):
    """The physical start of a multi-set run (one electronic state occupied):
    norm and energy conserved, every set's non-root tensors isometric, the
    empty sets filled through the couplings, and the oracle's populations
    matched to the start's conditioning (a loose bound)."""
    p = W.multiset_vibronic_problem(n_states=3, n_modes=6, d=6, chi=4)
    c = ctx_for(gpu_lib, p.tree, p.H, p.tensors, precision)
    n0, e0 = c.norm_energy()
    c.step(p.dt, 20)
    n1, e1 = c.norm_energy()
    tol = 1e-11 if precision == 0 else 1e-5
    assert abs(n1 - n0) <= tol and abs(e1 - e0) <= (1e-9 if precision == 0 else 1e-5) * max(1.0, abs(e0))
    for a in range(3):
        A = c.get_multiset_state(a)
        for z in range(1, p.tree.n):
            M = A[z].reshape(-1, A[z].shape[-1])
            np.testing.assert_allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-10 if precision == 0 else 1e-5)
    pops = c.set_populations()
    assert pops[1:].min() > 1e-6
    ref = MultiSetTTN(p.tree, p.H, p.tensors)
    ref.step(p.dt, 20)
    assert np.abs(pops - ref.set_populations()).max() <= 1e-4
    c.close()


def test_single_set_state_becomes_multiset(gpu_lib):
    """A single-set state given before the multi-set operator becomes set 0;
    the other sets start empty (set 0's isometries, zero top tensor)."""
    p = W.multiset_vibronic_problem(n_states=2, n_modes=4, d=5, chi=3)
    c = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    c.set_state(p.tensors[0])
    c.set_multiset_hamiltonian(p.H)
    np.testing.assert_allclose(c.set_populations(), [1.0, 0.0], atol=1e-14)
    A1 = c.get_multiset_state(1)
    assert np.abs(A1[0]).max() == 0.0
    for z in range(1, p.tree.n):
        np.testing.assert_array_equal(A1[z], p.tensors[0][z])
    ref = MultiSetTTN(p.tree, p.H, p.tensors)      # the same conversion (set 1 empty, set 0's isometries)
    ref.step(p.dt, 10)
    c.step(p.dt, 10)
    np.testing.assert_allclose(c.set_populations(), ref.set_populations(), atol=FP64_TOL)
    c.close()


def test_multiset_batch_equals_single_launches(gpu_lib):
    ps = [W.multiset_vibronic_problem(n_states=3, n_modes=5, d=5, chi=3, seed=s) for s in (1, 2, 3)]
    batch = [ctx_for(gpu_lib, p.tree, p.H, p.tensors, gpu_lib.TTN_FP64) for p in ps]
    single = [ctx_for(gpu_lib, p.tree, p.H, p.tensors, gpu_lib.TTN_FP64) for p in ps]
    gpu_lib.ttn_step_batch([c.h for c in batch], ps[0].dt, 6)
    for c, p in zip(single, ps):
        c.step(p.dt, 6)
    for a, b, p in zip(batch, single, ps):
        np.testing.assert_array_equal(gpu_full(a, p.tree, 3), gpu_full(b, p.tree, 3))
    for c in batch + single:
        c.close()


def test_multiset_refuses_single_set_calls(gpu_lib):
    p = W.multiset_vibronic_problem(n_states=2, n_modes=4, d=5, chi=3)
    c = ctx_for(gpu_lib, p.tree, p.H, p.tensors, gpu_lib.TTN_FP64)
    leaf = p.meta["modes"][0]
    for call in (lambda: c.rdm(leaf), lambda: c.ground_state(1),
                 lambda: c.set_state(p.tensors[0]), lambda: c.vacuum_projection(leaf),
                 lambda: c.step(p.dt, 1, {"expand": 1, "eps_spawn": 1e-6, "chi_max": 8})):
        with pytest.raises(gpu_lib.TTNError):
            call()
    c.step(p.dt, 2)                                   # still usable
    assert abs(c.set_populations().sum() - 1.0) < 1e-11
    c.close()


@pytest.mark.parametrize("blocks", [4])
def test_multiset_on_a_cluster_team_matches_oracle(gpu_lib, blocks):
    """The set blocks through the cluster team (row-split QR, dealt-out Gram
    tiles, DSMEM reductions) give the oracle's trajectory too."""
    name, t, H, A, dt = list(problems())[1]
    ref = MultiSetTTN(t, H, A)
    c = ctx_for(gpu_lib, t, H, A, gpu_lib.TTN_FP64)
    c.set_cluster(blocks)
    for _ in range(2):
        ref.step(dt, 5)
        c.step(dt, 5)
        np.testing.assert_allclose(gpu_full(c, t, H.n_sets), ref.full_state(), atol=FP64_TOL, err_msg=name)
    c.close()


def test_multiset_requests_through_the_server(gpu_lib):
    """Multi-set contexts served beside single-set ones give the tensors of
    the same contexts run alone with ttn_step."""
    ms = [W.multiset_vibronic_problem(n_states=3, n_modes=5, d=5, chi=3, seed=s, amps=OCCUPIED) for s in (1, 2)]
    ss = [W.vibronic_balanced_problem(6, 5, 3, seed=s, nsteps=6) for s in (3, 4)]
    steps = 6

    def fresh():
        out = [ctx_for(gpu_lib, p.tree, p.H, p.tensors, gpu_lib.TTN_MIXED) for p in ms]
        for p in ss:
            c = gpu_lib.Context(p.tree, gpu_lib.TTN_MIXED)
            c.set_state(p.tensors)
            c.set_hamiltonian(p.H)
            out.append(c)
        return out

    alone = fresh()
    for c, p in zip(alone, ms + ss):
        c.step(p.dt, steps)
    served = fresh()
    srv = gpu_lib.Server(gpu_lib.TTN_MIXED)
    for c, p in zip(served, ms + ss):
        srv.submit(c, p.dt, steps)
    srv.drain()
    for a, b, p in zip(alone[:2], served[:2], ms):
        np.testing.assert_array_equal(gpu_full(a, p.tree, 3), gpu_full(b, p.tree, 3))
    for a, b in zip(alone[2:], served[2:]):
        for x, y in zip(a.get_state(), b.get_state()):
            np.testing.assert_array_equal(x, y)
    srv.close()
    for c in alone + served:
        c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_multiset_checkpoint_resume_is_bit_identical(gpu_lib, precision):
    """Save a resident multi-set context mid-run, load it into a fresh
    context, and both continue with the same bits."""
    p = W.multiset_vibronic_problem(n_states=3, n_modes=5, d=5, chi=3, amps=OCCUPIED)
    a = ctx_for(gpu_lib, p.tree, p.H, p.tensors, precision)
    a.step(p.dt, 4)
    blob = a.save()
    other = W.config_c1()
    b = gpu_lib.Context(other.tree, precision)
    b.load(blob)
    assert b.n_sets() == 3
    a.step(p.dt, 4)
    b.step(p.dt, 4)
    np.testing.assert_array_equal(gpu_full(a, p.tree, 3), gpu_full(b, p.tree, 3))
    a.close()
    b.close()
