"""Pins of the multi-set oracle (paper Sec. II.A, multi-set ansatz) against
results fixed by other means: exact propagation of the assembled multi-set
Hamiltonian at full bond dimension (where the projector-splitting step is
exact), the single-set oracle on every set when no term couples two sets,
norm and energy conservation at truncated bond dimension, and the closed-form
Rabi oscillation cos^2(J t) of a pure set coupling."""
import numpy as np
import pytest

import workloads as W
from oracle import exact
from oracle.multiset import MultiSetTTN
from oracle.ttn import TTN


def small_tree(full: bool):
    """root(l0 [d 2], X(l1 [d 3], l2 [d 2])): full bonds are exact."""
    if full:
        spec = ("node", 1, [("leaf", 2, 2, "l0"), ("node", 6, [("leaf", 3, 3, "l1"), ("leaf", 2, 2, "l2")])])
    else:
        spec = ("node", 1, [("leaf", 2, 2, "l0"), ("node", 2, [("leaf", 3, 2, "l1"), ("leaf", 2, 2, "l2")])])
    return W.build_tree(spec)


def coupled_sop(t, rng, S=3, hermitian=True, cross=True):
    """Per-set local and two-body terms that differ between sets, and (cross)
    set couplings: a constant and a non-symmetric one-leaf factor (with its
    adjoint on the transposed pair when Hermitian)."""
    lv = t.leaves()

    def herm(d):
        X = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        return (X + X.conj().T) / 2

    def gen(d):
        return rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))

    H = W.MultiSetSOP(hermitian=hermitian, n_sets=S)
    for a in range(S):
        H.add_set(a, a, 0.1 * a + (0.0 if hermitian else -0.05j))
        for l in lv:
            H.add_set(a, a, 0.5, (l, herm(int(t.phys_dim[l])) if hermitian else gen(int(t.phys_dim[l]))))
        H.add_set(a, a, 0.2, (lv[0], herm(2)), (lv[2], herm(2)))
    if cross:
        for a in range(S):
            for b in range(a + 1, S):
                c = 0.3 + 0.1j * (a + b)
                M = gen(3)
                if hermitian:
                    H.add_set(a, b, c); H.add_set(b, a, np.conj(c))
                    H.add_set(a, b, 0.2, (lv[1], M)); H.add_set(b, a, 0.2, (lv[1], M.conj().T))
                else:
                    H.add_set(a, b, c); H.add_set(b, a, 0.5 * c)
                    H.add_set(a, b, 0.2, (lv[1], M), (lv[2], herm(2))); H.add_set(b, a, -0.1, (lv[1], gen(3)))
    return H


def random_vecs(t, rng):
    out = {}
    for l in t.leaves():
        d = int(t.phys_dim[l])
        v = rng.normal(size=d) + 1j * rng.normal(size=d)
        out[l] = v / np.linalg.norm(v)
    return out


@pytest.mark.parametrize("occupied", ["first_set", "all_sets"])
def test_full_bonds_match_exact_propagation(occupied):
    rng = np.random.default_rng(3)
    t = small_tree(True)
    H = coupled_sop(t, rng)
    amps = [1.0, 0.0, 0.0] if occupied == "first_set" else [0.6, 0.48j, 0.64]
    A = W.multiset_product_state(t, amps, [random_vecs(t, rng) for _ in range(3)])
    o = MultiSetTTN(t, H, A)
    psi0 = o.full_state()
    Hd = exact.full_multiset_hamiltonian(t, H, dense=True)
    assert np.allclose(Hd, Hd.conj().T)
    dt, n = 0.05, 12
    o.step(dt, n)
    ref = exact.propagate_eigh(Hd, psi0, [n * dt])[0]
    np.testing.assert_allclose(o.full_state(), ref, atol=1e-11)
    # the empty sets were filled through the set couplings
    assert o.set_populations().min() > 1e-3


def test_full_bonds_non_hermitian_match_exact_propagation():
    rng = np.random.default_rng(5)
    t = small_tree(True)
    H = coupled_sop(t, rng, S=2, hermitian=False)
    A = W.multiset_product_state(t, [0.8, 0.6], [random_vecs(t, rng) for _ in range(2)])
    o = MultiSetTTN(t, H, A)
    psi0 = o.full_state()
    dt, n = 0.04, 10
    o.step(dt, n)
    ref = exact.propagate_sparse(exact.full_multiset_hamiltonian(t, H), psi0, [n * dt])[0]
    np.testing.assert_allclose(o.full_state(), ref, atol=1e-10)


def test_uncoupled_sets_evolve_as_single_set_ttns():
    """With no set coupling each set follows the single-set integrator under
    its own block H^{alpha alpha}; the gauge moves are per set, so the tensors
    agree entry by entry."""
    rng = np.random.default_rng(8)
    t = small_tree(False)
    S = 3
    H = coupled_sop(t, rng, S=S, cross=False)
    amps = [0.6, 0.0, 0.8]
    A = W.multiset_product_state(t, amps, [random_vecs(t, rng) for _ in range(S)])
    o = MultiSetTTN(t, H, A)
    dt, n = 0.05, 8
    o.step(dt, n)
    for a in range(S):
        Ha = W.SOP(hermitian=True)
        for c, fs, b, k in zip(H.coeffs, H.factors, H.bra, H.ket):
            if b == a:
                Ha.add(c, *[(l, H.mats[m]) for (l, m) in fs])
        s = TTN(t, Ha, A[a])
        s.step(dt, n)
        for z in range(t.n):
            np.testing.assert_allclose(o.A[a][z], s.A[z], atol=1e-11)
    np.testing.assert_allclose(o.set_populations(), np.abs(amps) ** 2, atol=1e-12)


def test_truncated_bonds_conserve_norm_and_energy():
    rng = np.random.default_rng(13)
    t = small_tree(False)
    H = coupled_sop(t, rng)
    A = W.multiset_product_state(t, [1.0, 0.0, 0.0], [random_vecs(t, rng) for _ in range(3)])
    o = MultiSetTTN(t, H, A)
    e0 = o.energy()
    o.step(0.05, 20)
    assert abs(o.norm2() - 1.0) < 1e-11
    assert abs(o.energy() - e0) < 1e-9
    # truncation matters here: the state is not the exact one
    psi0 = MultiSetTTN(t, H, A).full_state()
    ref = exact.propagate_eigh(exact.full_multiset_hamiltonian(t, H, dense=True), psi0, [1.0])[0]
    assert np.abs(o.full_state() - ref).max() > 1e-4


@pytest.mark.parametrize("local", [False, True])
def test_pure_set_coupling_rabi_closed_form(local):
    """H = J (|0><1| + |1><0|) (x) 1 [+ 1 (x) h]: the set populations are
    cos^2(J t) and sin^2(J t) at any bond dimension, from set 0 alone."""
    rng = np.random.default_rng(21)
    t = W.build_tree(("node", 1, [("leaf", 4, 2, "l0"), ("node", 2, [("leaf", 3, 2, "l1"), ("leaf", 5, 2, "l2")])]))
    J = 0.7
    H = W.MultiSetSOP(hermitian=True, n_sets=2)
    H.add_set(0, 1, J); H.add_set(1, 0, J)
    if local:
        for l in t.leaves():
            d = int(t.phys_dim[l]); X = rng.normal(size=(d, d)); X = X + X.T
            for a in range(2):
                H.add_set(a, a, 0.3, (l, X))
    v = random_vecs(t, rng)
    o = MultiSetTTN(t, H, W.multiset_product_state(t, [1.0, 0.0], [v, v]))
    for _ in range(40):
        o.step(0.05)
        p = o.set_populations()
        # Krylov tolerance 1e-13 per exponential, ~40 exponentials per step
        assert abs(p[0] - np.cos(J * o.t_elapsed) ** 2) < 1e-9
        assert abs(p[1] - np.sin(J * o.t_elapsed) ** 2) < 1e-9


def test_set_leaf_densities_trace_to_populations():
    rng = np.random.default_rng(4)
    t = small_tree(False)
    H = coupled_sop(t, rng)
    o = MultiSetTTN(t, H, W.multiset_product_state(t, [1.0, 0.0, 0.0], [random_vecs(t, rng) for _ in range(3)]))
    o.step(0.05, 5)
    pops = o.set_populations()
    for l in t.leaves():
        for a in range(3):
            rho = o.reduced_density(a, l)
            assert abs(np.trace(rho) - pops[a]) < 1e-12
            assert np.allclose(rho, rho.conj().T)


def test_model_problem_runs_and_conserves():
    p = W.multiset_vibronic_problem(n_states=3, n_modes=5, d=5, chi=3, nsteps=10)
    o = MultiSetTTN(p.tree, p.H, p.tensors)
    e0 = o.energy()
    o.step(p.dt, p.nsteps)
    assert abs(o.norm2() - 1.0) < 1e-11
    assert abs(o.energy() - e0) < 1e-9
    assert o.set_populations()[1:].sum() > 1e-4


@pytest.mark.parametrize("mistake", ["swap_bra_ket", "identity_not_overlap"])
def test_full_bond_pin_catches_planted_mistakes(mistake):
    """The exact-propagation pin fails when a plausible slip is planted in the
    oracle: the set pair of the coupling terms read the wrong way round, or
    the overlap of two sets' functions taken as the identity."""
    rng = np.random.default_rng(3)
    t = small_tree(True)
    H = coupled_sop(t, rng)
    A = W.multiset_product_state(t, [0.6, 0.48j, 0.64], [random_vecs(t, rng) for _ in range(3)])
    o = MultiSetTTN(t, H, A)
    psi0 = o.full_state()
    if mistake == "swap_bra_ket":
        o.bra, o.ket = o.ket, o.bra
    else:
        leaves_of = [set(t.subtree_leaves(z)) for z in range(t.n)]
        for r in range(H.n_terms):
            ls = set(o.fac[r])
            for z in range(t.n):
                o.inside[z, r] = len(ls & leaves_of[z]) > 0
                o.outside[z, r] = z > 0 and len(ls - leaves_of[z]) > 0
    for z in o.postorder():
        if z > 0:
            o.build_up(z)
    o.step(0.05, 12)
    ref = exact.propagate_eigh(exact.full_multiset_hamiltonian(t, H, dense=True), psi0, [0.6])[0]
    assert np.abs(o.full_state() - ref).max() > 1e-3


def test_empty_set_start_is_ill_conditioned_occupied_is_not():
    """Conditioning behind the GPU tests' choice of starts: a 1e-15
    perturbation of the top tensors moves populations after 5 steps by more
    than 1e-8 when two sets start empty (their functions come from QR of zero
    or nearly zero matrices) and by less than 1e-12 when every set is
    occupied."""
    def moved(amps):
        rng = np.random.default_rng(3)
        t = small_tree(False)
        H = coupled_sop(t, rng)
        A = W.multiset_product_state(t, amps, [random_vecs(t, rng) for _ in range(3)])
        Ap = [[a.copy() for a in As] for As in A]
        r = np.random.default_rng(5)
        for As in Ap:
            As[0] = As[0] + 1e-15 * (r.normal(size=As[0].shape) + 1j * r.normal(size=As[0].shape))
        o0, o1 = MultiSetTTN(t, H, A), MultiSetTTN(t, H, Ap)
        o0.step(0.05, 5)
        o1.step(0.05, 5)
        return np.abs(o0.set_populations() - o1.set_populations()).max()
    assert moved([1.0, 0.0, 0.0]) > 1e-8
    assert moved([0.6, 0.48j, 0.64]) < 1e-12
