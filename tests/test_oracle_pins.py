"""Pins of the CPU oracle against things it does not compute itself: dense
brute force on tiny trees, exact state-vector propagation, LAPACK, SciPy's
matrix exponential, conservation laws, convergence order and closed forms."""
import numpy as np
import pytest
import scipy.linalg
import scipy.integrate

import workloads as W
from oracle import exact, heom
from oracle.ttn import TTN, full_state, householder_qr, expm_krylov, mode_product, qr_along


def random_canonical(tree, rng):
    """Random tensors in canonical gauge, centre at the root."""
    A = []
    for z in range(tree.n):
        dims = tree.mode_dims(z)
        M = rng.standard_normal((int(np.prod(dims[:-1])), dims[-1])) \
            + 1j * rng.standard_normal((int(np.prod(dims[:-1])), dims[-1]))
        if z > 0:
            M, _ = np.linalg.qr(M)
        else:
            M = M / np.linalg.norm(M)
        A.append(M.reshape(dims))
    return A


def random_sop(tree, rng, n_terms=7, max_factors=3, hermitian=False):
    H = W.SOP(hermitian=hermitian)
    leaves = tree.leaves()
    for _ in range(n_terms):
        k = rng.integers(1, max_factors + 1)
        ls = rng.choice(leaves, size=min(k, len(leaves)), replace=False)
        pairs = []
        for l in ls:
            d = int(tree.phys_dim[l])
            pairs.append((int(l), rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))))
        H.add(complex(rng.standard_normal(), rng.standard_normal()), *pairs)
    H.add(0.7)   # a constant term
    return H


def small_tree():
    spec = ("node", 1, [
        ("node", 3, [("leaf", 2, 2, "s"), ("leaf", 3, 3, "m1")]),
        ("leaf", 3, 3, "m2"),
        ("node", 4, [("leaf", 2, 2, "m3"), ("node", 3, [("leaf", 2, 2, "m4"), ("leaf", 3, 2, "m5")])]),
    ])
    return W.build_tree(spec)


def embedding(tree, A, z):
    """Columns: full state vectors obtained with A^z replaced by unit tensors."""
    dims = tree.mode_dims(z)
    S = int(np.prod(dims))
    cols = []
    for i in range(S):
        B = [a.copy() for a in A]
        e = np.zeros(S, dtype=np.complex128); e[i] = 1.0
        B[z] = e.reshape(dims)
        cols.append(full_state(tree, B))
    return np.stack(cols, axis=1)


def move_centre_to(s, target):
    """Walk the orthogonality centre from the root down to ``target``
    (building down-environments on the way)."""
    path = []
    u = target
    while u > 0:
        path.append(u); u = s.t.parent[u]
    for c in reversed(path):
        z = s.t.parent[c]
        s._move_down(z, s.ch[z].index(c))


# ---------------------------------------------------------------------------
def test_heff_matches_dense_projection():
    """Eq. psi_eom_1: H_eff at every node equals P^dag H P with P the map from
    node coefficients to the full state (other nodes isometric)."""
    rng = np.random.default_rng(0)
    t = small_tree()
    H = random_sop(t, rng)
    Hd = exact.full_hamiltonian(t, H, dense=True)
    for target in range(t.n):
        s = TTN(t, H, random_canonical(t, rng))
        move_centre_to(s, target)
        P = embedding(t, s.A, target)
        assert np.allclose(P.conj().T @ P, np.eye(P.shape[1]), atol=1e-12)
        dense = P.conj().T @ Hd @ P
        dims = t.mode_dims(target)
        S = int(np.prod(dims))
        mine = np.zeros((S, S), dtype=np.complex128)
        for i in range(S):
            e = np.zeros(S, dtype=np.complex128); e[i] = 1.0
            mine[:, i] = s.heff(target, e.reshape(dims)).ravel()
        assert np.abs(mine - dense).max() <= 1e-12 * max(1.0, np.abs(dense).max())


def test_environments_from_explicit_basis_functions():
    """Sec. II.C: h_r^z = <Phi^z|h_r|Phi^z>, H_r^z = <Psi^z|H_r|Psi^z> with the
    SPF / SHF basis vectors written out on the full space."""
    rng = np.random.default_rng(1)
    t = small_tree()
    H = random_sop(t, rng, n_terms=5)
    leaves = t.leaves()
    dims = [int(t.phys_dim[l]) for l in leaves]
    for target in [3, 5, 7]:
        s = TTN(t, H, random_canonical(t, rng))
        move_centre_to(s, target)
        Pz = embedding(t, s.A, target)      # columns: |Psi_i> (x) |Phi_I>
        zd = t.mode_dims(target)
        N = zd[-1]
        sub = set(t.subtree_leaves(target))
        for r in range(H.n_terms):
            fac = {l: H.mats[m] for (l, m) in H.factors[r]}
            def op(inside):
                M = np.eye(1)
                for l, d in zip(leaves, dims):
                    X = fac[l] if (l in fac and ((l in sub) == inside)) else np.eye(d)
                    M = np.kron(M, X)
                return M
            Hin, Hout = op(True), op(False)
            # SHF block: sum over the SPF multi-index I of the projected matrix
            Pr = Pz.reshape(-1, int(np.prod(zd[:-1])), N)
            if s.outside[target, r]:
                dense = np.einsum("xIi,xy,yIj->ij", Pr.conj(), Hout, Pr) / np.prod(zd[:-1])
                assert np.allclose(s.down[target][r], dense, atol=1e-12)
            # SPF matrix of a child of the target node (its up environment)
            for k, c in enumerate(s.ch[target]):
                if s.inside[c, r]:
                    subc = set(t.subtree_leaves(c))
                    Mc = np.eye(1)
                    for l, d in zip(leaves, dims):
                        X = fac[l] if (l in fac and l in subc) else np.eye(d)
                        Mc = np.kron(Mc, X)
                    Pk = np.moveaxis(Pz.reshape((-1,) + tuple(zd)), k + 1, -1)
                    Pk = Pk.reshape(Pk.shape[0], -1, zd[k])
                    dense = np.einsum("xOi,xy,yOj->ij", Pk.conj(), Mc, Pk) / (np.prod(zd) // zd[k])
                    assert np.allclose(s.up[c][r], dense, atol=1e-12)


def test_householder_qr_matches_lapack_up_to_phases():
    rng = np.random.default_rng(2)
    for (m, n) in [(7, 3), (16, 16), (40, 5), (6144 // 64, 16)]:
        M = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
        Q, R = householder_qr(M)
        assert np.allclose(Q @ R, M, atol=1e-13 * np.abs(M).max() * m)
        assert np.allclose(Q.conj().T @ Q, np.eye(n), atol=1e-13)
        assert np.all(np.abs(np.tril(R, -1)) == 0)
        assert np.all(np.diag(R).real >= 0) and np.allclose(np.diag(R).imag, 0)
        Ql, Rl = np.linalg.qr(M)
        ph = np.diag(Rl) / np.abs(np.diag(Rl))
        assert np.allclose(Q, Ql * ph[None, :], atol=1e-12)
        assert np.allclose(R, Rl * ph.conj()[:, None], atol=1e-12 * np.abs(M).max())


def test_householder_qr_rank_deficient():
    """Zero columns get the identity reflector: Q stays orthonormal, M = QR,
    and the product-state matricisation gives the leading unit vectors."""
    rng = np.random.default_rng(3)
    M = np.zeros((12, 4), dtype=np.complex128)
    M[0, 0] = 1.0
    Q, R = householder_qr(M)
    assert np.array_equal(Q, np.eye(12, 4))
    # a remainder below the rank threshold is dropped: the column of Q is the
    # deterministic completion, and the dropped part is below tol * ||M||_F
    M[5, 2] = 1e-12
    Q, R = householder_qr(M, tol=1e-10)
    assert np.array_equal(Q, np.eye(12, 4))
    assert np.abs(Q @ R - M).max() <= 1e-10
    B = rng.standard_normal((12, 2)) + 1j * rng.standard_normal((12, 2))
    M = np.concatenate([B, B @ np.array([[1.0, 2.0], [0.5, -1.0]])], axis=1)
    Q, R = householder_qr(M)
    assert np.allclose(Q.conj().T @ Q, np.eye(4), atol=1e-13)
    assert np.allclose(Q @ R, M, atol=1e-12)


def test_mode_product_definition():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5))
    M = rng.standard_normal((4, 4))
    ref = np.zeros_like(A)
    for a in range(3):
        for p in range(4):
            for b in range(5):
                ref[a, p, b] = sum(M[p, m] * A[a, m, b] for m in range(4))
    assert np.allclose(mode_product(M, A, 1), ref)
    Q, R = qr_along(A, 1)
    assert np.allclose(mode_product(R.T, Q, 1), A)


@pytest.mark.parametrize("hermitian", [True, False])
def test_krylov_exponential_matches_expm(hermitian):
    rng = np.random.default_rng(5 + hermitian)
    n = 60
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Hm = (X + X.conj().T) / 2 if hermitian else X / 3
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for tau in [0.01, 0.3, 2.0]:
        w = expm_krylov(lambda x: Hm @ x, v, tau, hermitian)
        ref = scipy.linalg.expm(-1j * tau * Hm) @ v
        assert np.abs(w - ref).max() <= 1e-11 * np.linalg.norm(v) * max(1, np.abs(ref).max())
        if hermitian:
            assert abs(np.linalg.norm(w) - np.linalg.norm(v)) < 1e-12 * np.linalg.norm(v)


def test_full_bond_dimension_is_exact():
    """With bond dimensions equal to min(subtree, complement) the TTN manifold
    is the whole space and the splitting step reproduces exact propagation."""
    p = W.config_c1(full_bonds=True, d=4)
    s = TTN(p.tree, p.H, p.tensors)
    psi0 = full_state(p.tree, s.A)
    Hd = exact.full_hamiltonian(p.tree, p.H, dense=True)
    n = 40
    ref = exact.propagate_eigh(Hd, psi0, [p.dt * (i + 1) for i in range(n)])
    worst = 0.0
    for i in range(n):
        s.step(p.dt)
        po = s.populations(p.obs_leaves)
        pr = exact.leaf_populations(p.tree, ref[i], p.obs_leaves)
        worst = max(worst, max(np.abs(a - b).max() for a, b in zip(po, pr)))
    assert worst <= 1e-11


def test_rank_threshold_removes_rounding_sensitivity():
    """Treating QR remainders below 1e-10 ||M||_F as exact zeros makes the
    trajectory insensitive to rounding-level perturbations of the state."""
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    def run(pert):
        A = [a.copy() for a in p.tensors]
        rng = np.random.default_rng(1)
        A[0] = A[0] + pert * (rng.standard_normal(A[0].shape) + 1j * rng.standard_normal(A[0].shape))
        s = TTN(p.tree, p.H, A)
        s.step(p.dt, 3)
        return np.concatenate(s.populations(p.obs_leaves))
    assert np.abs(run(1e-16) - run(0.0)).max() < 1e-12


def test_norm_and_energy_conserved_truncated():
    p = W.config_c1()
    s = TTN(p.tree, p.H, p.tensors)
    n0, e0 = s.norm2(), s.energy()
    s.step(p.dt, 60)
    assert abs(s.norm2() - n0) <= 1e-11
    assert abs(s.energy() - e0) <= 1e-11


def test_second_order_convergence():
    p = W.config_c1(d=6)
    def run(dt, T=4.0):
        s = TTN(p.tree, p.H, p.tensors)
        s.step(dt, int(round(T / dt)))
        return full_state(p.tree, s.A)
    ref = run(0.4 / 32)
    e = [np.linalg.norm(run(dt) - ref) for dt in (0.4, 0.2, 0.1)]
    for a, b in zip(e, e[1:]):
        assert 3.5 < a / b < 4.6


def test_uncoupled_spin_closed_form():
    eps, delta = 0.3, 1.0
    p = W.config_c1(g_scale=0.0, eps=eps, delta=delta)
    s = TTN(p.tree, p.H, p.tensors)
    Om = np.hypot(eps, delta)
    spin = p.meta["spin"]
    for i in range(1, 41):
        s.step(p.dt)
        pop = s.populations([spin])[0]
        t = i * p.dt
        assert abs((pop[0] - pop[1]) - (eps ** 2 + delta ** 2 * np.cos(Om * t)) / Om ** 2) < 1e-11


def test_free_oscillator_closed_form():
    """Uncoupled modes in a superposition: <a>(t) = <a>(0) exp(-i w t)."""
    p = W.config_c1(g_scale=0.0)
    t = p.tree
    rng = np.random.default_rng(7)
    vecs = {}
    for l in p.meta["modes"]:
        v = rng.standard_normal(8) + 1j * rng.standard_normal(8)
        vecs[l] = v / np.linalg.norm(v)
    A = W.product_state(t, vecs)
    s = TTN(t, p.H, A)
    a = W.boson_ops(8)["a"]
    a0 = {l: np.vdot(vecs[l], a @ vecs[l]) for l in vecs}
    for i in range(1, 21):
        s.step(p.dt)
        G = s.shf_gram()
        for k, l in enumerate(p.meta["modes"]):
            rho = s.reduced_density(l, G)
            val = np.trace(rho @ a) / np.trace(rho)     # Tr(rho a)
            assert abs(val - a0[l] * np.exp(-1j * p.meta["w"][k] * i * p.dt)) < 1e-11


def test_independent_boson_decoherence():
    """Delta = 0 from |+x> (x) vacuum: <sx>(t) = prod_k exp(-4 (g_k/w_k)^2 (1 - cos w_k t))
    (untruncated Fock space; here compared within the truncation error), and
    exactly against same-basis diagonalisation at full bond dimension."""
    d = 12
    p = W.config_c1(full_bonds=True, d=d, delta=0.0, g_scale=0.3)
    t = p.tree
    spin = p.meta["spin"]
    v = np.array([1.0, 1.0], dtype=np.complex128) / np.sqrt(2)
    A = W.product_state(t, {spin: v})
    s = TTN(t, p.H, A)
    w, g = p.meta["w"], p.meta["g"]
    sx = W.pauli()["x"]
    for i in range(1, 11):
        s.step(p.dt)
        tt = i * p.dt
        rho = s.reduced_density(spin)
        val = np.real(np.trace(rho @ sx) / np.trace(rho))
        cf = np.prod(np.exp(-4 * (g / w) ** 2 * (1 - np.cos(w * tt))))
        assert abs(val - cf) < 1e-9


def test_reduced_density_gauge_walk_matches_full_state():
    rng = np.random.default_rng(8)
    t = small_tree()
    H = random_sop(t, rng)
    s = TTN(t, H, random_canonical(t, rng))
    psi = full_state(t, s.A)
    leaves = t.leaves()
    dims = [int(t.phys_dim[l]) for l in leaves]
    G = s.shf_gram()
    for l in leaves:
        ref = exact.leaf_reduced_density(psi, dims, leaves.index(l))
        assert np.allclose(s.reduced_density(l, G), ref, atol=1e-13)


def test_vacuum_projection_matches_full_state():
    rng = np.random.default_rng(9)
    t = small_tree()
    H = random_sop(t, rng)
    s = TTN(t, H, random_canonical(t, rng))
    psi = full_state(t, s.A)
    leaves = t.leaves()
    dims = [int(t.phys_dim[l]) for l in leaves]
    for keep in leaves:
        T = psi.reshape(dims)
        idx = tuple(slice(None) if l == keep else 0 for l in leaves)
        assert np.allclose(s.vacuum_projection(keep), T[idx], atol=1e-13)


@pytest.mark.parametrize("Km,depth", [(0, 4), (1, 3)])
def test_heom_ttn_matches_elementwise_hierarchy(Km, depth):
    """The operator-form generator on a full-bond TTN reproduces rho_S from the
    hierarchy assembled element by element from SI Eq. fpheom_SM_rescaled."""
    p = W.config_c4(K_matsubara=Km, depth=depth, chi=1000, dt=0.02)
    s = TTN(p.tree, p.H, p.tensors)
    n = 30
    ts = [p.dt * (i + 1) for i in range(n)]
    rho0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    ref = heom.rho_system(p.meta["Hs"], W.pauli()["z"], p.meta["alpha"], p.meta["nu"], depth, rho0, ts)
    for i in range(n):
        s.step(p.dt)
        r = s.vacuum_projection(p.meta["sys"]).reshape(2, 2)
        assert np.abs(r - ref[i]).max() < 1e-11
        assert abs(np.trace(ref[i]) - 1) < 1e-12


def test_heom_pure_dephasing_closed_form():
    al, nu = W.drude_lorentz_exponentials(0.1, 5.0, 1.0, 1)
    ts = np.linspace(0.1, 2.0, 5)
    rho0 = 0.5 * np.ones((2, 2), dtype=np.complex128)
    ref = heom.rho_system(np.zeros((2, 2)), W.pauli()["z"], al, nu, 6, rho0, ts)
    cf = heom.pure_dephasing_coherence(al, nu, ts)
    for i in range(len(ts)):
        assert abs(ref[i][0, 1] / 0.5 - cf[i]) < 1e-10


def test_orthopol_discretisation_is_a_gauss_rule():
    """Sec. II.E.1: the n-point rule integrates w^k J(w) exactly for k <= 2n-1."""
    J = W.ohmic_J(0.5, 5.0)
    n = 6
    w, g = W.discretise_orthopol(J, 0.0, 50.0, n)
    for k in range(2 * n):
        ref = scipy.integrate.quad(lambda x: x ** k * J(x), 0.0, 50.0, limit=200)[0]
        got = np.sum(np.pi * g ** 2 * w ** k)
        assert abs(got - ref) <= 1e-9 * abs(ref)


def test_product_state_is_canonical():
    for p in [W.config_c1(), W.config_c2(), W.config_c4()]:
        for z in range(1, p.tree.n):
            A = p.tensors[z]
            M = A.reshape(-1, A.shape[-1])
            assert np.array_equal(M.conj().T @ M, np.eye(M.shape[1]))
        assert np.linalg.norm(p.tensors[0]) == 1.0


# ---------------------------------------------------------------------------
# Subspace expansion (Sec. II.D)
# ---------------------------------------------------------------------------
def test_two_site_action_matches_dense_projection():
    """G[J, Theta] = <Phi_J (x) Theta| H |Psi> built from explicit basis vectors."""
    from oracle.ttn import ExpandingTTN
    rng = np.random.default_rng(21)
    t = small_tree()
    H = random_sop(t, rng, n_terms=6)
    s = ExpandingTTN(t, H, random_canonical(t, rng))
    Hd = exact.full_hamiltonian(s.t, H, dense=True)
    for target in [0, 1, 4]:
        move_centre_to(s, target)
        for k, c in enumerate(s.ch[target]):
            T, G = s.two_site_action(target, k)
            # embedding of the two-site tensor into the full space
            cols = []
            for i in range(T.size):
                e = np.zeros(T.size, dtype=np.complex128); e[i] = 1.0
                E = e.reshape(T.shape)
                B = [a.copy() for a in s.A]
                nc = s.A[c].ndim - 1
                # write the two-site unit tensor back as A^c = identity-like, A^z = E
                Jdims = s.A[c].shape[:-1]
                NJ = int(np.prod(Jdims))
                B[c] = np.eye(NJ, dtype=np.complex128).reshape(Jdims + (NJ,))
                Ez = E.reshape((NJ,) + T.shape[nc:])
                B[target] = np.moveaxis(Ez, 0, k)
                tt = copy_tree_with_bond(s.t, c, NJ)
                cols.append(full_state(tt, B))
            P = np.stack(cols, axis=1)
            dense = (P.conj().T @ Hd @ full_state(s.t, s.A)).reshape(T.shape)
            assert np.abs(dense - G).max() <= 1e-12 * max(1.0, np.abs(G).max())


def copy_tree_with_bond(t, c, b):
    import copy
    tt = copy.deepcopy(t)
    tt.bond_dim[c] = b
    return tt


def test_expansion_leaves_state_unchanged_and_full_bonds_accept_nothing():
    from oracle.ttn import ExpandingTTN
    p = W.config_c1(chi=2, d=4)
    s = ExpandingTTN(p.tree, p.H, p.tensors)
    s.step(p.dt, 3)
    psi0 = full_state(s.t, s.A)
    added = s.expand_pass(p.dt, 1e-6, 4)
    assert added > 0
    psi1 = full_state(s.t, s.A)
    assert np.abs(psi0 - psi1).max() <= 1e-13
    f = W.config_c1(full_bonds=True, d=4)
    s2 = ExpandingTTN(f.tree, f.H, f.tensors)
    s2.step(f.dt, 2)
    assert s2.expand_pass(f.dt, 1e-12, 64) == 0


def test_spawned_vectors_are_dominant_singular_vectors_of_variance():
    """The accepted directions maximise the captured error: the spawned SPF
    span equals the span of the top left singular vectors of (1-P) G (1-P_S)
    built here from explicit projectors."""
    from oracle.ttn import ExpandingTTN, qr_along
    p = W.config_c1(chi=2, d=4)
    s = ExpandingTTN(p.tree, p.H, p.tensors)
    s.step(p.dt, 4)
    z, k = 1, 1                     # node L and its mode leaf (both sides of dimension 4)
    move_centre_to(s, z)
    c = s.ch[z][k]
    _, G = s.two_site_action(z, k)
    Ac = s.A[c]
    NJ = int(np.prod(Ac.shape[:-1]))
    Gm = G.reshape(NJ, -1)
    M = Ac.reshape(NJ, -1)
    Pc = np.eye(NJ) - M @ M.conj().T
    Qs, _ = qr_along(s.A[z], k)
    Q = np.moveaxis(Qs, k, -1).reshape(Gm.shape[1], -1)
    PS = np.eye(Gm.shape[1]) - Q.conj() @ Q.T
    Y = Pc @ Gm @ PS
    lam, V = np.linalg.eigh(Y @ Y.conj().T)
    top = V[:, np.argsort(lam)[::-1][:1]]
    chi = M.shape[1]
    assert s.spawn_spf(z, k, p.dt, 1e-9, chi + 1) == 1
    new = s.A[c].reshape(NJ, -1)[:, chi:]
    assert abs(abs(np.vdot(top[:, 0], new[:, 0])) - 1.0) < 1e-10


def test_adaptive_expansion_improves_accuracy():
    """Starting from a product state with chi = 2 (a local metric cannot grow
    a bond whose other side is already complete, hence not chi = 1), spawning
    approaches the exact dynamics much more closely than the fixed-chi run."""
    from oracle.ttn import ExpandingTTN
    p = W.config_c1(chi=2, d=4)
    full = W.config_c1(full_bonds=True, d=4)
    psi0 = full_state(full.tree, full.tensors)
    Hd = exact.full_hamiltonian(full.tree, full.H, dense=True)
    n = 30
    ref = exact.propagate_eigh(Hd, psi0, [p.dt * n])[0]
    want = np.concatenate(exact.leaf_populations(full.tree, ref, full.obs_leaves))
    fixed = TTN(p.tree, p.H, p.tensors)
    fixed.step(p.dt, n)
    adapt = ExpandingTTN(p.tree, p.H, p.tensors)
    adapt.step_adaptive(p.dt, 1e-7, 16, n)
    e_fixed = np.abs(np.concatenate(fixed.populations(p.obs_leaves)) - want).max()
    e_adapt = np.abs(np.concatenate(adapt.populations(p.obs_leaves)) - want).max()
    assert max(adapt.t.bond_dim[1:]) > 2
    assert e_adapt < 0.25 * e_fixed


# ---------------------------------------------------------------------------
# one-site ground-state sweeps (tree DMRG)
# ---------------------------------------------------------------------------
def test_ground_state_full_bonds_is_exact():
    """At full bond dimension the root's effective Hamiltonian is the whole
    Hamiltonian in a rotated basis, so one sweep ends at the exact ground
    energy (dense diagonalisation of the 512-dim spin-boson H)."""
    p = W.config_c1(full_bonds=True, d=4)
    e0 = np.linalg.eigvalsh(exact.full_hamiltonian(p.tree, p.H).toarray())[0]
    ref = TTN(p.tree, p.H, p.tensors)
    es = ref.ground_state(2)
    assert abs(es[-1] - e0) <= 1e-10 * max(1.0, abs(e0))
    assert abs(ref.energy().real - e0) <= 1e-10 * max(1.0, abs(e0))


def test_ground_state_variational_and_monotone():
    """Truncated bonds (chi = 4): energies never increase from sweep to sweep,
    stay above the exact ground energy (sparse Lanczos on the 8192-dim H),
    and equal <Psi|H|Psi> of the normalised state."""
    import scipy.sparse.linalg as spla
    p = W.config_c1()
    Hs = exact.full_hamiltonian(p.tree, p.H)
    e0 = spla.eigsh(Hs, k=1, which="SA", tol=1e-12, v0=np.ones(Hs.shape[0]))[0][0]
    rng = np.random.default_rng(3)
    ref = TTN(p.tree, p.H, random_canonical(p.tree, rng))
    es = ref.ground_state(4)
    for a, b in zip(es, es[1:]):
        assert b <= a + 1e-12
    assert es[-1] >= e0 - 1e-10
    assert es[-1] - e0 <= 0.05 * abs(e0)        # a good variational estimate already
    n2 = ref.norm2()
    assert abs(n2 - 1.0) <= 1e-12
    assert abs(ref.energy().real - es[-1]) <= 1e-10


def test_ground_state_uncoupled_is_product_of_local_minima():
    """Without couplings the ground energy is the sum of the local minima."""
    t = small_tree()
    rng = np.random.default_rng(5)
    H = W.SOP(hermitian=True)
    want = 0.0
    for l in t.leaves():
        d = int(t.phys_dim[l])
        X = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        h = X + X.conj().T
        H.add(1.0, (l, h))
        want += np.linalg.eigvalsh(h)[0]
    ref = TTN(t, H, random_canonical(t, rng))
    es = ref.ground_state(2)
    assert abs(es[-1] - want) <= 1e-10 * max(1.0, abs(want))


# ---------------------------------------------------------------------------
# time-dependent coefficients
# ---------------------------------------------------------------------------
def driven_bias(p, omega):
    """c(t) schedule: the spin's sigma_z coefficient times cos(omega t)."""
    spin = p.meta["spin"]
    r0 = next(r for r, f in enumerate(p.H.factors)
              if len(f) == 1 and f[0][0] == spin and np.allclose(np.diag(p.H.mats[f[0][1]]), [1, -1]))
    base = np.array(p.H.coeffs, dtype=np.complex128)

    def coeffs(t):
        c = base.copy()
        c[r0] = base[r0] * np.cos(omega * t)
        return c
    return coeffs, r0


def test_time_dependent_coefficients_midpoint_order_two():
    """Uncoupled driven spin: the splitting is exact, so the midpoint rule
    c(t + dt/2) is the only error; it falls by ~4 when dt halves, against a
    tight ODE solution of the two-level Schrodinger equation."""
    import scipy.integrate
    p = W.config_c1(eps=1.0, g_scale=0.0)
    spin = p.meta["spin"]
    coeffs, r0 = driven_bias(p, 1.3)
    sx_c = next(c for c, f in zip(p.H.coeffs, p.H.factors)
                if len(f) == 1 and f[0][0] == spin and np.allclose(np.diag(p.H.mats[f[0][1]]), 0))
    sz = np.diag([1.0, -1.0]).astype(complex)
    sx = np.array([[0, 1], [1, 0]], dtype=complex)
    T = 2.0
    sol = scipy.integrate.solve_ivp(
        lambda t, y: -1j * ((coeffs(t)[r0] * sz + sx_c * sx) @ y), (0.0, T),
        np.array([1.0, 0.0], dtype=complex), method="DOP853", rtol=1e-12, atol=1e-12)
    psi = sol.y[:, -1]
    want = abs(psi[0]) ** 2 - abs(psi[1]) ** 2
    errs = []
    for n in (20, 40):
        dt = T / n
        ref = TTN(p.tree, p.H, p.tensors)
        for i in range(n):
            ref.set_coefficients(coeffs((i + 0.5) * dt))
            ref.step(dt)
        pop = ref.populations([spin])[0]
        errs.append(abs((pop[0] - pop[1]) - want))
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_constant_coefficients_change_nothing():
    p = W.config_c1(eps=1.0)
    a = TTN(p.tree, p.H, p.tensors)
    b = TTN(p.tree, p.H, p.tensors)
    for _ in range(3):
        b.set_coefficients(list(p.H.coeffs))
        a.step(p.dt)
        b.step(p.dt)
    for x, y in zip(a.A, b.A):
        assert np.array_equal(x, y)


def test_ground_eigensolver_branches_agree():
    """heff_lowest uses ARPACK above 600 elements: on such a node it gives
    the lowest eigenpair of the dense H_eff formed column by column."""
    p = W.config_c2(bonds=(8, 6, 4, 3), d_range=(4, 6))
    ref = TTN(p.tree, p.H, random_canonical(p.tree, np.random.default_rng(8)))
    sizes = [a.size for a in ref.A]
    z = next(i for i, n in enumerate(sizes) if 600 < n <= 5000)
    # bring the centre to z by one partial sweep: the root's children first
    path = []
    u = z
    while u != 0:
        path.append(u)
        u = p.tree.parent[u]
    for c in reversed(path):
        par = p.tree.parent[c]
        ref._move_down(par, ref.ch[par].index(c))
    e, v = ref.heff_lowest(z)
    shape = ref.A[z].shape
    n = ref.A[z].size
    M = np.empty((n, n), dtype=np.complex128)
    for i in range(n):
        x = np.zeros(n, dtype=np.complex128)
        x[i] = 1.0
        M[:, i] = ref.heff(z, x.reshape(shape)).ravel()
    w, V = np.linalg.eigh(M)
    assert abs(e - w[0]) <= 1e-10 * max(1.0, abs(w[0]))
    assert abs(abs(np.vdot(V[:, 0], v.ravel())) - 1.0) <= 1e-8
    assert w[1] - w[0] > 1e-6                     # non-degenerate, so the vector is unique


def test_sparse_propagation_matches_eigh_at_uneven_times():
    p = W.config_c1(full_bonds=True, d=4)
    Hs = exact.full_hamiltonian(p.tree, p.H)
    psi0 = full_state(p.tree, p.tensors)
    times = [0.1, 0.35, 1.0, 1.05]
    a = exact.propagate_sparse(Hs, psi0, times)
    b = exact.propagate_eigh(Hs.toarray(), psi0, times)
    for x, y in zip(a, b):
        assert np.linalg.norm(x - y) <= 1e-10


def test_vibronic_sop_is_the_model_formula():
    """The shared vibronic generator against its formula written out with
    Kronecker products: sum w_i (n_i + 1/2) - delta sz + sum kappa_i^s |s><s| Q_i
    + sum gamma_j^s |s><s| Q_j^2 + sum lam_j sx Q_j, Q = (a + a^+)/sqrt 2."""
    t = W.build_tree(("node", 1, [("leaf", 2, 2, "el"), ("leaf", 3, 3, "m0"), ("leaf", 4, 4, "m1")]))
    el, m0, m1 = (t.leaf_of_label(x) for x in ("el", "m0", "m1"))
    d = [3, 4]
    rng = np.random.default_rng(12)
    omega = rng.uniform(0.05, 0.5, 2)
    kappa = rng.normal(0, 0.05, (2, 2))
    gq = rng.normal(0, 0.01, (1, 2))
    lam = rng.normal(0, 0.05, 1)
    H = W.vibronic_sop(el, [m0, m1], d, omega, kappa, gq, [1], lam, [0], 0.1)
    got = exact.full_hamiltonian(t, H).toarray()

    def Q(n):
        a = np.diag(np.sqrt(np.arange(1, n)), 1)
        return (a + a.T) / np.sqrt(2.0)
    I2, I3, I4 = np.eye(2), np.eye(3), np.eye(4)
    P = [np.diag([1.0, 0.0]), np.diag([0.0, 1.0])]
    sz, sx = np.diag([1.0, -1.0]), np.array([[0.0, 1.0], [1.0, 0.0]])
    k3 = lambda A, B, C: np.kron(np.kron(A, B), C)
    want = (omega[0] * k3(I2, np.diag(np.arange(3) + 0.5), I4)
            + omega[1] * k3(I2, I3, np.diag(np.arange(4) + 0.5))
            - 0.1 * k3(sz, I3, I4))
    for s in range(2):
        want = want + kappa[0, s] * k3(P[s], Q(3), I4) + kappa[1, s] * k3(P[s], I3, Q(4))
        want = want + gq[0, s] * k3(P[s], I3, Q(4) @ Q(4))
    want = want + lam[0] * k3(sx, Q(3), I4)
    assert np.abs(got - want).max() <= 1e-14


def test_spin_boson_sop_is_the_model_formula():
    """The shared spin-boson generator against eps/2 sz + delta/2 sx
    + sz sum_k g_k (a_k + a_k^+) + sum_k w_k n_k written with Kronecker
    products (basis |0> = up)."""
    t = W.build_tree(("node", 1, [("leaf", 2, 2, "s"), ("leaf", 3, 3, "b0"), ("leaf", 4, 4, "b1")]))
    s, b0, b1 = (t.leaf_of_label(x) for x in ("s", "b0", "b1"))
    g, w = [0.3, -0.2], [0.7, 1.9]
    H = W.spin_boson_sop(s, [b0, b1], [3, 4], 0.4, 1.1, g, w)
    got = exact.full_hamiltonian(t, H).toarray()

    def ops(n):
        a = np.diag(np.sqrt(np.arange(1, n)), 1)
        return a + a.T, np.diag(np.arange(n, dtype=float))
    (x3, n3), (x4, n4) = ops(3), ops(4)
    sz, sx = np.diag([1.0, -1.0]), np.array([[0.0, 1.0], [1.0, 0.0]])
    I2, I3, I4 = np.eye(2), np.eye(3), np.eye(4)
    k3 = lambda A, B, C: np.kron(np.kron(A, B), C)
    want = (0.2 * k3(sz, I3, I4) + 0.55 * k3(sx, I3, I4)
            + g[0] * k3(sz, x3, I4) + g[1] * k3(sz, I3, x4)
            + w[0] * k3(I2, n3, I4) + w[1] * k3(I2, I3, n4))
    assert np.abs(got - want).max() <= 1e-14
