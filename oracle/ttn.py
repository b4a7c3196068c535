"""Plain complex128 TTN projector-splitting integrator (test oracle).

State (paper Sec. II.A): node tensors A^z with shape [n_1..n_d, N] (children,
or the physical index of a leaf, then the parent bond; the root's N = 1).
Gauge: canonical, orthogonality centre at the root between steps (Sec. II.A,
"canonical gauge").

Hamiltonian (Sec. II.B.1, Eq. sop_ham): plain sum of products, one
environment matrix per (node, term), no grouping.  A term that does not act
inside the subtree of z has the identity as its single-particle operator
there; one that acts only inside has the identity as mean-field operator.

Effective equations (Sec. II.C, Eq. psi_eom_1 with hbar = 1):
    dA/dt = -i sum_r c_r (x_k h_r^(z,k)) A (H_r^z)^T
where h acts on the child indices and H_r^z[i, j] = <Psi_i|H_r^z|Psi_j> acts
on the parent index as sum_j H_r^z[i, j] A[.., j] (the printed "A H" read with
the transpose that makes it the matrix element ordering of Eq. for H_r^z).

Integrator: second-order recursive projector splitting, step(dt) =
S*(root, dt/2) o S(root, dt/2), children visited in index order by S and in
reverse order by S* (the paper defers the sweep to its Ref. lindoy_mctdh_2;
this is the standard recursive PSI of the works it cites in Sec. II.C).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

QR_TOL_FP64 = 1e-10   # rank threshold relative to ||M||_F (paper silent; see tests)
KRYLOV_TOL = 1e-13
KRYLOV_MAXDIM = 32


# ----------------------------------------------------------------------------
# Small dense building blocks
# ----------------------------------------------------------------------------
def mode_product(M: np.ndarray, A: np.ndarray, k: int) -> np.ndarray:
    """(M x_k A)[.., p, ..] = sum_m M[p, m] A[.., m, ..]."""
    return np.moveaxis(np.tensordot(M, A, axes=([1], [k])), 0, k)


def householder_qr(M: np.ndarray, tol: float = QR_TOL_FP64):
    """Householder QR of an m x n matrix with m >= n.

    Returns Q (m x n, orthonormal columns) and R (n x n upper triangular) with
    M = Q R and real non-negative diagonal of R.  Reflector j is the one that
    maps the remaining column x onto beta e_0 with beta = -sign(Re x_0) ||x||
    (then the sign is moved to Q); a column whose remainder has norm at most
    tol * ||M||_F is taken as zero and gets the identity reflector, so the
    corresponding column of Q is H_1 .. H_{j-1} e_j.
    """
    m, n = M.shape
    assert m >= n, "QR needs at least as many rows as columns"
    R = np.array(M, dtype=np.complex128, copy=True)
    thr = tol * np.linalg.norm(M)
    vs, taus = [], []
    for j in range(n):
        x = R[j:, j]
        nrm = np.linalg.norm(x)
        if nrm <= thr:
            vs.append(None); taus.append(0.0)
            R[j + 1:, j] = 0.0
            continue
        alpha = x[0]
        beta = -nrm if alpha.real >= 0 else nrm
        tau = (beta - alpha) / beta
        v = x / (alpha - beta)
        v[0] = 1.0
        R[j:, j:] -= np.conj(tau) * np.outer(v, v.conj() @ R[j:, j:])
        R[j, j] = beta
        R[j + 1:, j] = 0.0
        vs.append(v); taus.append(tau)
    Q = np.zeros((m, n), dtype=np.complex128)
    Q[np.arange(n), np.arange(n)] = 1.0
    for j in range(n - 1, -1, -1):
        if vs[j] is None:
            continue
        v = vs[j]
        Q[j:, :] -= taus[j] * np.outer(v, v.conj() @ Q[j:, :])
    R = np.triu(R[:n, :])
    for j in range(n):
        if vs[j] is not None and R[j, j].real < 0:
            R[j, :] *= -1.0
            Q[:, j] *= -1.0
    return Q, R


def qr_along(A: np.ndarray, k: int, tol: float = QR_TOL_FP64):
    """QR of tensor A matricised with index k as the column index:
    A = Q x_k R^T, Q with orthonormal 'columns' along index k."""
    Am = np.moveaxis(A, k, -1)
    sh = Am.shape
    Q, R = householder_qr(Am.reshape(-1, sh[-1]), tol)
    Q = np.moveaxis(Q.reshape(sh[:-1] + (Q.shape[1],)), -1, k)
    return Q, R


def expm_krylov(apply, v: np.ndarray, tau: float, hermitian: bool,
                tol: float = KRYLOV_TOL, maxdim: int = KRYLOV_MAXDIM, depth: int = 0):
    """w = exp(-i tau H) v by Lanczos (hermitian) or Arnoldi, with full
    re-orthogonalisation (two classical Gram-Schmidt passes) and the dense
    small exponential (eigh of the tridiagonal matrix, or expm of the upper
    Hessenberg matrix).  Stops when Saad's a-posteriori estimate
    beta * h_{m+1,m} * |e_m^T exp(-i tau H_m) e_1| <= tol * beta; if maxdim is
    reached first the interval is halved and the two halves are applied in
    turn."""
    beta0 = np.linalg.norm(v)
    if beta0 == 0.0:
        return v.copy()
    shape = v.shape
    V = [v.ravel() / beta0]
    Hm = np.zeros((maxdim + 1, maxdim), dtype=np.complex128)
    for j in range(maxdim):
        w = apply(V[j].reshape(shape)).ravel()
        for _ in range(2):
            for i in range(j + 1):
                h = np.vdot(V[i], w)
                Hm[i, j] += h
                w = w - h * V[i]
        if hermitian:
            # the projected matrix is real symmetric tridiagonal in exact arithmetic
            Hm[j, j] = Hm[j, j].real
            for i in range(j - 1):
                Hm[i, j] = 0.0
            if j > 0:
                Hm[j - 1, j] = Hm[j, j - 1]
        hnext = np.linalg.norm(w)
        Hm[j + 1, j] = hnext
        m = j + 1
        if hermitian:
            ev, U = np.linalg.eigh(Hm[:m, :m])
            y = U @ (np.exp(-1j * tau * ev) * U[0, :].conj())
        else:
            y = scipy.linalg.expm(-1j * tau * Hm[:m, :m])[:, 0]
        err = hnext * abs(y[m - 1])
        if err <= tol or hnext == 0.0:
            out = np.zeros_like(V[0])
            for i in range(m):
                out = out + y[i] * V[i]
            return (beta0 * out).reshape(shape)
        V.append(w / hnext)
    if depth > 20:
        raise RuntimeError("Krylov exponential did not converge")
    half = expm_krylov(apply, v, tau / 2.0, hermitian, tol, maxdim, depth + 1)
    return expm_krylov(apply, half, tau / 2.0, hermitian, tol, maxdim, depth + 1)


# ----------------------------------------------------------------------------
# TTN with a plain SOP Hamiltonian
# ----------------------------------------------------------------------------
class TTN:
    """Tree tensor network state plus per-term environments.

    ``tree`` is a workloads.Tree, ``H`` a workloads.SOP, ``A`` the list of node
    tensors (copied)."""

    def __init__(self, tree, H, A, qr_tol: float = QR_TOL_FP64,
                 krylov_tol: float = KRYLOV_TOL, krylov_maxdim: int = KRYLOV_MAXDIM):
        self.t = tree
        self.H = H
        self.A = [np.array(a, dtype=np.complex128, copy=True) for a in A]
        self.qr_tol = qr_tol
        self.ktol = krylov_tol
        self.kmax = krylov_maxdim
        n, R = tree.n, H.n_terms
        self.ch = [tree.children(z) for z in range(n)]
        # factor matrix of term r on leaf l, and where each term acts
        self.fac = [dict() for _ in range(R)]
        for r, fs in enumerate(H.factors):
            for (l, m) in fs:
                assert tree.is_leaf(l), "SOP factors must act on leaves"
                assert l not in self.fac[r], "one factor per leaf and term"
                self.fac[r][l] = H.mats[m]
        leaves_of = [set(tree.subtree_leaves(z)) for z in range(n)]
        self.inside = np.zeros((n, R), dtype=bool)   # term acts within subtree(z)
        self.outside = np.zeros((n, R), dtype=bool)  # term acts outside subtree(z)
        for r in range(R):
            ls = set(self.fac[r])
            for z in range(n):
                self.inside[z, r] = len(ls & leaves_of[z]) > 0
                self.outside[z, r] = len(ls - leaves_of[z]) > 0
        self.up = [dict() for _ in range(n)]     # h_r^z   (Sec. II.C, SPF operator matrices)
        self.down = [dict() for _ in range(n)]   # H_r^z   (Sec. II.C, mean-field matrices)
        for z in self.postorder():
            if z > 0:
                self.build_up(z)
        self.t_elapsed = 0.0

    # -- traversal -------------------------------------------------------------
    def postorder(self):
        out = []
        def rec(z):
            for c in self.ch[z]:
                rec(c)
            out.append(z)
        rec(0)
        return out

    # -- environments (Sec. II.B.1 Eqs. spf_hamiltonian_op / shf_hamiltonian_op,
    #    Sec. II.C matrix elements) ----------------------------------------------
    def _apply_child_ops(self, T, z, r, skip=None):
        """Apply term r's operators on the child indices of node z (leaf: the
        physical factor)."""
        if self.t.is_leaf(z):
            M = self.fac[r].get(z)
            if M is not None:
                T = mode_product(M, T, 0)
            return T
        for k, c in enumerate(self.ch[z]):
            if k == skip:
                continue
            if self.inside[c, r]:
                T = mode_product(self.up[c][r], T, k)
        return T

    def build_up(self, z):
        """h_r^z[i, i'] = <phi_i^z| h_r^z |phi_i'^z> for node z in isometric form
        towards its parent: A^dag (x_k h_r^(z,k)) A."""
        A = self.A[z]
        nd = A.ndim
        self.up[z] = {}
        for r in range(self.H.n_terms):
            if not self.inside[z, r]:
                continue
            T = self._apply_child_ops(A, z, r)
            self.up[z][r] = np.tensordot(A.conj(), T, axes=(list(range(nd - 1)), list(range(nd - 1))))

    def build_down(self, z, k):
        """Mean-field matrices of child c = children(z)[k] from Q = A^z in
        isometric form towards c:
        H_r^c[n, n'] = sum conj(Q[I;n, i]) (x_{j!=k} h_r^(z,j))_{I I'} H_r^z[i, i'] Q[I';n', i']."""
        c = self.ch[z][k]
        Q = self.A[z]
        nd = Q.ndim
        axes = [a for a in range(nd) if a != k]
        self.down[c] = {}
        for r in range(self.H.n_terms):
            if not self.outside[c, r]:
                continue
            T = self._apply_child_ops(Q, z, r, skip=k)
            if self.outside[z, r]:
                T = mode_product(self.down[z][r], T, nd - 1)
            self.down[c][r] = np.tensordot(Q.conj(), T, axes=(axes, axes))

    # -- effective operators --------------------------------------------------
    def heff(self, z, A):
        """sum_r c_r (x_k h_r^(z,k)) A (H_r^z)^T  (Eq. psi_eom_1 without -i)."""
        out = np.zeros_like(A)
        nd = A.ndim
        for r, cr in enumerate(self.H.coeffs):
            T = self._apply_child_ops(A, z, r)
            if self.outside[z, r]:
                T = mode_product(self.down[z][r], T, nd - 1)
            out += cr * T
        return out

    def kbond(self, c, C):
        """Bond operator on C[n, m] (n: SPF index of c, m: its SHF index):
        sum_r c_r h_r^c C (H_r^c)^T."""
        out = np.zeros_like(C)
        for r, cr in enumerate(self.H.coeffs):
            T = C
            if self.inside[c, r]:
                T = self.up[c][r] @ T
            if self.outside[c, r]:
                T = T @ self.down[c][r].T
            out += cr * T
        return out

    def _evolve_node(self, z, tau):
        self.A[z] = expm_krylov(lambda x: self.heff(z, x), self.A[z], tau,
                                self.H.hermitian, self.ktol, self.kmax)

    def _evolve_bond_back(self, c, C, tau):
        return expm_krylov(lambda x: self.kbond(c, x), C, -tau,
                           self.H.hermitian, self.ktol, self.kmax)

    # -- projector-splitting sweep --------------------------------------------
    def _move_down(self, z, k):
        """Centre z -> child k: A^z = Q x_k R^T, A^c <- A^c R^T."""
        c = self.ch[z][k]
        Q, R = qr_along(self.A[z], k, self.qr_tol)
        self.A[z] = Q
        self.A[c] = mode_product(R, self.A[c], self.A[c].ndim - 1)
        self.build_down(z, k)

    def _move_up(self, z, k):
        """Centre child k -> z: A^c = Q' R' (R' is the bond matrix C[n, m])."""
        c = self.ch[z][k]
        Ac = self.A[c]
        Q, R = qr_along(Ac, Ac.ndim - 1, self.qr_tol)
        self.A[c] = Q
        self.build_up(c)
        return R

    def sweep_S(self, z, tau):
        for k, c in enumerate(self.ch[z]):
            self._move_down(z, k)
            self.sweep_S(c, tau)
            C = self._move_up(z, k)
            C = self._evolve_bond_back(c, C, tau)
            self.A[z] = mode_product(C, self.A[z], k)
        self._evolve_node(z, tau)

    def sweep_Sstar(self, z, tau):
        self._evolve_node(z, tau)
        for k in range(len(self.ch[z]) - 1, -1, -1):
            c = self.ch[z][k]
            Q, R = qr_along(self.A[z], k, self.qr_tol)
            self.A[z] = Q
            self.build_down(z, k)
            C = R.T                      # C[n, m]: n SPF index of c, m SHF index
            C = self._evolve_bond_back(c, C, tau)
            self.A[c] = mode_product(C.T, self.A[c], self.A[c].ndim - 1)
            self.sweep_Sstar(c, tau)
            Cup = self._move_up(z, k)
            self.A[z] = mode_product(Cup, self.A[z], k)

    def step(self, dt: float, nsteps: int = 1):
        """step(dt) = S*(root, dt/2) o S(root, dt/2)."""
        for _ in range(nsteps):
            self.sweep_S(0, dt / 2.0)
            self.sweep_Sstar(0, dt / 2.0)
            self.t_elapsed += dt

    def set_coefficients(self, coeffs):
        """Time-dependent SOP coefficients c_r(t) (Sec. II.E: the bath
        mappings make them time dependent): the environments here are per
        term and carry no coefficient, so replacing c_r is all there is."""
        import dataclasses
        assert len(coeffs) == self.H.n_terms
        self.H = dataclasses.replace(self.H, coeffs=[complex(c) for c in coeffs])

    # -- one-site ground-state sweep (tree DMRG) --------------------------------
    # The paper names DMRG beside the time evolution (Sec. I, Sec. II.C): the
    # same environments, effective Hamiltonian and gauge moves, with each node
    # tensor replaced by the lowest eigenvector of its effective Hamiltonian
    # instead of being propagated.
    def heff_lowest(self, z):
        """Lowest eigenpair of H_eff^z (Hermitian): dense eigh of the matrix
        formed column by column for small nodes, ARPACK Lanczos (started from
        the current tensor) otherwise."""
        shape = self.A[z].shape
        n = int(np.prod(shape))
        if n <= 600:
            M = np.empty((n, n), dtype=np.complex128)
            for i in range(n):
                e = np.zeros(n, dtype=np.complex128)
                e[i] = 1.0
                M[:, i] = self.heff(z, e.reshape(shape)).ravel()
            w, V = np.linalg.eigh(M)
            return float(w[0]), V[:, 0].reshape(shape)
        import scipy.sparse.linalg as spla
        op = spla.LinearOperator((n, n), dtype=np.complex128,
                                 matvec=lambda v: self.heff(z, v.reshape(shape)).ravel())
        w, V = spla.eigsh(op, k=1, which="SA", tol=1e-14, v0=self.A[z].ravel().copy())
        v = V[:, 0]
        return float(w[0]), (v / np.linalg.norm(v)).reshape(shape)

    def sweep_ground(self, z):
        """Visiting order of S: centre to each child by QR, recursion, centre
        back (no bond step), then A^z <- lowest eigenvector of H_eff^z.
        Returns the eigenvalue found at z."""
        for k, c in enumerate(self.ch[z]):
            self._move_down(z, k)
            self.sweep_ground(c)
            C = self._move_up(z, k)
            self.A[z] = mode_product(C, self.A[z], k)
        e, self.A[z] = self.heff_lowest(z)
        return e

    def ground_state(self, nsweeps: int = 1):
        """Energies (root eigenvalue) after each of nsweeps sweeps."""
        return [self.sweep_ground(0) for _ in range(nsweeps)]

    # -- observables -----------------------------------------------------------
    def shf_gram(self):
        """G^z[m', m] = <Psi_m'^z | Psi_m^z> for every node with the centre at the
        root (Eq. shf_recursive_definition); G^root = [[1]]."""
        G = [None] * self.t.n
        G[0] = np.ones((1, 1), dtype=np.complex128)
        for z in range(self.t.n):
            A = self.A[z]
            nd = A.ndim
            for k, c in enumerate(self.ch[z]):
                axes = [a for a in range(nd) if a != k]
                T = mode_product(G[z], A, nd - 1)     # T[.., m'] = sum_m G[m', m] A[.., m]
                G[c] = np.tensordot(A.conj(), T, axes=(axes, axes))
        return G

    def reduced_density(self, leaf, G=None):
        """rho[a, a'] = sum_{i,i'} A[a, i] conj(A[a', i']) <Psi_i'|Psi_i>."""
        G = self.shf_gram() if G is None else G
        A = self.A[leaf]
        return A @ G[leaf].T @ A.conj().T

    def norm2(self):
        return float(np.vdot(self.A[0], self.A[0]).real)

    def energy(self):
        """<Psi|H|Psi> / <Psi|Psi> with the centre at the root."""
        return complex(np.vdot(self.A[0], self.heff(0, self.A[0])) / self.norm2())

    def populations(self, leaves):
        G = self.shf_gram()
        out = []
        for l in leaves:
            rho = self.reduced_density(l, G)
            out.append(np.real(np.diag(rho)) / np.real(np.trace(rho)))
        return out

    def vacuum_projection(self, keep_leaf):
        """Contract every leaf except ``keep_leaf`` with the basis vector e_0 and
        return the remaining vector on keep_leaf's physical index (HEOM:
        rho_S = <0_bath|rho), paper SI Sec. S2)."""
        t = self.t
        vec = [None] * t.n
        keep_path = set()
        u = keep_leaf
        while u >= 0:
            keep_path.add(u); u = t.parent[u]
        for z in reversed(range(t.n)):
            A = self.A[z]
            if t.is_leaf(z):
                vec[z] = A if z == keep_leaf else A[0, :]
                continue
            T = A
            # contract children not on the kept path (from the last index down)
            kept_axis = None
            for k in range(len(self.ch[z]) - 1, -1, -1):
                c = self.ch[z][k]
                if c in keep_path:
                    kept_axis = k
                    continue
                T = np.tensordot(vec[c], T, axes=([0], [k]))  # removes axis k
            if kept_axis is not None:
                c = self.ch[z][kept_axis]
                # T now has axes [n_kept, N]; vec[c] has axes [d, n_kept]
                T = np.tensordot(vec[c], T, axes=([1], [0]))  # [d, N]
            vec[z] = T
        return vec[0][..., 0]


# ----------------------------------------------------------------------------
# Full state vectors (small trees only)
# ----------------------------------------------------------------------------
def full_state(tree, A):
    """Contract the whole TTN into a dense vector over the leaves in increasing
    node order (row-major)."""
    def rec(z):
        if tree.is_leaf(z):
            return A[z], [z]                           # [d, N]
        T = A[z]
        leaves = []
        # replace child index k by the child's leaves, left to right
        pieces = []
        for c in tree.children(z):
            Tc, lc = rec(c)
            pieces.append((Tc, lc))
        # contract in order; keep track of axes
        cur = T
        off = 0
        for (Tc, lc) in pieces:
            nl = len(lc)
            cur = np.tensordot(Tc, cur, axes=([Tc.ndim - 1], [off]))  # [leaves.., rest]
            # move the new leaf axes to position off
            cur = np.moveaxis(cur, list(range(nl)), list(range(off, off + nl)))
            off += nl
            leaves += lc
        return cur, leaves
    T, leaves = rec(0)
    perm = np.argsort(leaves)
    T = T[..., 0]
    T = np.transpose(T, perm)
    return T.reshape(-1)


# ----------------------------------------------------------------------------
# Subspace expansion (paper Sec. II.D): spawning of single-particle functions
# ----------------------------------------------------------------------------
class ExpandingTTN(TTN):
    """TTN with bond-dimension expansion by the two-site energy variance.

    With the orthogonality centre at z, the bond to child c = children(z)[k]
    is expanded by the dominant left singular vectors u of
        Y = (1 - P_c) G (1 - P_S),
    where G[J, Theta] = <Phi^c_J (x) Theta| H |Psi> is the two-site projection
    of H Psi onto c's children-product basis J and the orthonormal basis Theta
    of everything outside c, P_c = A^c A^c^dag projects onto c's current SPFs
    and P_S onto c's single-hole functions (the columns of the QR of A^z
    along k); Y Y^dag is the operator Delta^(z,k) of Sec. II.D.  A vector is
    added when dt * sqrt(lambda) >= eps (Sec. II.D spawning criterion with
    c = dt), at most up to chi_max and the sizes of the two sides; the new
    columns are appended to A^c and A^z is zero-padded along k, which leaves
    Psi unchanged.  Dense "full approach" (Sec. III.B).

    One expansion pass visits the bonds in sweep order (children in index
    order, centre moved by QR); at the first bond that accepts vectors it
    expands, moves the centre back to the root and starts over, until a
    pass accepts nothing."""

    def __init__(self, tree, H, A, **kw):
        import copy
        tree = copy.deepcopy(tree)
        super().__init__(tree, H, A, **kw)
        self.spawn_log = []

    def two_site_action(self, z, k):
        """Two-site tensor T = A^c x_last,k A^z and G = H_two-site T (plain SOP,
        per-term environments).  Axes: c's child indices, then z's indices
        without k (other children in order, then the parent)."""
        c = self.ch[z][k]
        Ac, Az = self.A[c], self.A[z]
        nc = Ac.ndim - 1
        T = np.tensordot(Ac, Az, axes=([nc], [k]))
        zmodes = [j for j in range(Az.ndim) if j != k]
        G = np.zeros_like(T)
        for r, cr in enumerate(self.H.coeffs):
            X = T
            if self.t.is_leaf(c):
                M = self.fac[r].get(c)
                if M is not None:
                    X = mode_product(M, X, 0)
            else:
                for j, cj in enumerate(self.ch[c]):
                    if self.inside[cj, r]:
                        X = mode_product(self.up[cj][r], X, j)
            for pos, j in enumerate(zmodes):
                ax = nc + pos
                if j == Az.ndim - 1:
                    if self.outside[z, r]:
                        X = mode_product(self.down[z][r], X, ax)
                else:
                    cj = self.ch[z][j]
                    if self.inside[cj, r]:
                        X = mode_product(self.up[cj][r], X, ax)
            G += cr * X
        return T, G

    def spawn_spf(self, z, k, dt, eps, chi_max):
        c = self.ch[z][k]
        chi = int(self.t.bond_dim[c])
        _, G = self.two_site_action(z, k)
        Ac = self.A[c]
        NJ = int(np.prod(Ac.shape[:-1]))
        NT = G.size // NJ
        cap = min(chi_max, NJ, NT) - chi
        if cap <= 0:
            return 0
        Gm = G.reshape(NJ, NT)
        Mm = Ac.reshape(NJ, chi)
        Qs, _ = qr_along(self.A[z], k, self.qr_tol)
        Qm = np.moveaxis(Qs, k, -1).reshape(NT, chi)
        Y = Gm - Mm @ (Mm.conj().T @ Gm)
        Y = Y - (Y @ Qm.conj()) @ Qm.T
        U, s, _ = np.linalg.svd(Y, full_matrices=False)
        acc = [i for i in range(len(s)) if dt * s[i] >= eps][:cap]
        self.spawn_log.append((z, k, s[: min(len(s), cap + 2)].copy()))
        p = len(acc)
        if p == 0:
            return 0
        newM = np.concatenate([Mm, U[:, acc]], axis=1)
        self.A[c] = newM.reshape(Ac.shape[:-1] + (chi + p,))
        Az = np.moveaxis(self.A[z], k, -1)
        pad = np.zeros(Az.shape[:-1] + (p,), dtype=np.complex128)
        self.A[z] = np.moveaxis(np.concatenate([Az, pad], axis=-1), -1, k)
        self.t.bond_dim[c] = chi + p
        self.build_up(c)
        return p

    def _visit(self, z, dt, eps, chi_max):
        for k, c in enumerate(self.ch[z]):
            p = self.spawn_spf(z, k, dt, eps, chi_max)
            if p > 0:
                return z, p
            self._move_down(z, k)
            hit = self._visit(c, dt, eps, chi_max)
            if hit is not None:
                return hit
            C = self._move_up(z, k)
            self.A[z] = mode_product(C, self.A[z], k)
        return None

    def _centre_to_root(self, z):
        while z != 0:
            p = int(self.t.parent[z])
            k = self.ch[p].index(z)
            C = self._move_up(p, k)
            self.A[p] = mode_product(C, self.A[p], k)
            z = p

    def expand_pass(self, dt, eps, chi_max):
        """Returns the number of functions added."""
        added = 0
        while True:
            hit = self._visit(0, dt, eps, chi_max)
            if hit is None:
                return added
            added += hit[1]
            self._centre_to_root(hit[0])

    def step_adaptive(self, dt, eps, chi_max, nsteps=1):
        for _ in range(nsteps):
            self.expand_pass(dt, eps, chi_max)
            self.step(dt)
