"""Plain complex128 multi-set TTN projector-splitting integrator (test oracle).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and nothing in the product
path.

State (paper Sec. II.A, multi-set ansatz): |Psi> = sum_alpha |alpha> |Psi^alpha>
with one TTN per set state alpha, all on the same tree with the same bond
dimensions.  ``A[alpha][z]`` has the single-set layout [n_1..n_d, N]; every
set is in canonical gauge with its orthogonality centre at the same node, so
between steps the state norm is sum_alpha ||A[alpha][root]||^2.

Hamiltonian (workloads.MultiSetSOP): H = sum_r c_r |a_r><b_r| (x) prod_leaf M_r,leaf.

Equations (the paper states the ansatz, not its equations of motion; this is
the reading used here).  The |alpha> are orthonormal and each set's tensors
are independent parameters, so the tangent space of the multi-set manifold
is the direct sum of the single-set tangent spaces of the |Psi^alpha>, and its
projector sum_alpha |alpha><alpha| (x) P^alpha splits node by node and bond by
bond exactly like the single-set one (Sec. II.C).  Taking the same node and
bond order in every set, each sub-step is a linear equation that couples the
sets' tensors at one node:
    dA^alpha/dt = -i sum_{r: a_r = alpha} c_r (x_k h_r^(z,k)) A^{b_r} (H_r^z)^T
with cross-set matrix elements h_r^z[i, i'] = <phi_i^{a_r}| h_r |phi_i'^{b_r}>
and H_r^z[n, n'] = <Psi_n^{a_r}| H_r |Psi_n'^{b_r}>.  For a_r != b_r the identity
on a subtree (or on its complement) becomes the overlap of the two sets'
functions there, so every environment of such a term is a real matrix; for
a_r == b_r the single-set identities hold.  Gauge moves (QR, Sec. II.A) act on
each set by itself; the Krylov exponentials act on all sets' tensors of the
node (or bond) as one vector.

Pinned against (tests/test_multiset_oracle.py): exact propagation of the full
multi-set Hamiltonian at full bond dimension, the single-set oracle on each
set when the sets are uncoupled, norm and energy conservation at truncated
bond dimension, and the closed-form Rabi oscillation of a pure set coupling.
"""
from __future__ import annotations

import numpy as np

from .ttn import QR_TOL_FP64, KRYLOV_TOL, KRYLOV_MAXDIM, expm_krylov, full_state, mode_product, qr_along


class MultiSetTTN:
    """Multi-set TTN plus per-term cross-set environments.

    ``tree`` is a workloads.Tree, ``H`` a workloads.MultiSetSOP, ``A`` the list
    (over sets) of node-tensor lists (copied)."""

    def __init__(self, tree, H, A, qr_tol: float = QR_TOL_FP64,
                 krylov_tol: float = KRYLOV_TOL, krylov_maxdim: int = KRYLOV_MAXDIM):
        assert len(A) == H.n_sets, "one tensor list per set"
        self.t = tree
        self.H = H
        self.S = H.n_sets
        self.A = [[np.array(a, dtype=np.complex128, copy=True) for a in As] for As in A]
        for As in self.A:
            for z in range(tree.n):
                assert As[z].shape == self.A[0][z].shape, "every set has the same bond dimensions"
        self.qr_tol = qr_tol
        self.ktol = krylov_tol
        self.kmax = krylov_maxdim
        n, R = tree.n, H.n_terms
        self.ch = [tree.children(z) for z in range(n)]
        self.bra = [int(a) for a in H.bra]
        self.ket = [int(b) for b in H.ket]
        self.fac = [dict() for _ in range(R)]
        for r, fs in enumerate(H.factors):
            for (l, m) in fs:
                assert tree.is_leaf(l), "factors act on leaves"
                assert l not in self.fac[r], "one factor per leaf and term"
                self.fac[r][l] = H.mats[m]
        leaves_of = [set(tree.subtree_leaves(z)) for z in range(n)]
        # inside[z, r]: term r needs a matrix for the subtree of z (it acts
        # there, or it connects two different sets: the overlap).  outside[z, r]:
        # the same for the complement (never at the root).
        self.inside = np.zeros((n, R), dtype=bool)
        self.outside = np.zeros((n, R), dtype=bool)
        for r in range(R):
            ls = set(self.fac[r])
            cross = self.bra[r] != self.ket[r]
            for z in range(n):
                self.inside[z, r] = cross or len(ls & leaves_of[z]) > 0
                self.outside[z, r] = z > 0 and (cross or len(ls - leaves_of[z]) > 0)
        self.up = [dict() for _ in range(n)]     # h_r^z between sets a_r (bra) and b_r (ket)
        self.down = [dict() for _ in range(n)]   # H_r^z between the same sets
        for z in self.postorder():
            if z > 0:
                self.build_up(z)
        self.t_elapsed = 0.0

    def postorder(self):
        out = []
        def rec(z):
            for c in self.ch[z]:
                rec(c)
            out.append(z)
        rec(0)
        return out

    def _stack(self, z):
        return np.stack([self.A[a][z] for a in range(self.S)])

    def _unstack(self, z, X):
        for a in range(self.S):
            self.A[a][z] = np.ascontiguousarray(X[a])

    # -- environments ----------------------------------------------------------
    def _apply_child_ops(self, T, z, r, skip=None):
        """Term r's operators on the child indices of node z (a leaf: its
        physical factor, identity if none)."""
        if self.t.is_leaf(z):
            M = self.fac[r].get(z)
            return T if M is None else mode_product(M, T, 0)
        for k, c in enumerate(self.ch[z]):
            if k != skip and self.inside[c, r]:
                T = mode_product(self.up[c][r], T, k)
        return T

    def build_up(self, z):
        """h_r^z = (A^{a_r})^dag (x_k h_r^(z,k)) A^{b_r}, node z isometric towards its parent."""
        nd = self.A[0][z].ndim
        ax = list(range(nd - 1))
        self.up[z] = {}
        for r in range(self.H.n_terms):
            if not self.inside[z, r]:
                continue
            T = self._apply_child_ops(self.A[self.ket[r]][z], z, r)
            self.up[z][r] = np.tensordot(self.A[self.bra[r]][z].conj(), T, axes=(ax, ax))

    def build_down(self, z, k):
        """Mean-field matrices of child c = children(z)[k] from node z isometric
        towards c (every set): H_r^c = (Q^{a_r})^dag (x_{j!=k} h_r^(z,j)) H_r^z Q^{b_r}."""
        c = self.ch[z][k]
        nd = self.A[0][z].ndim
        axes = [a for a in range(nd) if a != k]
        self.down[c] = {}
        for r in range(self.H.n_terms):
            if not self.outside[c, r]:
                continue
            T = self._apply_child_ops(self.A[self.ket[r]][z], z, r, skip=k)
            if self.outside[z, r]:
                T = mode_product(self.down[z][r], T, nd - 1)
            self.down[c][r] = np.tensordot(self.A[self.bra[r]][z].conj(), T, axes=(axes, axes))

    # -- effective operators on all sets of one node / bond ----------------------
    def heff(self, z, X):
        """Y[a] = sum_{r: a_r = a} c_r (x_k h_r^(z,k)) X[b_r] (H_r^z)^T, X of shape [S, dims..]."""
        Y = np.zeros_like(X)
        nd = X.ndim - 1
        for r, cr in enumerate(self.H.coeffs):
            T = self._apply_child_ops(X[self.ket[r]], z, r)
            if self.outside[z, r]:
                T = mode_product(self.down[z][r], T, nd - 1)
            Y[self.bra[r]] += cr * T
        return Y

    def kbond(self, c, C):
        """Bond operator on C[S, n, m]: Y[a] = sum_{r: a_r = a} c_r h_r^c C[b_r] (H_r^c)^T."""
        Y = np.zeros_like(C)
        for r, cr in enumerate(self.H.coeffs):
            T = C[self.ket[r]]
            if self.inside[c, r]:
                T = self.up[c][r] @ T
            if self.outside[c, r]:
                T = T @ self.down[c][r].T
            Y[self.bra[r]] += cr * T
        return Y

    def _evolve_node(self, z, tau):
        X = expm_krylov(lambda x: self.heff(z, x), self._stack(z), tau,
                        self.H.hermitian, self.ktol, self.kmax)
        self._unstack(z, X)

    def _evolve_bond_back(self, c, C, tau):
        return expm_krylov(lambda x: self.kbond(c, x), C, -tau,
                           self.H.hermitian, self.ktol, self.kmax)

    # -- projector-splitting sweep (per-set gauge moves) --------------------------
    def _move_down(self, z, k):
        c = self.ch[z][k]
        for a in range(self.S):
            Q, R = qr_along(self.A[a][z], k, self.qr_tol)
            self.A[a][z] = Q
            self.A[a][c] = mode_product(R, self.A[a][c], self.A[a][c].ndim - 1)
        self.build_down(z, k)

    def _move_up(self, z, k):
        c = self.ch[z][k]
        Rs = []
        for a in range(self.S):
            Ac = self.A[a][c]
            Q, R = qr_along(Ac, Ac.ndim - 1, self.qr_tol)
            self.A[a][c] = Q
            Rs.append(R)
        self.build_up(c)
        return np.stack(Rs)

    def _absorb_bond(self, z, k, C):
        for a in range(self.S):
            self.A[a][z] = mode_product(C[a], self.A[a][z], k)

    def sweep_S(self, z, tau):
        for k, c in enumerate(self.ch[z]):
            self._move_down(z, k)
            self.sweep_S(c, tau)
            C = self._move_up(z, k)
            C = self._evolve_bond_back(c, C, tau)
            self._absorb_bond(z, k, C)
        self._evolve_node(z, tau)

    def sweep_Sstar(self, z, tau):
        self._evolve_node(z, tau)
        for k in range(len(self.ch[z]) - 1, -1, -1):
            c = self.ch[z][k]
            Cs = []
            for a in range(self.S):
                Q, R = qr_along(self.A[a][z], k, self.qr_tol)
                self.A[a][z] = Q
                Cs.append(R.T)           # C[n, m]: n SPF index of c, m SHF index
            self.build_down(z, k)
            C = self._evolve_bond_back(c, np.stack(Cs), tau)
            for a in range(self.S):
                self.A[a][c] = mode_product(C[a].T, self.A[a][c], self.A[a][c].ndim - 1)
            self.sweep_Sstar(c, tau)
            self._absorb_bond(z, k, self._move_up(z, k))

    def step(self, dt: float, nsteps: int = 1):
        """step(dt) = S*(root, dt/2) o S(root, dt/2), as for a single set."""
        for _ in range(nsteps):
            self.sweep_S(0, dt / 2.0)
            self.sweep_Sstar(0, dt / 2.0)
            self.t_elapsed += dt

    # -- observables (centre at the root) -----------------------------------------
    def set_populations(self):
        """<Psi^alpha|Psi^alpha> = ||A^alpha[root]||^2 for every set."""
        return np.array([float(np.vdot(self.A[a][0], self.A[a][0]).real) for a in range(self.S)])

    def norm2(self):
        return float(self.set_populations().sum())

    def energy(self):
        """<Psi|H|Psi> / <Psi|Psi>."""
        X = self._stack(0)
        return complex(np.vdot(X, self.heff(0, X)) / self.norm2())

    def reduced_density(self, alpha, leaf):
        """Unnormalised leaf density of set alpha, <Psi^alpha| . |Psi^alpha> traced
        over every other leaf (trace = the set's population)."""
        A = self.A[alpha]
        G = np.ones((1, 1), dtype=np.complex128)
        path = []
        u = leaf
        while u > 0:
            path.append(u); u = self.t.parent[u]
        z = 0
        for c in reversed(path):
            k = self.ch[z].index(c)
            nd = A[z].ndim
            axes = [a for a in range(nd) if a != k]
            T = mode_product(G, A[z], nd - 1)
            G = np.tensordot(A[z].conj(), T, axes=(axes, axes))
            z = c
        return A[leaf] @ G.T @ A[leaf].conj().T

    def full_state(self):
        """Dense vector over (set, leaves in node order), set index slowest."""
        return np.concatenate([full_state(self.t, self.A[a]) for a in range(self.S)])
