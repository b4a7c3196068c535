"""Exact state-vector references for small problems (test oracle).

The full Hamiltonian of a sum-of-product operator (paper Eq. sop_ham) is
assembled as a sparse matrix over the leaves in increasing node order, and the
state is propagated exactly: by diagonalisation for Hermitian H, by
``scipy.sparse.linalg.expm_multiply`` otherwise.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def full_hamiltonian(tree, H, dense: bool = False):
    """sum_r c_r kron_{leaves} (factor or identity), leaves in node order."""
    leaves = tree.leaves()
    dims = [int(tree.phys_dim[l]) for l in leaves]
    D = int(np.prod(dims))
    out = sp.csr_matrix((D, D), dtype=np.complex128)
    for c, fs in zip(H.coeffs, H.factors):
        fac = {l: H.mats[m] for (l, m) in fs}
        M = sp.identity(1, dtype=np.complex128, format="csr")
        for l, d in zip(leaves, dims):
            X = sp.csr_matrix(fac[l]) if l in fac else sp.identity(d, dtype=np.complex128, format="csr")
            M = sp.kron(M, X, format="csr")
        out = out + c * M
    return out.toarray() if dense else out


def propagate_eigh(Hd: np.ndarray, psi0: np.ndarray, times):
    """psi(t) = V exp(-i Lambda t) V^dag psi0 for Hermitian dense Hd."""
    ev, V = np.linalg.eigh(Hd)
    c0 = V.conj().T @ psi0
    return [V @ (np.exp(-1j * ev * t) * c0) for t in times]


def propagate_sparse(Hs, psi0: np.ndarray, times):
    """psi(t_i) = exp(-i H t_i) psi0 for increasing times t_i >= 0 (any H),
    by scipy's expm_multiply over each interval in turn."""
    out, psi, t_prev = [], np.asarray(psi0, dtype=np.complex128), 0.0
    for t in times:
        psi = spla.expm_multiply(-1j * (float(t) - t_prev) * Hs, psi)
        out.append(psi)
        t_prev = float(t)
    return out


def leaf_reduced_density(psi: np.ndarray, dims, pos: int) -> np.ndarray:
    """rho[a, a'] = sum_rest psi[.., a, ..] conj(psi[.., a', ..])."""
    T = np.moveaxis(psi.reshape(dims), pos, 0).reshape(dims[pos], -1)
    return T @ T.conj().T


def leaf_populations(tree, psi: np.ndarray, leaves):
    all_leaves = tree.leaves()
    dims = [int(tree.phys_dim[l]) for l in all_leaves]
    out = []
    for l in leaves:
        rho = leaf_reduced_density(psi, dims, all_leaves.index(l))
        out.append(np.real(np.diag(rho)) / np.real(np.trace(rho)))
    return out


def full_multiset_hamiltonian(tree, H, dense: bool = False):
    """sum_r c_r |a_r><b_r| (x) kron_{leaves} (factor or identity) for a
    workloads.MultiSetSOP: the set index is the slowest index."""
    leaves = tree.leaves()
    dims = [int(tree.phys_dim[l]) for l in leaves]
    D = int(np.prod(dims))
    S = int(H.n_sets)
    out = sp.csr_matrix((S * D, S * D), dtype=np.complex128)
    for c, fs, a, b in zip(H.coeffs, H.factors, H.bra, H.ket):
        fac = {l: H.mats[m] for (l, m) in fs}
        E = sp.csr_matrix(([1.0], ([int(a)], [int(b)])), shape=(S, S), dtype=np.complex128)
        M = E
        for l, d in zip(leaves, dims):
            X = sp.csr_matrix(fac[l]) if l in fac else sp.identity(d, dtype=np.complex128, format="csr")
            M = sp.kron(M, X, format="csr")
        out = out + c * M
    return out.toarray() if dense else out
