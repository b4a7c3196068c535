"""Brute-force free-pole HEOM (test oracle).

The auxiliary-density-operator hierarchy of paper SI Eq. fpheom_SM_rescaled is
assembled element by element (without the ADO rescaling), for a two-level
system, K exponentials C(t) = sum_k alpha_k exp(-nu_k t) (SI Eq.
corr_func_expansion) and a fixed depth L per index, and propagated exactly.
It is independent of the operator form used for the TTN generator.
"""
from __future__ import annotations

import itertools
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def heom_generator(Hs, S, alpha, nu, depth):
    """Matrix G with d/dt vec(rho_{m,n}) = G vec(rho) over all ADOs.

    Ordering: index = ((m_0, n_0, m_1, n_1, ..., ) flattened row-major over
    depth+1 levels) * 4 + (2 i + j) for rho[i, j] -- i.e. the bosonic indices
    of the pairs (a_k, b_k) interleaved, the system index fastest."""
    K = len(alpha)
    Ld = depth + 1
    nb = Ld ** (2 * K)
    dim = nb * 4
    G = sp.lil_matrix((dim, dim), dtype=np.complex128)
    sq = [np.sqrt(complex(a)) for a in alpha]
    sqc = [np.sqrt(np.conj(complex(a))) for a in alpha]
    I2 = np.eye(2)

    def vecop_left(X):   # rho -> X rho
        return np.kron(X, I2)

    def vecop_right(X):  # rho -> rho X
        return np.kron(I2, X.T)

    Ls = vecop_left(Hs) - vecop_right(Hs)
    SL, SR = vecop_left(S), vecop_right(S)
    Scomm = SL - SR

    def idx(occ):
        i = 0
        for o in occ:
            i = i * Ld + o
        return i

    for occ in itertools.product(range(Ld), repeat=2 * K):
        row = idx(occ) * 4
        m = occ[0::2]; n = occ[1::2]
        blk = -1j * Ls - sum(nu[k] * m[k] + np.conj(nu[k]) * n[k] for k in range(K)) * np.eye(4)
        G[row:row + 4, row:row + 4] += blk
        for k in range(K):
            # -i sqrt(m_k alpha_k) S rho_{m_k^-}
            if m[k] > 0:
                o = list(occ); o[2 * k] -= 1
                c = idx(o) * 4
                G[row:row + 4, c:c + 4] += -1j * np.sqrt(m[k]) * sq[k] * SL
            # +i sqrt(n_k alpha_k^*) rho_{n_k^-} S
            if n[k] > 0:
                o = list(occ); o[2 * k + 1] -= 1
                c = idx(o) * 4
                G[row:row + 4, c:c + 4] += 1j * np.sqrt(n[k]) * sqc[k] * SR
            # -i sqrt((m_k+1) alpha_k) [S, rho_{m_k^+}]
            if m[k] + 1 < Ld:
                o = list(occ); o[2 * k] += 1
                c = idx(o) * 4
                G[row:row + 4, c:c + 4] += -1j * np.sqrt(m[k] + 1) * sq[k] * Scomm
            # -i sqrt((n_k+1) alpha_k^*) [S, rho_{n_k^+}]
            if n[k] + 1 < Ld:
                o = list(occ); o[2 * k + 1] += 1
                c = idx(o) * 4
                G[row:row + 4, c:c + 4] += -1j * np.sqrt(n[k] + 1) * sqc[k] * Scomm
    return G.tocsr()


def rho_system(Hs, S, alpha, nu, depth, rho0: np.ndarray, times):
    """rho_S(t) = rho_{0,0}(t) (2x2) from exact propagation of the hierarchy."""
    G = heom_generator(Hs, S, alpha, nu, depth)
    v0 = np.zeros(G.shape[0], dtype=np.complex128)
    v0[:4] = rho0.reshape(-1)
    out = []
    prev, v = 0.0, v0
    for t in times:
        v = spla.expm_multiply(G * (t - prev), v)
        prev = t
        out.append(v[:4].reshape(2, 2))
    return out


def pure_dephasing_coherence(alpha, nu, times):
    """rho_updown(t)/rho_updown(0) for H_s = 0, S = sigma_z:
    exp(-4 Re sum_k alpha_k [t/nu_k - (1 - exp(-nu_k t))/nu_k^2])."""
    out = []
    for t in times:
        s = sum(a * (t / v - (1 - np.exp(-v * t)) / v ** 2) for a, v in zip(alpha, nu))
        out.append(np.exp(-4.0 * np.real(s)))
    return np.array(out)
