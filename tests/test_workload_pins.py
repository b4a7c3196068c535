"""Pins of the shared input generators that carry bath physics (paper
Sec. II.E.1 and Sec. II.E.3), checked against definitions computed another
way: the Drude-Lorentz exponential expansion against the bath correlation
function integrated numerically, and the thermal spectral density against
detailed balance.  Both the oracle and the GPU path consume these arrays, so
GPU parity cannot catch an error in them; these tests can."""
import numpy as np
import pytest
from scipy import integrate

import workloads as W


def correlation_numeric(lam, gamma, beta, t):
    """C(t) = (1/pi) int_0^inf J(w) [coth(beta w / 2) cos(w t) - i sin(w t)] dw
    for J(w) = 2 lam gamma w / (w^2 + gamma^2), by QUADPACK's Fourier
    quadrature on the half line (QAWF)."""
    def J(w):
        return 2.0 * lam * gamma * w / (w * w + gamma * gamma)

    def Jcoth(w):
        x = 0.5 * beta * w
        if x < 1e-6:               # J(w) coth(beta w / 2) -> 4 lam / (beta gamma) as w -> 0
            return 4.0 * lam / (beta * gamma) * (1.0 + x * x / 3.0) / (1.0 + (w / gamma) ** 2)
        return J(w) / np.tanh(x)

    re, _ = integrate.quad(Jcoth, 0.0, np.inf, weight="cos", wvar=t, limlst=200)
    im, _ = integrate.quad(J, 0.0, np.inf, weight="sin", wvar=t, limlst=200)
    return (re - 1j * im) / np.pi


def matsubara_tail(lam, gamma, beta, n, t, jmax=200000):
    """Sum of |terms| of the Matsubara series beyond the first n terms."""
    j = np.arange(n + 1, jmax + 1, dtype=np.float64)
    v = 2.0 * np.pi * j / beta
    return float(np.sum(np.abs(4.0 * lam * gamma * v / (beta * (v * v - gamma * gamma))) * np.exp(-v * t)))


@pytest.mark.parametrize("beta", [1.0, 2.0])
@pytest.mark.parametrize("t", [0.1, 0.3, 1.0, 3.0])
def test_drude_lorentz_expansion_equals_correlation_function(beta, t):
    lam, gamma, n = 0.1, 5.0, 15
    al, nu = W.drude_lorentz_exponentials(lam, gamma, beta, n)
    series = complex(np.sum(al * np.exp(-nu * t)))
    exact = correlation_numeric(lam, gamma, beta, t)
    bound = matsubara_tail(lam, gamma, beta, n, t) + 1e-8 * abs(exact) + 1e-10
    assert abs(series - exact) <= bound, (series, exact, bound)


def test_drude_lorentz_more_matsubara_terms_converge():
    """At small t the tail matters: adding terms approaches the integral."""
    lam, gamma, beta, t = 0.1, 5.0, 1.0, 0.02
    exact = correlation_numeric(lam, gamma, beta, t)
    errs = []
    for n in (5, 50, 500):
        al, nu = W.drude_lorentz_exponentials(lam, gamma, beta, n)
        errs.append(abs(complex(np.sum(al * np.exp(-nu * t))) - exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= matsubara_tail(lam, gamma, beta, 500, t) + 1e-9


def test_thermal_spectral_density_detailed_balance():
    J = W.ohmic_J(0.3, 5.0)
    for beta in (0.5, 1.0, 5.0):
        Jb = W.thermal_J(J, beta)
        w = np.linspace(0.05, 30.0, 400)
        # detailed balance J_beta(-w) = exp(-beta w) J_beta(w)
        # (coth - 1 cancels for large beta w: relative 1e-9 with a floor at the density's scale)
        np.testing.assert_allclose(Jb(-w), np.exp(-beta * w) * Jb(w), rtol=1e-9, atol=1e-14 * Jb(w).max())
        # emission minus absorption is the zero-temperature density
        np.testing.assert_allclose(Jb(w) - Jb(-w), J(w), rtol=1e-12)
        assert np.all(Jb(w) > 0) and np.all(Jb(-w) >= 0)


def test_thermal_spectral_density_zero_temperature_limit():
    J = W.ohmic_J(0.3, 5.0)
    w = np.linspace(-20.0, 20.0, 401)
    np.testing.assert_allclose(W.thermal_J(J, np.inf)(w), np.where(w > 0, J(w), 0.0), rtol=0, atol=0)
    # a large but finite beta approaches it
    np.testing.assert_allclose(W.thermal_J(J, 200.0)(w[np.abs(w) > 0.5]),
                               np.where(w[np.abs(w) > 0.5] > 0, J(w[np.abs(w) > 0.5]), 0.0), atol=1e-30)


def test_multiset_vibronic_generator_is_the_model_formula():
    """The shared multi-set vibronic generator against its formula written
    with Kronecker products (set index slowest, leaves in node order):
    sum_s |s><s| (x) [E_s + sum_i w_i (n_i + 1/2) + sum_i kappa_i^s Q_i]
    + sum_{s != s'} |s><s'| (x) [J_{ss'} + sum_j lam_j^{ss'} Q_{c_j}],
    J and lam symmetric in (s, s'), Q = (a + a^+)/sqrt 2."""
    from oracle import exact
    p = W.multiset_vibronic_problem(n_states=3, n_modes=3, d=3, chi=3, seed=4)
    m = p.meta
    S, d = 3, m["d"]
    leaves = p.tree.leaves()
    pos = {int(l): k for k, l in enumerate(leaves)}           # leaf -> Kronecker position
    mode_pos = [pos[int(l)] for l in m["modes"]]
    a = np.diag(np.sqrt(np.arange(1, d)), 1)
    Q = (a + a.T) / np.sqrt(2.0)
    num = np.diag(np.arange(d) + 0.5)
    I = np.eye(d)

    def on(k, M):                                              # M on Kronecker position k
        out = np.ones((1, 1))
        for j in range(len(leaves)):
            out = np.kron(out, M if j == k else I)
        return out

    D = d ** len(leaves)
    want = np.zeros((S * D, S * D), dtype=np.complex128)
    for s in range(S):
        blk = m["E"][s] * np.eye(D)
        for i in range(3):
            blk = blk + m["omega"][i] * on(mode_pos[i], num) + m["kappa"][i, s] * on(mode_pos[i], Q)
        want[s * D:(s + 1) * D, s * D:(s + 1) * D] += blk
    for s in range(S):
        for s2 in range(S):
            if s == s2:
                continue
            lo, hi = min(s, s2), max(s, s2)
            blk = m["J"][lo, hi] * np.eye(D)
            for j, i in enumerate(m["coupling_modes"]):
                blk = blk + m["lam"][j, lo, hi] * on(mode_pos[i], Q)
            want[s * D:(s + 1) * D, s2 * D:(s2 + 1) * D] += blk
    got = exact.full_multiset_hamiltonian(p.tree, p.H, dense=True)
    assert np.abs(got - want).max() <= 1e-14
    assert np.abs(got - got.conj().T).max() <= 1e-15
