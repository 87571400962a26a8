"""Identities the register-tile adjoint relies on, checked with dense numpy
algebra on small random Hamiltonians (CPU).

The adjoint of one Taylor step T = sum_{k<=K} c_k H^k, c_k = (-i dt)^k / k!,
is formed on the GPU from two chains (Sec. 2.3's polynomial, differentiated
term by term):
  - lambda_n = T^dagger lambda_{n+1} = lambda + H mu_0, the mu recurrence
    taken one level further instead of a separate Taylor step;
  - in the variables of the dt-weighted stencil Hh = dt H,
    phi_a = Hh^a psi and mu_a with coefficients i^k / k!, the gradient
    2 Re sum_a <mu_a, dH phi_a> equals dt 2 Re sum_a <mu_a^h, dH phi_a^h>.
Both are checked here against the direct definitions, and the gradient
against central differences of the step itself.
"""
import math

import numpy as np


def _herm(rng, n):
    a = rng.standard_normal((n, n))
    return (a + a.T) / 2.0


def _step(H, dt, K):
    n = H.shape[0]
    T = np.zeros((n, n), dtype=np.complex128)
    P = np.eye(n, dtype=np.complex128)
    for k in range(K + 1):
        if k > 0:
            P = P @ H
        T += ((-1j * dt) ** k / math.factorial(k)) * P
    return T


def _mu(H, lam, dt, K):
    """mu_a = sum_{b < K - a} conj(c_{a+b+1}) H^b lambda, by the recurrence."""
    cbar = [(1j * dt) ** k / math.factorial(k) for k in range(K + 1)]
    mus = [None] * K
    mus[K - 1] = cbar[K] * lam
    for a in range(K - 2, -1, -1):
        mus[a] = cbar[a + 1] * lam + H @ mus[a + 1]
    return mus


def test_next_adjoint_state_is_lambda_plus_h_mu0():
    rng = np.random.default_rng(0)
    for K in (1, 2, 5, 14):
        H = _herm(rng, 9)
        lam = rng.standard_normal(9) + 1j * rng.standard_normal(9)
        dt = 0.07
        mus = _mu(H, lam, dt, K)
        direct = _step(H, dt, K).conj().T @ lam
        assert np.max(np.abs(lam + H @ mus[0] - direct)) <= 1e-14 * np.max(np.abs(direct))


def test_scaled_chains_give_the_same_gradient():
    rng = np.random.default_rng(1)
    n, K, dt = 8, 9, 0.05
    H = _herm(rng, n)
    dH = _herm(rng, n)
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    # unscaled: phi_a = H^a psi, mu_a from conj(c_k)
    phis = [psi]
    for _ in range(1, K):
        phis.append(H @ phis[-1])
    mus = _mu(H, lam, dt, K)
    g = sum(2.0 * np.real(np.vdot(mus[a], dH @ phis[a])) for a in range(K))
    # scaled: Hh = dt H, phi^h_a = Hh^a psi, mu^h with i^k / k!
    Hh = dt * H
    ph = [psi]
    for _ in range(1, K):
        ph.append(Hh @ ph[-1])
    co = [1j ** k / math.factorial(k) for k in range(K + 1)]
    mh = [None] * K
    mh[K - 1] = co[K] * lam
    for a in range(K - 2, -1, -1):
        mh[a] = co[a + 1] * lam + Hh @ mh[a + 1]
    gh = dt * sum(2.0 * np.real(np.vdot(mh[a], dH @ ph[a])) for a in range(K))
    assert abs(g - gh) <= 1e-13 * max(1.0, abs(g))
    # and lambda_n = lambda + Hh mu^h_0 in the scaled variables
    direct = _step(H, dt, K).conj().T @ lam
    assert np.max(np.abs(lam + Hh @ mh[0] - direct)) <= 1e-14 * np.max(np.abs(direct))


def test_gradient_matches_central_differences_of_the_step():
    """d/dtheta Re <lambda, T(H + theta dH) psi> at theta = 0 is the sum."""
    rng = np.random.default_rng(2)
    n, K, dt = 7, 6, 0.1
    H = _herm(rng, n)
    dH = _herm(rng, n)
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    phis = [psi]
    for _ in range(1, K):
        phis.append(H @ phis[-1])
    mus = _mu(H, lam, dt, K)
    g = sum(2.0 * np.real(np.vdot(mus[a], dH @ phis[a])) for a in range(K))
    h = 1e-5
    f = lambda t: 2.0 * np.real(np.vdot(lam, _step(H + t * dH, dt, K) @ psi))
    fd = (f(h) - f(-h)) / (2 * h)
    assert abs(g - fd) <= 1e-8 * max(1.0, abs(g))
