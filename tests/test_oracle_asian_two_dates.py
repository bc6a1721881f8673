"""Oracle pin for the arithmetic-Asian estimators against a semi-analytic
reference.

With xi = 0 the variance is deterministic: V_0 = v0, V_1 = theta +
(v0 - theta)(1 - kappa dt) (the Milstein step of Sec. 2.4.2 with no noise),
and with N = M = 2 steps and dates the log-price increments of the scheme
are independent Gaussians, X_1 ~ N((r - V_0/2) dt, V_0 dt) and
X_2 - X_1 ~ N((r - V_1/2) dt, V_1 dt), dt = T/2.  The discounted payoff of
the Asian of Eq. (asian_pw), e^{-rT} ((S_1 + S_2)/2 - K)^+, then has a
one-dimensional integral: given S_1 = s, with c = 2K - s,
    E[(A - K)^+ | s] = s/2 + (s/2) e^{mu_2 + sigma_2^2/2} - K            (c <= 0)
                     = (1/2) [s e^{mu_2 + sigma_2^2/2} Phi(d_1) - c Phi(d_2)]  (c > 0)
with d_2 = (ln(s/c) + mu_2)/sigma_2, d_1 = d_2 + sigma_2; the outer
expectation over S_1 is a quadrature.  Puts follow from put-call parity of
the integrand.  The oracle's six Monte Carlo estimators (price, Delta, Gamma
= pathwise/likelihood-ratio mix, Vega = d/dv0, Rho, Theta = -d/dT at fixed
N and M) must match the integral and its central differences in
(S0, v0, r, T) within 4 standard errors: this checks the Asian estimators,
the corrected Asian Rho (reading C5) and the Theta convention against a
reference that shares nothing with the path recursion.
"""
import math

import numpy as np
import pytest

import oracle

integrate = pytest.importorskip("scipy.integrate")
special = pytest.importorskip("scipy.special")


def _phi(x):
    return 0.5 * special.erfc(-x / math.sqrt(2.0))


def asian2_price(S0, v0, kappa, theta, r, T, K, put):
    dt = T / 2.0
    V0 = v0
    V1 = theta + (v0 - theta) * (1.0 - kappa * dt)
    mu1, s1 = (r - 0.5 * V0) * dt, math.sqrt(V0 * dt)
    mu2, s2 = (r - 0.5 * V1) * dt, math.sqrt(V1 * dt)
    g2 = math.exp(mu2 + 0.5 * s2 * s2)

    def call_given(z):
        s = S0 * math.exp(mu1 + s1 * z)
        c = 2.0 * K - s
        if c <= 0.0:
            return 0.5 * s + 0.5 * s * g2 - K
        d2 = (math.log(s / c) + mu2) / s2
        return 0.5 * (s * g2 * _phi(d2 + s2) - c * _phi(d2))

    def given(z):
        cv = call_given(z)
        if not put:
            return cv
        s = S0 * math.exp(mu1 + s1 * z)
        return cv - (0.5 * s + 0.5 * s * g2 - K)        # (K - A)^+ = (A - K)^+ - (A - K)

    f = lambda z: given(z) * math.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    val, _ = integrate.quad(f, -12.0, 12.0, limit=400, epsabs=1e-13, epsrel=1e-12,
                            points=[0.0])
    return math.exp(-r * T) * val


def reference(p, K, T, put):
    a = dict(S0=p["S0"], v0=p["v0"], kappa=p["kappa"], theta=p["theta"], r=p["r"], T=T, K=K, put=put)

    def at(**kw):
        b = dict(a)
        b.update(kw)
        return asian2_price(**b)

    price = at()
    hs = 1e-2 * a["S0"]
    delta = (at(S0=a["S0"] + hs) - at(S0=a["S0"] - hs)) / (2 * hs)
    gamma = (at(S0=a["S0"] + hs) - 2 * price + at(S0=a["S0"] - hs)) / (hs * hs)
    hv = 1e-4 * a["v0"]
    vega = (at(v0=a["v0"] + hv) - at(v0=a["v0"] - hv)) / (2 * hv)
    hr = 1e-4
    rho = (at(r=a["r"] + hr) - at(r=a["r"] - hr)) / (2 * hr)
    hT = 1e-4 * T
    theta_ = -(at(T=T + hT) - at(T=T - hT)) / (2 * hT)
    return np.array([price, delta, gamma, vega, rho, theta_])


@pytest.mark.parametrize("put", [0, 1])
@pytest.mark.parametrize("K", [95.0, 105.0])
def test_two_date_asian_estimators_match_the_integral(put, K):
    p = dict(S0=100.0, v0=0.05, kappa=1.2, theta=0.03, xi=0.0, rho=-0.5, r=0.04)
    T = 1.0
    ref = reference(p, K, T, put)
    est, se = oracle.mc_price_greeks(oracle.Params(**p), [oracle.Contract(1, K, T, put, 2)],
                                     1 << 20, 2, 2024)
    d = np.abs(est[0] - ref)
    assert (d <= 4.0 * se[0] + 1e-6).all(), (d / se[0], est[0], ref)


def test_the_integral_reproduces_black_scholes_limits():
    """Self-check of the reference: with K -> 0 the Asian call is the mean of
    the two discounted forwards, e^{-rT} S0 (e^{r dt} + e^{r T}) / 2, for any
    variance path; and its put is worth ~0."""
    p = dict(S0=100.0, v0=0.05, kappa=1.2, theta=0.03, r=0.04)
    T = 1.0
    c = asian2_price(p["S0"], p["v0"], p["kappa"], p["theta"], p["r"], T, 1e-9, 0)
    fwd = math.exp(-p["r"] * T) * p["S0"] * (math.exp(p["r"] * T / 2) + math.exp(p["r"] * T)) / 2
    assert abs(c - fwd) < 1e-8
    assert asian2_price(p["S0"], p["v0"], p["kappa"], p["theta"], p["r"], T, 1e-9, 1) < 1e-12
