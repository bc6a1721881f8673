"""Pins for the closed forms the Monte Carlo oracle is checked against."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import closed_form as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_heston_closed_form_reproduces_paper_values():
    g = json.load(open(os.path.join(GOLDEN, "paper_table1.json")))
    p, e = g["params"], g["european_closed_form"]
    r = cf.heston_price_greeks(p["S0"], p["K"], p["T"], p["r"], p["v0"], p["kappa"], p["theta"],
                               p["xi"], p["rho"])
    for k in ("price", "delta", "rho"):
        assert round(r[k], e["digits"]) == pytest.approx(e[k], abs=1e-12), (k, r[k])


def test_heston_zero_vol_of_vol_limit_is_black_scholes():
    # v0 = theta and xi -> 0: constant variance theta.  With rho = 0 the first
    # correction is O(xi^2), so shrinking xi by 10/3 shrinks the gap ~11x.
    S0, K, T, r, th = 100.0, 110.0, 0.7, 0.02, 0.05
    b = cf.bs_total_variance(S0, K, T, r, th * T, dw_dv0=0.0, dw_dT=th)
    keys = ("price", "delta", "gamma", "rho", "theta")
    gap = {}
    for xi in (1e-2, 3e-3, 1e-3):
        h = cf.heston_price_greeks(S0, K, T, r, th, 1.5, th, xi, 0.0)
        gap[xi] = {k: abs(h[k] - b[k]) / abs(b[k]) for k in keys}
    for k in keys:
        assert gap[1e-3][k] < 2e-6, k
        assert 8.0 < gap[1e-2][k] / gap[3e-3][k] < 14.0, k


def test_heston_vega_matches_finite_difference_of_price():
    args = dict(S0=100.0, K=95.0, T=1.3, r=0.04, kappa=2.0, theta=0.05, xi=0.5, rho=-0.6)
    v0, hv = 0.03, 1e-5
    g = cf.heston_price_greeks(v0=v0, **args)
    f = lambda v: cf.heston_call_price(args["S0"], args["K"], args["T"], args["r"], v,
                                       args["kappa"], args["theta"], args["xi"], args["rho"])
    fd = (f(v0 + hv) - f(v0 - hv)) / (2 * hv)
    assert g["vega"] == pytest.approx(fd, rel=1e-6)


def test_heston_characteristic_function_matches_quadrature_of_the_pde_free_moments():
    # phi(-i) = E[S_T] = S0 e^{rT} and phi(0) = 1 for any parameters
    args = (100.0, 0.04, 2.0, 0.04, 0.3, -0.7, 0.05, 1.0)
    phi_mi, _ = cf.heston_cf(-1j, *args)
    phi_0, _ = cf.heston_cf(0.0 + 0j, *args)
    assert phi_mi == pytest.approx(100.0 * math.exp(0.05), rel=1e-12)
    assert phi_0 == pytest.approx(1.0, rel=1e-14)
    # E[V_T]-driven variance: -d^2/dw^2 log phi at 0 equals Var(ln S_T) > 0
    h = 1e-3
    lp = lambda w: np.log(cf.heston_cf(w + 0j, *args)[0])
    var = -((lp(h) - 2 * lp(0.0) + lp(-h)) / h**2).real
    # mean integrated variance: theta T + (v0 - theta)(1 - e^{-kT})/k = 0.04
    assert 0.03 < var < 0.05


@pytest.mark.parametrize("is_put", [False, True])
def test_black_scholes_greeks_are_derivatives_of_price(is_put):
    S0, K, T, r, s2 = 100.0, 97.0, 0.9, 0.03, 0.06
    f = lambda S=S0, t=T, rr=r, v=s2: cf.bs_total_variance(S, K, t, rr, v * t, is_put=is_put)["price"]
    g = cf.bs_total_variance(S0, K, T, r, s2 * T, dw_dv0=T, dw_dT=s2, is_put=is_put)
    h = 1e-5
    assert g["delta"] == pytest.approx((f(S=S0 + h) - f(S=S0 - h)) / (2 * h), rel=1e-6)
    assert g["gamma"] == pytest.approx((f(S=S0 + 1e-3) - 2 * f() + f(S=S0 - 1e-3)) / 1e-6,
                                       rel=1e-4)
    assert g["rho"] == pytest.approx((f(rr=r + h) - f(rr=r - h)) / (2 * h), rel=1e-6)
    assert g["vega"] == pytest.approx((f(v=s2 + h) - f(v=s2 - h)) / (2 * h), rel=1e-6)
    assert g["theta"] == pytest.approx(-(f(t=T + h) - f(t=T - h)) / (2 * h), rel=1e-6)
    # and the price is the discounted lognormal expectation
    sd = math.sqrt(s2 * T)
    mu = math.log(S0) + (r - 0.5 * s2) * T
    payoff = (lambda x: max(K - math.exp(x), 0.0)) if is_put else (lambda x: max(math.exp(x) - K, 0.0))
    ev, _ = integrate.quad(lambda x: payoff(x) * stats.norm.pdf(x, mu, sd),
                           mu - 12 * sd, mu + 12 * sd, limit=200)
    assert f() == pytest.approx(math.exp(-r * T) * ev, rel=1e-9)
