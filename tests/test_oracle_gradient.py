"""Pins for the oracle's parameter gradient (forward-mode tangents in seven
directions), which the GPU adjoint is checked against."""
import numpy as np
import pytest

import oracle
from oracle import Contract, Params
from oracle import closed_form as cf

BASE = Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)


@pytest.mark.parametrize("c", [Contract(0, 100.0, 1.0), Contract(1, 100.0, 1.0),
                               Contract(0, 95.0, 1.0, 1), Contract(1, 105.0, 1.0, 1, 4)],
                         ids=["euro", "asian", "euro_put", "asian4_put"])
def test_gradient_matches_crn_finite_differences(c):
    n, N, seed = 1 << 14, 32, 13
    m, _ = oracle.mc_gradient(BASE, c, n, N, seed)
    for i, name in enumerate(oracle.PARAM_NAMES):
        x = getattr(BASE, name)
        h = 1e-4 * abs(x)
        up = oracle.mc_price_greeks(BASE.replace(**{name: x + h}), [c], n, N, seed)[0][0, 0]
        dn = oracle.mc_price_greeks(BASE.replace(**{name: x - h}), [c], n, N, seed)[0][0, 0]
        fd = (up - dn) / (2 * h)
        assert abs(m[1 + i] - fd) <= 2e-3 * max(1.0, abs(fd)), (name, m[1 + i], fd)


def test_gradient_components_equal_the_greek_estimators():
    for c in (Contract(0, 100.0, 1.0), Contract(1, 95.0, 1.0, 1, 8)):
        m, _ = oracle.mc_gradient(BASE, c, 4096, 16, 2)
        g, _ = oracle.mc_price_greeks(BASE, [c], 4096, 16, 2)
        # price, delta (S0), vega (v0), rho (r)
        np.testing.assert_allclose([m[0], m[1], m[2], m[7]], [g[0, 0], g[0, 1], g[0, 3], g[0, 4]],
                                   rtol=1e-12, atol=1e-12)


def test_gradient_matches_closed_form():
    c = Contract(0, 100.0, 1.0)
    m, se = oracle.mc_gradient(BASE, c, 1 << 19, 64, 21)

    def price(**kw):
        q = dict(BASE.__dict__, **kw)
        return cf.heston_call_price(q["S0"], 100.0, 1.0, q["r"], q["v0"], q["kappa"], q["theta"],
                                    q["xi"], q["rho"])
    for i, name in enumerate(oracle.PARAM_NAMES):
        x = getattr(BASE, name)
        h = 1e-4 * abs(x)
        ref = (price(**{name: x + h}) - price(**{name: x - h})) / (2 * h)
        assert abs(m[1 + i] - ref) < 4 * se[1 + i] + 5e-3 * max(1.0, abs(ref)), (name, m[1 + i], ref)
