"""Pins for the oracle's Broadie-Kaya exact simulation (Sec. 2.2-2.3)."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import closed_form as cf
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
E1 = oracle.Params(S0=100.0, v0=0.010201, kappa=6.21, theta=0.019, xi=0.61, rho=-0.7, r=0.0319)
C1 = oracle.Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)


@pytest.mark.parametrize("a", [0.3, 1.0, 2.5, 10.0])
def test_marsaglia_tsang_gamma(a):
    rng = np.random.default_rng(1)
    x = exact._gamma_mt(rng, np.full(100000, a))
    n = len(x)
    assert abs(x.mean() - a) < 5 * math.sqrt(a / n)
    assert abs(x.var() - a) < 5 * math.sqrt((6 * a + 2 * a * a) / n) + 5 * math.sqrt(a / n)
    assert stats.kstest(x, "gamma", args=(a,)).pvalue > 1e-4


@pytest.mark.parametrize("kappa,theta,xi,v0", [(6.21, 0.019, 0.61, 0.010201),   # d = 1.27
                                               (1.0, 0.02, 0.5, 0.03),           # d = 0.32 (Poisson mixture)
                                               (2.0, 0.04, 0.3, 0.04)])          # d = 3.56
def test_cir_transition_moments(kappa, theta, xi, v0):
    rng = np.random.default_rng(2)
    dt, n = 0.25, 200000
    Vt = exact.sample_variance(rng, np.full(n, v0), dt, kappa, theta, xi)
    e = math.exp(-kappa * dt)
    mean = theta + (v0 - theta) * e
    var = v0 * xi**2 * e / kappa * (1 - e) + theta * xi**2 / (2 * kappa) * (1 - e) ** 2
    assert (Vt >= 0).all()
    assert abs(Vt.mean() - mean) < 5 * math.sqrt(var / n)
    assert abs(Vt.var() - var) < 0.05 * var


def test_characteristic_function_and_integrated_variance_mean():
    p = C1
    rng = np.random.default_rng(3)
    dt, n = 0.5, 2000
    Vu = np.full(n, p.v0)
    Vt = exact.sample_variance(rng, Vu, dt, p.kappa, p.theta, p.xi)
    nu = 2 * p.kappa * p.theta / p.xi**2 - 1
    ek = math.exp(-p.kappa * dt)
    z0 = np.sqrt(Vu * Vt) * 4 * p.kappa * math.exp(-0.5 * p.kappa * dt) / (p.xi**2 * (1 - ek))
    a = np.linspace(0.0, 2000.0, 400)[None, :].repeat(4, 0)
    ph = exact._phi(a, Vu[:4], Vt[:4], dt, p.kappa, p.xi, nu, z0[:4])
    np.testing.assert_allclose(ph[:, 0], 1.0, atol=1e-12)
    assert (np.abs(ph) <= 1.0 + 1e-9).all()
    I = exact.sample_integrated_variance(rng, Vu, Vt, dt, p.kappa, p.theta, p.xi)
    # E[int V] = theta dt + (v0 - theta)(1 - e^{-kappa dt}) / kappa (unconditionally)
    ref = p.theta * dt + (p.v0 - p.theta) * (1 - ek) / p.kappa
    assert (I > 0).all()
    assert abs(I.mean() - ref) < 5 * I.std() / math.sqrt(n)


def test_exact_paths_are_discounted_martingales():
    S = exact.simulate(E1, 1.0, 4, 2000, 9)
    t = np.arange(1, 5) / 4
    assert (np.abs(S.mean(axis=0) - 100 * np.exp(E1.r * t)) < 4 * S.std(axis=0) / math.sqrt(2000)).all()


@pytest.mark.parametrize("p", [E1, C1], ids=["paper_table", "base"])
def test_exact_european_matches_closed_form(p):
    m, se = exact.price_delta_rho(p, 100.0, 1.0, 1, 4000, 3)
    ref = cf.heston_price_greeks(100.0, 100.0, 1.0, p.r, p.v0, p.kappa, p.theta, p.xi, p.rho)
    for j, k in enumerate(("price", "delta", "rho")):
        assert abs(m[j] - ref[k]) < 4 * se[j], (k, m[j], ref[k], se[j])


def test_exact_asian_matches_paper_exact_simulation():
    g = json.load(open(os.path.join(GOLDEN, "paper_table1.json")))["asian_4_dates"]
    m, se = exact.price_delta_rho(E1, 100.0, 1.0, 4, 1500, 4, asian=True)
    assert abs(m[0] - g["exact_price"]) < 3 * math.hypot(se[0], g["exact_price_std_error"])
    assert abs(m[1] - g["ex_delta"]) < 4 * se[1]
    assert abs(m[2] - g["ex_rho"]) < 4 * se[2]
    # and the discretised scheme (Milstein, 128 steps) agrees with the exact paths
    mm, mse = oracle.mc_price_greeks(E1, [oracle.Contract(1, 100.0, 1.0, 0, 4)], 1 << 17, 128, 5)
    for j, k in ((0, 0), (1, 1), (2, 4)):
        assert abs(m[j] - mm[0, k]) < 4 * math.hypot(se[j], mse[0, k])
