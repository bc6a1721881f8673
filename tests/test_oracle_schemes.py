"""Pins for the oracle's Euler (Sec. 2.4.1) and Andersen QE schemes.

As for the Milstein scheme, each check is against something the mathematics
fixes, not a retyped copy of the oracle:

* Euler, one step: S_T is lognormal with variance v0*T (Black-Scholes); the
  variance step has the Gaussian moments of the Euler update and no third
  moment (the Milstein term is what creates one); the discrete martingale
  E[S_T] = S0 e^{rT}; the Heston closed form at fine steps.
* QE, one step: the mean and variance of V(t+dt) equal those of the exact
  CIR transition, a scaled noncentral chi-square (scipy.stats.ncx2), in the
  quadratic and in the exponential branch.
* QE with rho = 0 and a tiny vol-of-vol: the variance path is the ODE
  solution and ln S_T is Gaussian with the trapezoidal integrated variance,
  a closed form with its v0- and T-derivatives.
* QE at a coarse grid against the Heston closed form (all six Greeks).
* Both: pathwise tangents per path against central differences on the same
  normals; put-call identities and Asian-with-one-date per path.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import (ASIAN, EUROPEAN, SCHEME_EULER, SCHEME_MILSTEIN, SCHEME_QE, TRUNC_FLOOR,
                    TRUNC_FULL, Contract, Params)
from oracle import closed_form as cf

EST = oracle.ESTIMATORS
CFG1 = Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)
# far from the Feller condition: 2 kappa theta = 0.02 < xi^2 = 1
ROUGH = Params(S0=100.0, v0=0.01, kappa=0.5, theta=0.02, xi=1.0, rho=-0.7, r=0.05)


def _assert_within(mean, se, ref, n_se, label, slack=0.0):
    for j, k in enumerate(EST):
        assert abs(mean[j] - ref[k]) <= n_se * se[j] + slack * max(1.0, abs(ref[k])), (
            f"{label} {k}: mc={mean[j]:.6g} se={se[j]:.3g} ref={ref[k]:.6g}")


def _heston(p, K, T, is_put):
    return cf.heston_price_greeks(p.S0, K, T, p.r, p.v0, p.kappa, p.theta, p.xi, p.rho,
                                  is_put=bool(is_put))


# --------------------------------------------------------------------------
# Euler
# --------------------------------------------------------------------------

@pytest.mark.parametrize("is_put", [0, 1])
def test_euler_one_step_equals_black_scholes(is_put):
    p = Params(S0=100.0, v0=0.05, kappa=3.0, theta=0.02, xi=0.8, rho=-0.6, r=0.04)
    T, K = 0.75, 104.0
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 20, 1, 11,
                                   scheme=SCHEME_EULER)
    ref = cf.bs_total_variance(p.S0, K, T, p.r, p.v0 * T, dw_dv0=T, dw_dT=p.v0, is_put=bool(is_put))
    _assert_within(m[0], se[0], ref, 4.0, "Euler N=1")


def test_euler_one_step_variance_moments():
    p = Params(S0=100.0, v0=0.04, kappa=1.5, theta=0.06, xi=1.0, rho=-0.6, r=0.02)
    T = 0.5
    n = 1 << 17
    rec, _ = oracle.debug_paths(p, [Contract(EUROPEAN, 100.0, T)], np.arange(n), 1, 3,
                                scheme=SCHEME_EULER)
    X, V = rec[:, 0], rec[:, 1]
    b = p.xi * math.sqrt(p.v0 * T)          # diffusion coefficient of the step
    mu = p.v0 + p.kappa * (p.theta - p.v0) * T
    mux = (p.r - 0.5 * p.v0) * T
    checks = {
        "mean": (V - mu, 0.0),
        "var": ((V - mu) ** 2, b * b),
        "m3": ((V - mu) ** 3, 0.0),          # Gaussian step: no skew
        "cov": ((X - mux) * (V - mu), math.sqrt(p.v0 * T) * b * p.rho),
    }
    for name, (sample, ref) in checks.items():
        se = sample.std() / math.sqrt(n)
        assert abs(sample.mean() - ref) < 5 * se, (name, sample.mean(), ref, se)


@pytest.mark.parametrize("trunc", [TRUNC_FULL, TRUNC_FLOOR])
def test_euler_discrete_martingale(trunc):
    p = ROUGH
    T, N = 1.0, 32
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, 0.0, T)], 1 << 18, N, 21, trunc,
                                   scheme=SCHEME_EULER)
    assert abs(m[0, 0] - p.S0) < 4 * se[0, 0]


def test_euler_differs_from_milstein_only_in_the_variance_term():
    """Same normals: ln S agrees until the variance paths part, and one step
    of V differs by exactly the Milstein term's contribution to the sample
    third moment (checked above), so here only the first step of ln S."""
    p = CFG1
    cs = [Contract(EUROPEAN, 100.0, 1.0)]
    za, zb = oracle.path_normals(5, 3, 16)
    _, _, Xm, Vm = oracle.path_from_normals(p, cs, za, zb, scheme=SCHEME_MILSTEIN)
    _, _, Xe, Ve = oracle.path_from_normals(p, cs, za, zb, scheme=SCHEME_EULER)
    assert Xm[1] == Xe[1] and Vm[0] == Ve[0]
    assert Vm[1] != Ve[1]


@pytest.mark.parametrize("is_put", [0, 1])
def test_euler_matches_heston_closed_form(is_put):
    p, T, K = CFG1, 1.0, 100.0
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 18, 128, 17,
                                   scheme=SCHEME_EULER)
    # weak order one: the remaining bias at dt = 1/128 is below 0.5 % here
    _assert_within(m[0], se[0], _heston(p, K, T, is_put), 3.0, "Euler", slack=5e-3)


# --------------------------------------------------------------------------
# QE
# --------------------------------------------------------------------------

def _cir_moments(p, V, dt):
    """Mean and variance of V(t+dt) | V(t) = V from scipy's noncentral chi-square."""
    e = math.exp(-p.kappa * dt)
    c = p.xi**2 * (1.0 - e) / (4.0 * p.kappa)
    d = 4.0 * p.kappa * p.theta / p.xi**2
    lam = V * e / c
    return c * stats.ncx2.mean(d, lam), c * c * stats.ncx2.var(d, lam)


# (V(t), dt): quadratic branch (psi = 0.25, 1.24), exponential branch (4.7, 50)
ONE_STEP_CASES = [(0.2, 0.05), (0.04, 0.05), (0.01, 0.05), (1e-5, 0.25)]


@pytest.mark.parametrize("V0,T", ONE_STEP_CASES)
def test_qe_one_step_matches_cir_moments(V0, T):
    p = ROUGH.replace(v0=V0)
    mean, var = _cir_moments(p, V0, T)
    n = 1 << 20
    g = np.random.Generator(np.random.PCG64(99))
    za, zb = g.standard_normal((n, 1)), g.standard_normal((n, 1))
    rec, _ = oracle.paths_from_normals(p, [Contract(EUROPEAN, 100.0, T)], za, zb, scheme=SCHEME_QE)
    Vn = rec[:, 1]
    assert (Vn >= 0.0).all()
    se_mean = Vn.std() / math.sqrt(n)
    assert abs(Vn.mean() - mean) < 5 * se_mean, (Vn.mean(), mean, se_mean)
    d2 = (Vn - mean) ** 2
    assert abs(d2.mean() - var) < 5 * d2.std() / math.sqrt(n), (d2.mean(), var)


def test_qe_one_step_cases_cover_both_branches():
    # psi = var / mean^2 of the exact transition decides the branch (1.5)
    psis = [v / m**2 for m, v in (_cir_moments(ROUGH, V0, T) for V0, T in ONE_STEP_CASES)]
    assert max(psis[:2]) < 1.5 < min(psis[2:])


def _trapezoid_reference(p, K, T, N, is_put):
    """rho = 0, xi -> 0: V_k = theta + (v0 - theta) e^{-kappa t_k} and ln S_T is
    Gaussian with total variance w = sum_k dt (V_k + V_{k+1}) / 2."""
    k = np.arange(N + 1)
    t = T * k / N
    e = np.exp(-p.kappa * t)
    V = p.theta + (p.v0 - p.theta) * e
    trap = lambda f: (T / N) * 0.5 * (f[:-1] + f[1:]).sum()
    w = trap(V)
    dw_dv0 = trap(e)
    # d/dT at fixed N: t_k = k T / N moves with T
    dV_dT = (p.v0 - p.theta) * e * (-p.kappa * k / N)
    dw_dT = w / T + trap(dV_dT)
    return cf.bs_total_variance(p.S0, K, T, p.r, w, dw_dv0=dw_dv0, dw_dT=dw_dT, is_put=is_put)


@pytest.mark.parametrize("is_put", [0, 1])
def test_qe_small_vol_of_vol_equals_trapezoid_black_scholes(is_put):
    p = Params(S0=100.0, v0=0.09, kappa=2.0, theta=0.04, xi=1e-3, rho=0.0, r=0.03)
    T, K, N = 1.0, 105.0, 8
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 19, N, 5,
                                   scheme=SCHEME_QE)
    ref = _trapezoid_reference(p, K, T, N, bool(is_put))
    _assert_within(m[0], se[0], ref, 4.0, "QE xi->0", slack=1e-5)


@pytest.mark.parametrize("is_put", [0, 1])
@pytest.mark.parametrize("p", [CFG1, ROUGH], ids=["feller", "rough"])
def test_qe_coarse_grid_matches_heston_closed_form(p, is_put):
    T, K = 1.0, 100.0
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 18, 32, 23,
                                   scheme=SCHEME_QE)
    ref = _heston(p, K, T, is_put)
    _assert_within(m[0], se[0], ref, 3.5, "QE N=32", slack=5e-3)


def test_qe_rejects_degenerate_parameters():
    cs = [Contract(EUROPEAN, 100.0, 1.0)]
    for bad in (CFG1.replace(xi=0.0), CFG1.replace(kappa=0.0), CFG1.replace(theta=0.0)):
        with pytest.raises(ValueError):
            oracle.mc_price_greeks(bad, cs, 64, 4, 1, scheme=SCHEME_QE)
    with pytest.raises(ValueError):
        oracle.mc_price_greeks(CFG1, cs, 64, 4, 1, scheme=7)


# --------------------------------------------------------------------------
# Both schemes: tangents, identities
# --------------------------------------------------------------------------

@pytest.mark.parametrize("scheme,trunc", [(SCHEME_EULER, TRUNC_FULL), (SCHEME_EULER, TRUNC_FLOOR),
                                          (SCHEME_QE, TRUNC_FULL)])
@pytest.mark.parametrize("p", [CFG1, ROUGH], ids=["feller", "rough"])
def test_tangents_match_central_differences_per_path(p, scheme, trunc):
    N, h = 16, 1e-8
    cs = [Contract(EUROPEAN, 100.0, 1.0), Contract(ASIAN, 100.0, 1.0, 0, 4)]
    shift = lambda dT: [Contract(c.payoff, c.K, c.T + dT, c.is_put, c.n_monitor) for c in cs]
    run = lambda q, c, za, zb: oracle.path_from_normals(q, c, za, zb, trunc, scheme)[0]
    checked = 0
    for path in range(200):
        za, zb = oracle.path_normals(7, path, N)
        rec = run(p, cs, za, zb)
        if rec[14] < 1e-4 * p.theta:          # a branch decision inside the difference window
            continue
        up, dn = run(p.replace(v0=p.v0 + h), cs, za, zb), run(p.replace(v0=p.v0 - h), cs, za, zb)
        tu, td = run(p, shift(h), za, zb), run(p, shift(-h), za, zb)
        for i, fd in ((2, (up[0] - dn[0]) / (2 * h)), (3, (up[1] - dn[1]) / (2 * h)),
                      (8, (up[6] - dn[6]) / (2 * h)),
                      (4, (tu[0] - td[0]) / (2 * h)), (5, (tu[1] - td[1]) / (2 * h)),
                      (9, (tu[6] - td[6]) / (2 * h))):
            assert abs(rec[i] - fd) <= 2e-5 * max(1.0, abs(fd)), (path, oracle.PATH_FIELDS[i], rec[i], fd)
        checked += 1
    assert checked >= 150


@pytest.mark.parametrize("scheme", [SCHEME_EULER, SCHEME_QE])
@pytest.mark.parametrize("payoff,M", [(EUROPEAN, 0), (ASIAN, 4)])
def test_put_call_identities_per_path(scheme, payoff, M):
    p = CFG1
    T, K, N = 1.0, 100.0, 32
    cs = [Contract(payoff, K, T, 0, M), Contract(payoff, K, T, 1, M)]
    rec, est = oracle.debug_paths(p, cs, np.arange(2048), N, 2, scheme=scheme)
    f = {k: rec[:, i] for i, k in enumerate(oracle.PATH_FIELDS)}
    D = math.exp(-p.r * T)
    A = p.S0 * np.exp(f["X"]) if payoff == EUROPEAN else f["sumS"] / M
    c, q = est[:, 0, :], est[:, 1, :]
    ok = np.abs(A - K) > 1e-9
    np.testing.assert_allclose((c[:, 0] - q[:, 0])[ok], (D * (A - K))[ok], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose((c[:, 1] - q[:, 1])[ok], (D * A / p.S0)[ok], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("scheme", [SCHEME_EULER, SCHEME_QE])
def test_asian_with_one_date_equals_european(scheme):
    p = CFG1
    T, K, N = 1.0, 95.0, 20
    cs = [Contract(EUROPEAN, K, T, 0), Contract(ASIAN, K, T, 0, n_monitor=1)]
    _, est = oracle.debug_paths(p, cs, np.arange(1024), N, 8, scheme=scheme)
    np.testing.assert_allclose(est[:, 1, :], est[:, 0, :], rtol=1e-12, atol=1e-12)
