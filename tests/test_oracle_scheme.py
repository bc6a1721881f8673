"""Pins for the oracle's Milstein scheme, estimators and Monte Carlo driver.

Each test checks the oracle against something the paper or the mathematics
fixes, not against a retyped copy of the oracle:

* one step (N = 1): S_T is exactly lognormal with variance v0*T, so all six
  estimators must reproduce Black-Scholes with sigma^2 = v0;
* zero vol-of-vol: the variance path is deterministic and the scheme's S_T is
  lognormal with total variance dt * sum_k V_k -- a closed form for the
  discrete scheme, derivatives in v0 and T included;
* one step of V: its mean, variance, third central moment and covariance
  with ln S are closed forms of the Milstein update (Sec. 2.4.2), which pins
  the drift, the diffusion, the Milstein term and the correlation step;
* the discrete martingale E[S_ti] = S0 e^{r t_i} (both truncations);
* full-truncation and floor invariants on whole trajectories;
* put-call identities per path; Asian with one date equals European;
* pathwise Greeks against common-random-number finite differences of the
  oracle's own price;
* the paper's printed numbers (tests/golden/paper_table1.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import ASIAN, EUROPEAN, TRUNC_FLOOR, TRUNC_FULL, Contract, Params
from oracle import closed_form as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EST = oracle.ESTIMATORS
CFG1 = Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)


def _paper_params():
    g = json.load(open(os.path.join(GOLDEN, "paper_table1.json")))
    p = g["params"]
    return g, Params(S0=p["S0"], v0=p["v0"], kappa=p["kappa"], theta=p["theta"], xi=p["xi"],
                     rho=p["rho"], r=p["r"])


def _assert_within(mean, se, ref, n_se, label, slack=0.0):
    for j, k in enumerate(EST):
        assert abs(mean[j] - ref[k]) <= n_se * se[j] + slack * max(1.0, abs(ref[k])), (
            f"{label} {k}: mc={mean[j]:.6g} se={se[j]:.3g} ref={ref[k]:.6g}")


# --------------------------------------------------------------------------
# Closed-form limits
# --------------------------------------------------------------------------

@pytest.mark.parametrize("is_put", [0, 1])
def test_one_step_equals_black_scholes(is_put):
    p = Params(S0=100.0, v0=0.05, kappa=3.0, theta=0.02, xi=0.8, rho=-0.6, r=0.04)
    T, K = 0.75, 104.0
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 20, 1, 11)
    ref = cf.bs_total_variance(p.S0, K, T, p.r, p.v0 * T, dw_dv0=T, dw_dT=p.v0, is_put=bool(is_put))
    _assert_within(m[0], se[0], ref, 4.0, "N=1")


def _xi0_reference(p, K, T, N, is_put):
    dt = T / N
    a = 1.0 - p.kappa * dt
    k = np.arange(N)
    V = p.theta + (p.v0 - p.theta) * a**k
    w = dt * V.sum()
    dw_dv0 = dt * (a**k).sum()
    # d/dT at fixed N: dt = T/N and a = 1 - kappa T/N both move
    dV_dT = (p.v0 - p.theta) * k * a**np.maximum(k - 1, 0) * (-p.kappa / N)
    dw_dT = V.sum() / N + dt * dV_dT.sum()
    return cf.bs_total_variance(p.S0, K, T, p.r, w, dw_dv0=dw_dv0, dw_dT=dw_dT, is_put=is_put)


@pytest.mark.parametrize("trunc", [TRUNC_FULL, TRUNC_FLOOR])
@pytest.mark.parametrize("is_put", [0, 1])
def test_zero_vol_of_vol_equals_discrete_black_scholes(trunc, is_put):
    p = Params(S0=100.0, v0=0.09, kappa=2.0, theta=0.04, xi=0.0, rho=-0.5, r=0.03)
    T, K, N = 1.0, 105.0, 16
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 20, N, 5, trunc)
    ref = _xi0_reference(p, K, T, N, bool(is_put))
    _assert_within(m[0], se[0], ref, 4.0, "xi=0")


def test_one_step_variance_moments_pin_milstein_update():
    p = Params(S0=100.0, v0=0.04, kappa=1.5, theta=0.06, xi=1.0, rho=-0.6, r=0.02)
    T = 0.5
    n = 1 << 17
    rec, _ = oracle.debug_paths(p, [Contract(EUROPEAN, 100.0, T)], np.arange(n), 1, 3)
    X, V = rec[:, 0], rec[:, 1]
    b = p.xi * math.sqrt(p.v0 * T)          # diffusion coefficient of the step
    c = 0.25 * p.xi**2 * T                  # Milstein coefficient
    mu = p.v0 + p.kappa * (p.theta - p.v0) * T
    mux = (p.r - 0.5 * p.v0) * T
    checks = {
        "mean": (V - mu, 0.0),
        "var": ((V - mu) ** 2, b * b + 2 * c * c),
        "m3": ((V - mu) ** 3, 6 * b * b * c + 8 * c**3),
        "cov": ((X - mux) * (V - mu), math.sqrt(p.v0 * T) * b * p.rho),
    }
    for name, (sample, ref) in checks.items():
        se = sample.std() / math.sqrt(n)
        assert abs(sample.mean() - ref) < 5 * se, (name, sample.mean(), ref, se)


def test_mean_variance_follows_linear_recursion():
    # little truncation: E[V_N] = theta + (v0 - theta)(1 - kappa dt)^N
    p = Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.09, xi=0.1, rho=-0.3, r=0.01)
    T, N, n = 1.0, 8, 1 << 16
    rec, _ = oracle.debug_paths(p, [Contract(EUROPEAN, 100.0, T)], np.arange(n), N, 9)
    V = rec[:, 1]
    ref = p.theta + (p.v0 - p.theta) * (1 - p.kappa * T / N) ** N
    assert abs(V.mean() - ref) < 5 * V.std() / math.sqrt(n)


# --------------------------------------------------------------------------
# Martingale, truncation invariants, identities
# --------------------------------------------------------------------------

@pytest.mark.parametrize("trunc", [TRUNC_FULL, TRUNC_FLOOR])
def test_discrete_martingale(trunc):
    _, p = _paper_params()          # Feller-violating set: truncation is active
    T, N, M = 1.0, 32, 8
    cs = [Contract(EUROPEAN, 0.0, T), Contract(ASIAN, 0.0, T, n_monitor=M)]
    m, se = oracle.mc_price_greeks(p, cs, 1 << 18, N, 21, trunc)
    D = math.exp(-p.r * T)
    ref_e = p.S0
    ref_a = D * np.mean([p.S0 * math.exp(p.r * i * T / M) for i in range(1, M + 1)])
    assert abs(m[0, 0] - ref_e) < 4 * se[0, 0]
    assert abs(m[1, 0] - ref_a) < 4 * se[1, 0]
    # with K = 0 the pathwise Delta is the price over S0 on every path
    assert abs(m[0, 1] - m[0, 0] / p.S0) < 1e-12
    assert abs(m[1, 1] - m[1, 0] / p.S0) < 1e-12


def test_truncation_invariants_on_trajectories():
    _, p = _paper_params()
    T, N = 1.0, 64
    dt = T / N
    cs = [Contract(EUROPEAN, 100.0, T)]
    n_neg = n_zero = 0
    for path in range(300):
        za, zb = oracle.path_normals(4, path, N)
        _, _, X, V = oracle.path_from_normals(p, cs, za, zb, TRUNC_FULL)
        for k in range(N):
            if V[k] <= 0.0:
                n_neg += 1
                # full truncation: a non-positive state only drifts up by kappa theta dt,
                # and ln S moves by r dt alone
                assert abs(V[k + 1] - V[k] - p.kappa * p.theta * dt) < 1e-15
                assert abs(X[k + 1] - X[k] - p.r * dt) < 1e-15
        _, _, Xf, Vf = oracle.path_from_normals(p, cs, za, zb, TRUNC_FLOOR)
        assert (Vf >= 0.0).all()
        n_zero += int((Vf == 0.0).sum())
        # both schemes agree until the first step where V leaves (0, inf)
        first = next((k for k in range(N + 1) if V[k] <= 0.0), N + 1)
        assert np.array_equal(V[:first], Vf[:first])
    assert n_neg > 0 and n_zero > 0


@pytest.mark.parametrize("payoff,M", [(EUROPEAN, 0), (ASIAN, 4)])
def test_put_call_identities_per_path(payoff, M):
    p = CFG1
    T, K, N = 1.0, 100.0, 32
    cs = [Contract(payoff, K, T, 0, M), Contract(payoff, K, T, 1, M)]
    rec, est = oracle.debug_paths(p, cs, np.arange(4096), N, 2)
    f = {k: rec[:, i] for i, k in enumerate(oracle.PATH_FIELDS)}
    D = math.exp(-p.r * T)
    sq = math.sqrt(1 - p.rho**2)
    if payoff == EUROPEAN:
        A = p.S0 * np.exp(f["X"])
        dA_v, dA_T, dA_r = A * f["X_v"], A * f["X_T"], T * A
        lr = f["GE"] / (sq * f["QE"])
    else:
        A = f["sumS"] / M
        dA_v, dA_T, dA_r = f["sumS_Xv"] / M, f["sumS_XT"] / M, f["sumtS"] / M
        lr = f["GA"] / (sq * f["QA"])
    c, q = est[:, 0, :], est[:, 1, :]
    ok = np.abs(A - K) > 1e-9
    tol = dict(rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose((c[:, 0] - q[:, 0])[ok], (D * (A - K))[ok], **tol)
    np.testing.assert_allclose((c[:, 1] - q[:, 1])[ok], (D * A / p.S0)[ok], **tol)
    np.testing.assert_allclose((c[:, 2] - q[:, 2])[ok], (D * A / p.S0**2 * (lr - 1))[ok], **tol)
    np.testing.assert_allclose((c[:, 3] - q[:, 3])[ok], (D * dA_v)[ok], **tol)
    np.testing.assert_allclose((c[:, 4] - q[:, 4])[ok], (D * dA_r - T * D * (A - K))[ok], **tol)
    np.testing.assert_allclose((c[:, 5] - q[:, 5])[ok], (p.r * D * (A - K) - D * dA_T)[ok], **tol)


@pytest.mark.parametrize("is_put", [0, 1])
def test_asian_with_one_date_equals_european(is_put):
    p = CFG1
    T, K, N = 1.0, 95.0, 20
    cs = [Contract(EUROPEAN, K, T, is_put), Contract(ASIAN, K, T, is_put, n_monitor=1)]
    _, est = oracle.debug_paths(p, cs, np.arange(2048), N, 8)
    np.testing.assert_allclose(est[:, 1, :], est[:, 0, :], rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Pathwise Greeks against common-random-number finite differences
# --------------------------------------------------------------------------

def _price(p, c, n, N, seed):
    m, _ = oracle.mc_price_greeks(p, [c], n, N, seed)
    return m[0, 0]


@pytest.mark.parametrize("payoff,M", [(EUROPEAN, 0), (ASIAN, 8)])
@pytest.mark.parametrize("is_put", [0, 1])
def test_pathwise_greeks_match_crn_finite_differences(payoff, M, is_put):
    p = CFG1
    T, K, N, n, seed = 1.0, 100.0, 32, 1 << 15, 13
    c = Contract(payoff, K, T, is_put, M)
    m, _ = oracle.mc_price_greeks(p, [c], n, N, seed)
    m = dict(zip(EST, m[0]))
    h = 1e-4

    def fd(field, x):
        hp = h * abs(x)
        if field == "T":
            up = _price(p, Contract(payoff, K, T + hp, is_put, M), n, N, seed)
            dn = _price(p, Contract(payoff, K, T - hp, is_put, M), n, N, seed)
        else:
            up = _price(p.replace(**{field: x + hp}), c, n, N, seed)
            dn = _price(p.replace(**{field: x - hp}), c, n, N, seed)
        return (up - dn) / (2 * hp)

    checks = {"delta": fd("S0", p.S0), "vega": fd("v0", p.v0), "rho": fd("r", p.r),
              "theta": -fd("T", T)}
    for k, v in checks.items():
        assert abs(m[k] - v) <= 2e-3 * max(1.0, abs(m[k])), (k, m[k], v)


# --------------------------------------------------------------------------
# Against the Heston closed form and the paper's printed values
# --------------------------------------------------------------------------

@pytest.mark.parametrize("is_put", [0, 1])
def test_milstein_matches_heston_closed_form(is_put):
    p = CFG1
    T, K, N = 1.0, 100.0, 100
    m, se = oracle.mc_price_greeks(p, [Contract(EUROPEAN, K, T, is_put)], 1 << 20, N, 42)
    ref = cf.heston_price_greeks(p.S0, K, T, p.r, p.v0, p.kappa, p.theta, p.xi, p.rho,
                                 is_put=bool(is_put))
    _assert_within(m[0], se[0], ref, 4.0, "closed form", slack=2e-3)


def test_paper_printed_milstein_estimates():
    g, p = _paper_params()
    a = g["asian_4_dates"]
    T, K, N = g["params"]["T"], g["params"]["K"], a["n_steps"]
    cs = [Contract(ASIAN, K, T, 0, len(a["monitoring_dates"])), Contract(EUROPEAN, K, T)]
    m, se = oracle.mc_price_greeks(p, cs, 1 << 19, N, 7)
    # Asian price against the exact-simulation QMC value and its printed std error
    band = 3 * math.hypot(se[0, 0], a["exact_price_std_error"])
    assert abs(m[0, 0] - a["exact_price"]) < band
    # Asian Delta and Rho against the exact-simulation Greeks (no std error printed)
    assert abs(m[0, 1] - a["ex_delta"]) < a["ex_band_rel"] * a["ex_delta"]
    assert abs(m[0, 4] - a["ex_rho"]) < a["ex_band_rel"] * a["ex_rho"]
    # European against the analytic values
    e = g["european_closed_form"]
    assert abs(m[1, 0] - e["price"]) < 4 * se[1, 0] + 0.01
    assert abs(m[1, 1] - e["delta"]) < 4 * se[1, 1] + 1e-3
    assert abs(m[1, 4] - e["rho"]) < 4 * se[1, 4] + 0.05


def test_thread_count_does_not_change_bits():
    cs = [Contract(EUROPEAN, 100.0, 1.0), Contract(ASIAN, 100.0, 1.0)]
    a = oracle.mc_sums(CFG1, cs, 10000, 12, 3, n_threads=1)
    b = oracle.mc_sums(CFG1, cs, 10000, 12, 3, n_threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_invalid_inputs_are_rejected():
    with pytest.raises(ValueError):
        oracle.mc_price_greeks(CFG1, [Contract(EUROPEAN, 100.0, 1.0),
                                      Contract(EUROPEAN, 100.0, 2.0)], 100, 10, 1)
    with pytest.raises(ValueError):
        oracle.mc_price_greeks(CFG1, [Contract(ASIAN, 100.0, 1.0, 0, 3)], 100, 10, 1)
