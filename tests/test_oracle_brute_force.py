"""Brute-force pin of the oracle on tiny inputs: N in {1, 2} steps and
n_paths in {1, 2, 3}, with the Milstein step of Sec. 2.4.2 (full truncation
and the paper's floor), the correlation of Sec. 2.4.1, the tangents, the
Gamma weights and the six per-path estimators of Eq. (euro_pw) /
Eq. (asian_pw) (Asian Rho without the printed K*T factor) written out by
hand below -- each step spelled out, no loop -- and the Monte Carlo mean and
standard error of Sec. 2.5 formed from the per-path values.  The oracle
must agree to 1e-14 relative.

Normals come from the oracle's Philox4x32-10 / Box-Muller (pinned to
cuRAND separately) and from hand-picked values that drive the variance
negative, so that the truncation branches are exercised.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_10477_gb300 import workloads as wl

TOL = 1e-14

PARAMS = {
    "base": wl.BASE_PARAMS,
    "paper": wl.PAPER_PARAMS,
    # large vol-of-vol: the variance goes negative after one step for the picked normals
    "wild": dict(S0=100.0, v0=0.01, kappa=1.5, theta=0.02, xi=1.8, rho=-0.6, r=0.04),
}


def _close(a, b, tol=TOL):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b)))


def two_steps_by_hand(p, T, N, Za, Zb, floor):
    """X, V and tangents after N = 1 or 2 Milstein steps, with the Gamma
    weights and the per-step X tangents (for the Asian dates).  Returns a
    dict of the oracle record fields plus the states after each step."""
    S0, v0, ka, th, xi, rho, r = (p[k] for k in ("S0", "v0", "kappa", "theta", "xi", "rho", "r"))
    dt, ddt = T / N, 1.0 / N
    s = math.sqrt(1.0 - rho * rho)
    c4, c4T = 0.25 * xi * xi * dt, 0.25 * xi * xi * ddt

    # ---- step 1 (k = 0): V0 = v0 > 0 -------------------------------------
    za0, zb0 = Za[0], Zb[0]
    z2_0 = rho * za0 + s * zb0                      # correlated normal
    w_0 = s * za0 - rho * zb0                       # part of Z1 orthogonal to Z2
    u0 = math.sqrt(v0 * dt)
    u0_v = dt / (2.0 * u0)                          # d/dv0 of sqrt(v0 dt)
    u0_T = v0 * ddt / (2.0 * u0)                    # d/dT of sqrt(v0 T / N)
    X1 = (r - 0.5 * v0) * dt + u0 * za0
    X1_v = -0.5 * dt + u0_v * za0
    X1_T = (r - 0.5 * v0) * ddt + u0_T * za0
    V1 = v0 + ka * (th - v0) * dt + xi * u0 * z2_0 + c4 * (z2_0 * z2_0 - 1.0)
    V1_v = 1.0 - ka * dt + xi * u0_v * z2_0
    V1_T = ka * (th - v0) * ddt + xi * u0_T * z2_0 + c4T * (z2_0 * z2_0 - 1.0)
    minV = min(abs(v0), abs(V1))
    V1_before_floor = V1
    if floor and V1 <= 0.0:                         # the paper's max(V, 0) after the update
        V1, V1_v, V1_T = 0.0, 0.0, 0.0
    G1, Q1 = u0 * w_0, v0 * dt
    out = dict(X1=X1, X1_v=X1_v, X1_T=X1_T, V1=V1_before_floor)
    if N == 1:
        out.update(X=X1, V=V1, X_v=X1_v, V_v=V1_v, X_T=X1_T, V_T=V1_T, GE=G1, QE=Q1, minabsV=minV)
        return out

    # ---- step 2 (k = 1): the pre-update variance may be <= 0 -------------
    za1, zb1 = Za[1], Zb[1]
    z2_1 = rho * za1 + s * zb1
    w_1 = s * za1 - rho * zb1
    pos = V1 > 0.0
    V1p = V1 if pos else 0.0
    V1p_v = V1_v if pos else 0.0
    V1p_T = V1_T if pos else 0.0
    u1 = math.sqrt(V1p * dt)
    u1_v = V1p_v * dt / (2.0 * u1) if u1 > 0.0 else 0.0
    u1_T = (V1p_T * dt + V1p * ddt) / (2.0 * u1) if u1 > 0.0 else 0.0
    X2 = X1 + (r - 0.5 * V1p) * dt + u1 * za1
    X2_v = X1_v - 0.5 * V1p_v * dt + u1_v * za1
    X2_T = X1_T + (r - 0.5 * V1p) * ddt - 0.5 * V1p_T * dt + u1_T * za1
    if not floor:
        mil = 1.0 if pos else 0.0                   # full truncation: the Milstein term needs V > 0
        V2 = V1 + ka * (th - V1p) * dt + xi * u1 * z2_1 + c4 * (z2_1 * z2_1 - 1.0) * mil
        V2_v = V1_v - ka * V1p_v * dt + xi * u1_v * z2_1
        V2_T = (V1_T + ka * (th - V1p) * ddt - ka * V1p_T * dt + xi * u1_T * z2_1
                + c4T * (z2_1 * z2_1 - 1.0) * mil)
        minV = min(minV, abs(V2))
    else:                                           # V1 >= 0 here
        Vt = V1 + ka * (th - V1) * dt + xi * u1 * z2_1 + c4 * (z2_1 * z2_1 - 1.0)
        Vt_v = V1_v - ka * V1_v * dt + xi * u1_v * z2_1
        Vt_T = (V1_T + ka * (th - V1) * ddt - ka * V1_T * dt + xi * u1_T * z2_1
                + c4T * (z2_1 * z2_1 - 1.0))
        minV = min(minV, abs(Vt))
        keep = Vt > 0.0
        V2, V2_v, V2_T = (Vt, Vt_v, Vt_T) if keep else (0.0, 0.0, 0.0)
    out.update(X=X2, V=V2, X_v=X2_v, V_v=V2_v, X_T=X2_T, V_T=V2_T,
               GE=G1 + u1 * w_1, QE=Q1 + V1p * dt, G1=G1, Q1=Q1, minabsV=minV)
    return out


def record_by_hand(p, T, N, M, Za, Zb, floor):
    """The oracle's 15-field record: Asian sums over the M dates (N = M or M = 1)."""
    h = two_steps_by_hand(p, T, N, Za, Zb, floor)
    S0, dt = p["S0"], T / N
    if M == N == 2:
        S1, S2 = S0 * math.exp(h["X1"]), S0 * math.exp(h["X"])
        sumS, sumtS = S1 + S2, dt * S1 + 2.0 * dt * S2
        sumS_Xv, sumS_XT = S1 * h["X1_v"] + S2 * h["X_v"], S1 * h["X1_T"] + S2 * h["X_T"]
        GA, QA = h["G1"], h["Q1"]                  # steps before the first date: step 1 only
    else:                                          # one date, at T
        ST = S0 * math.exp(h["X"])
        sumS, sumtS, sumS_Xv, sumS_XT = ST, N * dt * ST, ST * h["X_v"], ST * h["X_T"]
        GA, QA = h["GE"], h["QE"]
    return np.array([h["X"], h["V"], h["X_v"], h["V_v"], h["X_T"], h["V_T"], sumS, sumtS,
                     sumS_Xv, sumS_XT, h["GE"], h["QE"], GA, QA, h["minabsV"]])


def estimators_by_hand(p, contract, N, rec):
    """Price, Delta, Gamma, Vega (d/dv0), Rho, Theta (-d/dT) of one path."""
    payoff, K, T, put, Mc = contract
    S0, r, rho = p["S0"], p["r"], p["rho"]
    D = math.exp(-r * T)
    s = math.sqrt(1.0 - rho * rho)
    X, X_v, X_T, sumS, sumtS, sumS_Xv, sumS_XT, GE, QE, GA, QA = (
        rec[0], rec[2], rec[4], rec[6], rec[7], rec[8], rec[9], rec[10], rec[11], rec[12], rec[13])
    M = Mc or N
    if payoff == 0:
        A = S0 * math.exp(X)
        dA_v, dA_T = A * X_v, A * X_T
        lr = GE / (s * QE)
    else:
        A = sumS / M
        dA_v, dA_T = sumS_Xv / M, sumS_XT / M
        lr = GA / (s * QA)
    if not put:
        ind = 1.0 if A > K else 0.0
        pay = A - K if A > K else 0.0
        sign = 1.0
    else:
        ind = 1.0 if A < K else 0.0
        pay = K - A if A < K else 0.0
        sign = -1.0
    price = D * pay
    delta = sign * D * (A / S0) * ind
    gamma = sign * D * ind * (A / (S0 * S0)) * (lr - 1.0)
    vega = sign * D * ind * dA_v
    if payoff == 0:
        rho_ = sign * D * K * T * ind                       # Eq. (euro_pw)
    else:
        rho_ = sign * D * ind * (sumtS / M - T * (A - K))   # d/dr of e^{-rT} (Sbar - K)+
    theta = r * price - sign * D * ind * dA_T
    return np.array([price, delta, gamma, vega, rho_, theta])


CONTRACTS = [(0, 100.0, 1.0, 0, 0), (0, 100.0, 1.0, 1, 0), (1, 98.0, 1.0, 0, 0), (1, 102.0, 1.0, 1, 0),
             (0, 60.0, 1.0, 0, 0), (0, 150.0, 1.0, 1, 0)]


def _oc(cs):
    return [oracle.Contract(*c) for c in cs]


@pytest.mark.parametrize("floor", [0, 1])
@pytest.mark.parametrize("name", sorted(PARAMS))
@pytest.mark.parametrize("N", [1, 2])
def test_per_path_records_and_estimators_by_hand(name, N, floor):
    p = PARAMS[name]
    seed = 2309
    for path in range(3):
        Za, Zb = oracle.path_normals(seed, path, N)
        rec_o, est_o = oracle.debug_paths(oracle.Params(**p), _oc(CONTRACTS), [path], N, seed, floor)
        rec_h = record_by_hand(p, 1.0, N, N, Za, Zb, floor)
        assert _close(rec_o[0], rec_h), (path, rec_o[0] - rec_h)
        for ci, c in enumerate(CONTRACTS):
            assert _close(est_o[0, ci], estimators_by_hand(p, c, N, rec_h)), (path, c)


# picked normals: (Za, Zb) per step; with the "wild" set the first pair
# drives V below zero, so the second step runs on V+ = 0
PICKED = [
    ([0.3, -1.2], [1.1, 0.4]),
    ([-2.4, 0.7], [-1.9, -0.2]),
    ([1.7, 2.2], [0.05, -2.6]),
    ([-0.1, -0.3], [2.8, 1.5]),
]


@pytest.mark.parametrize("floor", [0, 1])
@pytest.mark.parametrize("name", sorted(PARAMS))
def test_picked_normals_through_both_branches(name, floor):
    p = PARAMS[name]
    P = oracle.Params(**p)
    went_negative = 0
    for Za, Zb in PICKED:
        for M, cs in ((2, CONTRACTS), (1, [(c[0], c[1], c[2], c[3], 1) for c in CONTRACTS])):
            rec_o, est_o, tx, tv = oracle.path_from_normals(P, _oc(cs), np.array(Za), np.array(Zb), floor)
            rec_h = record_by_hand(p, 1.0, 2, M, Za, Zb, floor)
            assert _close(rec_o, rec_h), (Za, Zb, M, rec_o - rec_h)
            for ci, c in enumerate(cs):
                assert _close(est_o[ci], estimators_by_hand(p, c, 2, rec_h)), (Za, Zb, c)
        h = two_steps_by_hand(p, 1.0, 2, Za, Zb, floor)
        went_negative += h["V1"] < 0.0
        assert np.isfinite(h["X"])
    if name == "wild":
        assert went_negative >= 1          # the truncation branch was exercised


@pytest.mark.parametrize("begin", [0, 2**32 - 2])
@pytest.mark.parametrize("n_paths", [1, 2, 3])
@pytest.mark.parametrize("N", [1, 2])
def test_monte_carlo_sums_mean_and_se_by_hand(n_paths, N, begin):
    """Alg. "Monte Carlo option pricing estimation": sum over the paths, then
    mean = sum / n and SE = sqrt((sum x^2 - n mean^2) / (n - 1) / n).  A range
    of paths [begin, begin + n) sums the paths of those global indices (the
    contract a path-range shard relies on), here across the low counter
    word's wrap at 2^32."""
    p = PARAMS["paper"]
    seed = 77
    cs = CONTRACTS[:4]
    est = []
    for path in range(begin, begin + n_paths):
        Za, Zb = oracle.path_normals(seed, path, N)
        rec = record_by_hand(p, 1.0, N, N, Za, Zb, 0)
        est.append([estimators_by_hand(p, c, N, rec) for c in cs])
    est = np.array(est)                              # (n, C, 6)
    s_h = est.sum(axis=0)
    s2_h = (est * est).sum(axis=0)
    s_o, s2_o = oracle.mc_sums(oracle.Params(**p), _oc(cs), n_paths, N, seed, path_begin=begin)
    assert _close(s_o, s_h) and _close(s2_o, s2_h)
    if n_paths >= 2 and begin == 0:
        mean_h = s_h / n_paths
        se_h = np.sqrt(np.maximum((s2_h - n_paths * mean_h * mean_h) / (n_paths - 1), 0.0) / n_paths)
        mean_o, se_o = oracle.mc_price_greeks(oracle.Params(**p), _oc(cs), n_paths, N, seed)
        assert _close(mean_o, mean_h)
        assert np.all(np.abs(se_o - se_h) <= 1e-12 * np.maximum(1.0, se_h))
