"""How well-conditioned an estimate is for an FP32 path, measured with the
oracle.

An FP32 path rounds every input (S0, K, T, v0, kappa, theta, xi, rho, r) to
FP32, and its normals differ from the FP64 ones by up to 1e-7 + 1.5e-6 R
(R = sqrt(Za^2 + Zb^2); the bound the random-number parity test holds the
FP32 Box-Muller to), before any rounding of the path arithmetic itself.  The
oracle measures how far its own estimates move under exactly that:

    delta = max over DRAWS draws |o(p) - o~(fl32(p))| / max(1, |o(p)|),

where o~ is the oracle with every normal moved uniformly within that bound
(a separate Philox stream per draw; several draws, because near V = 0 a few
paths dominate the change and one draw can miss them).  Where delta is small against the 1e-4
bound (delta <= BOUND / 3), the estimate is well-conditioned at FP32
precision and an FP32 path is held to both bounds: within 3 standard errors
and within 1e-4 * max(1, |oracle|).  Where it is not, perturbations of the
size an FP32 path makes already move the FP64 result by a third of the
bound or more, so no FP32 path can be held to it: the estimate is
ill-conditioned.  This happens for the pathwise Vega and Theta (the v0- and
T-tangents pass through 1 / sqrt(V)) when paths come close to V = 0 with
many steps, and in extreme cases for the price itself.  The tests then
record that evidence; a finite GPU value is held to max(3 SE, 3 delta) when
delta <= 1e-3 and to nothing numeric beyond that.
"""
import numpy as np

import oracle

BOUND = 1e-4
WELL = BOUND / 3.0        # delta at most a third of the bound: both bounds apply
MODERATE = 1e-3           # up to here a finite GPU value is held to max(3 SE, 3 delta)
DRAWS = 4
FP32_NORMAL_ABS, FP32_NORMAL_REL = 1e-7, 1.5e-6


def f32(x: float) -> float:
    return float(np.float32(x))


def rounded_params(params: dict) -> dict:
    return {k: f32(v) for k, v in params.items()}


def rounded_contract(c):
    payoff, K, T, put, M = c
    return (payoff, f32(K), f32(T), put, M)


def oracle_with_sensitivity(params: dict, contracts, n_paths, n_steps, seed, trunc=0, scheme=0):
    """Oracle estimates and SEs (C, 6) on exact inputs, and delta (C, 6): the
    relative change of those estimates with FP32-rounded inputs and normals
    perturbed within the FP32 normal-error bound (largest of DRAWS draws)."""
    cs = [oracle.Contract(*c) for c in contracts]
    cs32 = [oracle.Contract(*rounded_contract(c)) for c in contracts]
    P, P32 = oracle.Params(**params), oracle.Params(**rounded_params(params))
    om, ose = oracle.mc_price_greeks(P, cs, n_paths, n_steps, seed, trunc, scheme=scheme)
    delta = np.zeros_like(om)
    for draw in range(1, DRAWS + 1):
        o32, _ = oracle.mc_price_greeks_perturbed(P32, cs32, n_paths, n_steps, seed, FP32_NORMAL_ABS,
                                                  FP32_NORMAL_REL, draw, trunc, scheme)
        with np.errstate(invalid="ignore"):
            d = np.abs(om - o32) / np.maximum(1.0, np.abs(om))
        d[~np.isfinite(d)] = np.inf
        delta = np.maximum(delta, d)
    return om, ose, delta


def check_fp32_estimates(gm, om, ose, delta, label=""):
    """Both bounds (3 SE and 1e-4 * max(1, |oracle|)) where delta <= WELL;
    max(3 SE, 3 delta * max(1, |oracle|)) for finite GPU values where
    WELL < delta <= MODERATE; no numeric bound beyond.  Returns the mask of
    ill-conditioned cells (delta > WELL)."""
    gm, om, ose, delta = (np.asarray(a, float) for a in (gm, om, ose, delta))
    scale = np.maximum(1.0, np.abs(om))
    d = np.abs(gm - om)
    ill = delta > WELL
    well = ~ill
    assert np.isfinite(gm[well]).all(), (label, "non-finite GPU value on a well-conditioned cell")
    assert (d[well] <= 3.0 * ose[well] + 1e-12 * scale[well]).all(), \
        (label, np.max(d[well] / np.maximum(ose[well], 1e-300)))
    assert (d[well] <= BOUND * scale[well]).all(), (label, np.max(d[well] / scale[well]))
    mod = ill & (delta <= MODERATE) & np.isfinite(gm)
    assert (d[mod] <= np.maximum(3.0 * ose[mod], 3.0 * delta[mod] * scale[mod])).all(), \
        (label, "moderately ill-conditioned cell beyond max(3 SE, 3 delta)", d[mod], ose[mod], delta[mod])
    return ill


# ---------------------------------------------------------------------------
# Per path
# ---------------------------------------------------------------------------
FP64_NORMAL_REL = 1e-15   # FP64 Box-Muller: a few ulp of CUDA's log / sincospi against the C library's


def paths_with_sensitivity(params: dict, contracts, Za, Zb, trunc=0, scheme=0, prec="fp32",
                           eps_abs=None, eps_rel=None, seed=0, draws=DRAWS):
    """Oracle records (n, 15) and estimators (n, C, 6) of paths from given
    normals (n, N), and the largest absolute change of each over `draws` runs
    with every normal moved uniformly within eps_abs + eps_rel * R (default:
    the FP32 or FP64 Box-Muller bound) and, for FP32, the inputs rounded to
    FP32."""
    cs = [oracle.Contract(*c) for c in contracts]
    rec, est = oracle.paths_from_normals(oracle.Params(**params), cs, Za, Zb, trunc, scheme)
    if prec == "fp32":
        P = oracle.Params(**rounded_params(params))
        cs_p = [oracle.Contract(*rounded_contract(c)) for c in contracts]
        ea, er = FP32_NORMAL_ABS, FP32_NORMAL_REL
    else:
        P, cs_p = oracle.Params(**params), cs
        ea, er = 0.0, FP64_NORMAL_REL
    ea = ea if eps_abs is None else eps_abs
    er = er if eps_rel is None else eps_rel
    bound = ea + er * np.hypot(Za, Zb)
    g = np.random.default_rng(seed ^ 0x5EED)
    drec = np.zeros_like(rec)
    dest = np.zeros_like(est)
    for _ in range(draws):
        r, e = oracle.paths_from_normals(P, cs_p, Za + bound * g.uniform(-1, 1, Za.shape),
                                         Zb + bound * g.uniform(-1, 1, Zb.shape), trunc, scheme)
        with np.errstate(invalid="ignore"):
            drec = np.fmax(drec, np.abs(r - rec))
            dest = np.fmax(dest, np.abs(e - est))
    return rec, est, drec, dest


def oracle_paths_with_sensitivity(params: dict, contracts, paths, n_steps, seed, trunc=0, scheme=0,
                                  prec="fp32", draws=DRAWS):
    """paths_with_sensitivity on the paths' own Philox normals: the change
    measures how much rounding of the size the GPU path makes can move each
    per-path quantity; the tangents, which pass through 1 / sqrt(V), move
    most on paths that come near V = 0."""
    paths = np.asarray(paths, dtype=np.uint64)
    Za = np.empty((len(paths), n_steps))
    Zb = np.empty_like(Za)
    for i, q in enumerate(paths):
        Za[i], Zb[i] = oracle.path_normals(seed, int(q), n_steps)
    return paths_with_sensitivity(params, contracts, Za, Zb, trunc, scheme, prec, seed=seed, draws=draws)


# Randomised-QMC normals in FP32: the Brownian bridge forms each W by
# interpolation from two stored values and each step normal as W_{k+1} - W_k,
# so the rounding of a step normal scales with the size of the path's W
# (|W| ~ sqrt(N) in step units), not with the normal's own size.  A time-ordered
# FP32 bridge stays within 3 * 2^-24 * max_k |W_k| per step normal on the
# Sobol points (tested against an emulation on the CPU); the bound below takes
# 4, plus the Box-Muller-sized terms for the inverse normal of each node.
QMC_BRIDGE_ABS = 4.0 * 2.0 ** -24


def qmc_normal_bound(Za, Zb):
    """Per-path absolute bound (n, 1) on the FP32 error of bridge step normals."""
    Wmax = np.maximum(np.abs(np.cumsum(Za, axis=1)).max(axis=1), np.abs(np.cumsum(Zb, axis=1)).max(axis=1))
    return (QMC_BRIDGE_ABS * Wmax + FP32_NORMAL_ABS)[:, None]


def qmc_paths_with_sensitivity(params: dict, contracts, Za, Zb, trunc=0, seed=0, draws=DRAWS):
    """paths_with_sensitivity on QMC bridge normals, with the bridge's FP32
    error bound (qmc_normal_bound) in place of the Box-Muller one."""
    return paths_with_sensitivity(params, contracts, Za, Zb, trunc, 0, "fp32",
                                  qmc_normal_bound(Za, Zb), FP32_NORMAL_REL, seed, draws)


def path_scales(rec_o, est_o, params, contracts, n_steps):
    """The scale each per-path quantity is compared relative to: X (= ln S_T/S0)
    max(1, |X|); V max(|V|, theta, v0); dV/dT also at least max(theta, v0) / T
    (the variance's own scale per unit time: its error comes from V's); the
    discounted payoff max(K, A) (A = S_T or the Asian average); every other
    record field and estimator max(|x|, the median |x| of that quantity over
    the sample) -- the tangents start at zero and change sign, so a purely
    relative bound has no meaning where they cross it."""
    sc = np.maximum(np.abs(rec_o[:, :14]), np.median(np.abs(rec_o[:, :14]), axis=0))
    sc[:, 0] = np.maximum(1.0, np.abs(rec_o[:, 0]))
    vs = max(params["theta"], params["v0"])
    sc[:, 1] = np.maximum(np.abs(rec_o[:, 1]), vs)
    sc[:, 5] = np.maximum(sc[:, 5], vs / contracts[0][2])
    # estimators: the median over the paths where the estimator is not zero (an
    # out-of-the-money path contributes an exact zero, not a typical size)
    a = np.abs(est_o)
    nz = np.where(a > 0, a, np.nan)
    with np.errstate(all="ignore"):
        med = np.nan_to_num(np.nanmedian(nz, axis=0), nan=0.0)
    esc = np.maximum(a, med)
    for ci, c in enumerate(contracts):
        A = params["S0"] * np.exp(rec_o[:, 0]) if c[0] == 0 else rec_o[:, 6] / (c[4] or n_steps)
        esc[:, ci, 0] = np.maximum(esc[:, ci, 0], np.maximum(A, c[1]))
    return sc, esc


def check_paths(rec_g, est_g, rec_o, est_o, drec, dest, params, contracts, n_steps, ok, rel, label=""):
    """|gpu - oracle| <= rel * scale + 4 * change, on every record field and
    estimator of the paths in `ok` (rel: one number, or a pair of arrays per
    record field (14) and per estimator (6); see path_scales and
    oracle_paths_with_sensitivity).  The factor 4 allows for the GPU's normal
    errors being deterministic functions of the angle and radius (the
    special-function approximations), not the uniform draws of the probe.
    Returns the number of (path, quantity) pairs that needed the change
    term, i.e. were beyond rel * scale."""
    sc, esc = path_scales(rec_o, est_o, params, contracts, n_steps)
    rel_r, rel_e = rel if isinstance(rel, tuple) else (rel, rel)   # per record field / estimator
    d = np.abs(rec_g[:, :14] - rec_o[:, :14])
    de = np.abs(est_g - est_o)
    lim = rel_r * sc + 4.0 * drec[:, :14]
    elim = rel_e * esc + 4.0 * dest
    bad = (d > lim)[ok]
    ebad = (de > elim)[ok]
    assert not bad.any(), (label, "record", np.argwhere(bad)[:5], (d / lim)[ok].max(axis=0))
    assert not ebad.any(), (label, "estimators", np.argwhere(ebad)[:5], (de / elim)[ok].max(axis=0))
    return int((d > rel_r * sc)[ok].sum() + (de > rel_e * esc)[ok].sum())


def oracle_gradients_with_sensitivity(params: dict, contract, paths, n_steps, seed, draws=DRAWS):
    """Per-path (payoff, 7 derivatives) of the oracle's forward-mode gradient
    on the paths' own normals (n, 8), and their largest absolute change over
    `draws` runs with FP32-rounded inputs and normals moved within the FP32
    normal-error bound."""
    paths = np.asarray(paths, dtype=np.uint64)
    Za = np.empty((len(paths), n_steps))
    Zb = np.empty_like(Za)
    for i, q in enumerate(paths):
        Za[i], Zb[i] = oracle.path_normals(seed, int(q), n_steps)
    g = oracle.gradients_from_normals(oracle.Params(**params), oracle.Contract(*contract), Za, Zb)
    P = oracle.Params(**rounded_params(params))
    c32 = oracle.Contract(*rounded_contract(contract))
    bound = FP32_NORMAL_ABS + FP32_NORMAL_REL * np.hypot(Za, Zb)
    rng = np.random.default_rng(seed ^ 0x6AD)
    dg = np.zeros_like(g)
    for _ in range(draws):
        h = oracle.gradients_from_normals(P, c32, Za + bound * rng.uniform(-1, 1, Za.shape),
                                          Zb + bound * rng.uniform(-1, 1, Zb.shape))
        dg = np.fmax(dg, np.abs(h - g))
    return g, dg
