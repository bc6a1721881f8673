"""GPU path vs the FP64 CPU oracle, through the C ABI, on identical normals.

Tolerances:
  * random-number contract: Philox words bit-exact; FP64 normals within
    1e-14; FP32 normals within 1e-7 + 1.5e-6 R (R = sqrt(Za^2 + Zb^2)): the
    documented bounds of sqrt.approx (2^-22 relative), lg2.approx (2^-22
    absolute, used only where R >= 0.46, giving |dR| <= 3.6e-7) or the
    near-1 polynomial (8.4e-9 relative), and sin/cos.approx (2^-20.9 absolute on
    [-pi, pi]) give about 9e-7 R + 3.6e-7 at the switch.
  * per path, FP64 path: every record field and estimator within 1e-12 of
    its scale (tests/conditioning.py path_scales: max(1, |X|) for ln S_T/S0,
    max(|V|, theta, v0) for V, max(K, A) for the payoff, max(|x|, the
    sample's median |x|) for tangents, sums and the other estimators) plus
    four times the oracle's own change when its normals move by a few ulp.
  * per path, FP32 path (the packed two-path kernel): every record field
    (X_N, V_N, the v0- and T-tangents, Asian sums, Gamma weights G and Q)
    and all six per-path estimators within 1e-5 of the same scales plus four
    times the oracle's own change under FP32-rounded inputs and normals
    moved within the FP32 normal-error bound (that term matters only for
    tangents of paths near V = 0); paths whose truncation branch or payoff
    indicator can flip between FP32 and FP64 (min |V_k| or |A - K| within
    the FP32 error band) are counted, not compared, and must stay below
    1e-3 of the sample.
  * estimates: FP64 within 1e-11 relative; FP32 within 3 standard errors
    and within 1e-4 * max(1, |oracle|), on cells that are well-conditioned
    at FP32 precision (all of them for these parameter sets).
"""
import math

import numpy as np
import pytest

import oracle
from conditioning import (check_fp32_estimates, check_paths, oracle_paths_with_sensitivity,
                          oracle_with_sensitivity)
from exact_rounding import round_exact
from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BASE = wl.BASE_PARAMS
PAPER = wl.PAPER_PARAMS


@pytest.fixture(scope="module")
def nv(cuda_lib):
    from paper_2309_10477_gb300 import native
    return native


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    return torch


def _gp(nv, d):
    return nv.make_params(**d)


def _gc(nv, cs):
    return [nv.make_contract(*c) for c in cs]


def _oc(cs):
    return [oracle.Contract(c[0], c[1], c[2], c[3], c[4]) for c in cs]


def _prec(nv, name):
    return nv.HESTON_FP32 if name == "fp32" else nv.HESTON_FP64


# ---------------------------------------------------------------------------
# Random-number contract
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [42, 0, 2**64 - 1, 0x9E3779B97F4A7C15])
def test_rng_contract(nv, seed):
    rng = np.random.default_rng(1)
    paths = np.concatenate([[0, 1, 63, 64, 2**32 - 1, 2**32, 2**40 + 7],
                            rng.integers(0, 2**34, 2000)]).astype(np.uint64)
    steps = np.concatenate([[0, 1, 2, 3, 251, 252, 99999],
                            rng.integers(0, 600, 2000)]).astype(np.uint32)
    w64, n64 = nv.heston_rng_debug(seed, paths, steps, nv.HESTON_FP64)
    _, n32 = nv.heston_rng_debug(seed, paths, steps, nv.HESTON_FP32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(len(paths)):
        p, s = int(paths[i]), int(steps[i])
        assert oracle.philox4x32_10([s // 2, p & 0xFFFFFFFF, p >> 32, 0], key) == list(w64[i])
        za, zb = oracle.path_normals(seed, p, s + 1)
        ref = np.array([za[s], zb[s]])
        assert np.abs(n64[i] - ref).max() < 1e-14
        # FP32: |dZ| <= R (rel. error of sqrt and log + abs. error of sin/cos + angle rounding)
        R = math.hypot(*ref)
        assert (np.abs(n32[i] - ref) <= 1e-7 + 1.5e-6 * R).all(), (p, s, n32[i], ref)


def test_fp64_box_muller_functions_against_cuda(nv):
    """The FP64 Box-Muller's table-driven logarithm and sine/cosine (Tang's
    method: a table entry and a short polynomial) against CUDA's log and
    sincospi over every 24-bit input: ln u1 within 3 ulp of CUDA's (each is
    within about 1.5 ulp of the exact value), sin and cos of 2 pi u2 within
    3e-16 absolute everywhere and 4 ulp where |x| > 1e-3 (the table form is
    within 2.3 ulp there, CUDA's within about 1)."""
    chunk = 1 << 22
    for first in range(0, 1 << 24, chunk):
        o = nv.heston_bm64_debug(first, chunk)
        ln_t, ln_c, s_t, c_t, s_c, c_c = o.T
        assert np.isfinite(o).all()
        d = np.abs(ln_t - ln_c)
        assert (d <= 3 * np.spacing(np.abs(ln_c))).all(), (first, np.argmax(d / np.spacing(np.abs(ln_c))))
        for t, c in ((s_t, s_c), (c_t, c_c)):
            e = np.abs(t - c)
            assert e.max() <= 3e-16, (first, e.max())
            big = np.abs(c) > 1e-3
            assert (e[big] <= 4 * np.spacing(np.abs(c[big]))).all(), first
    # the ends of the range: u1 = 2^-24 and 1, angle 0
    o = nv.heston_bm64_debug(0, 1)[0]
    assert o[0] == o[1] and o[2] == 0.0 and o[3] == 1.0
    o = nv.heston_bm64_debug((1 << 24) - 1, 1)[0]
    assert o[0] == 0.0 and o[1] == 0.0


# ---------------------------------------------------------------------------
# Per-path parity
# ---------------------------------------------------------------------------

CASES = [
    ("base", BASE, 1), ("base", BASE, 2), ("base", BASE, 7), ("base", BASE, 64),
    ("paper", PAPER, 3), ("paper", PAPER, 64), ("paper", PAPER, 128),
]


def _contracts_for(N):
    return [(0, 100.0, 1.0, 0, 0), (1, 95.0, 1.0, 0, 0), (0, 105.0, 1.0, 1, 0),
            (1, 100.0, 1.0, 1, 0)]


def _paths():
    return np.concatenate([np.arange(0, 700), 2**32 - 3 + np.arange(6),
                           2**36 + 11 * np.arange(50)]).astype(np.uint64)


@pytest.mark.parametrize("trunc", [0, 1])
@pytest.mark.parametrize("name,params,N", CASES)
def test_per_path_fp64(nv, name, params, N, trunc):
    """FP64 path: every record field and estimator within 1e-12 of the
    oracle's (relative to the scales of conditioning.path_scales), plus four
    times the oracle's own change when its normals move by a few ulp (the
    difference of CUDA's and the C library's log / sincospi): that term
    matters only for the tangents of paths that pass near V = 0."""
    cs = _contracts_for(N)
    paths = _paths()
    rec_g, est_g = nv.heston_mc_debug_paths(_gp(nv, params), _gc(nv, cs), N, 42,
                                            nv.make_options(trunc=trunc, prec=nv.HESTON_FP64), paths)
    rec_o, est_o, drec, dest = oracle_paths_with_sensitivity(params, cs, paths, N, 42, trunc,
                                                             prec="fp64")
    rec_d, _ = oracle.debug_paths(oracle.Params(**params), _oc(cs), paths, N, 42, trunc)
    assert np.array_equal(rec_d, rec_o)               # the same oracle path either way
    flips = rec_o[:, 14] < 1e-12                      # a truncation branch at |V| ~ 1e-16 may differ
    assert flips.sum() <= max(1, len(paths) // 1000)
    check_paths(rec_g, est_g, rec_o, est_o, drec, dest, params, cs, N, ~flips, 1e-12, name)


def _fp32_flip_mask(rec_o, est_o, cs, params, N, T=1.0):
    """Paths whose FP32 run can take another branch than the FP64 oracle."""
    near_zero = rec_o[:, 14] < 1e-5 * max(params["theta"], params["v0"])
    S0 = params["S0"]
    A_euro = S0 * np.exp(rec_o[:, 0])
    near_k = np.zeros(len(rec_o), bool)
    for c in cs:
        M = c[4] or N
        A = A_euro if c[0] == 0 else rec_o[:, 6] / M
        near_k |= np.abs(A - c[1]) < 2e-5 * max(c[1], 1.0)
    return near_zero | near_k


@pytest.mark.parametrize("trunc", [0, 1])
@pytest.mark.parametrize("name,params,N", CASES + [("base", BASE, 252)])
def test_per_path_fp32(nv, name, params, N, trunc):
    """The shipped packed FP32 path, per path: all 14 record fields (X_N, V_N,
    the v0- and T-tangents, the Asian sums, the Gamma weights G and Q) and
    all six per-path estimators of every contract within 1e-5 of the
    oracle's (relative to the scales of conditioning.path_scales), plus four
    times the oracle's own change under FP32-rounded inputs and normals moved
    within the FP32 normal-error bound.  Paths whose truncation branch or
    payoff indicator can flip are counted, not compared; the change term is
    needed on at most 5 % of the compared quantities."""
    cs = _contracts_for(N)
    paths = _paths()
    rec_g, est_g = nv.heston_mc_debug_paths(_gp(nv, params), _gc(nv, cs), N, 42,
                                            nv.make_options(trunc=trunc, prec=nv.HESTON_FP32), paths)
    rec_o, est_o, drec, dest = oracle_paths_with_sensitivity(params, cs, paths, N, 42, trunc)
    flips = _fp32_flip_mask(rec_o, est_o, cs, params, N)
    assert flips.sum() <= max(2, len(paths) // 1000)
    n_wide = check_paths(rec_g, est_g, rec_o, est_o, drec, dest, params, cs, N, ~flips, 1e-5, name)
    n_cmp = (~flips).sum() * (14 + 6 * len(cs))
    assert n_wide <= 0.05 * n_cmp, (n_wide, n_cmp)


# ---------------------------------------------------------------------------
# Estimates
# ---------------------------------------------------------------------------

def _gpu_estimates(nv, params, cs, n, N, seed, prec, trunc=0, **opt):
    res = nv.heston_mc_price_greeks_ex(_gp(nv, params), _gc(nv, cs), n, N, seed,
                                       nv.make_options(trunc=trunc, prec=prec, **opt))
    return nv.results_to_arrays(res)


@pytest.mark.parametrize("n", [2, 31, 33, 64, 65, 2381, (1 << 16) + 5])
@pytest.mark.parametrize("N", [1, 3, 50])
def test_estimates_fp64_match_oracle(nv, n, N):
    cs = _contracts_for(N)
    gm, gse = _gpu_estimates(nv, BASE, cs, n, N, 7, nv.HESTON_FP64)
    om, ose = oracle.mc_price_greeks(oracle.Params(**BASE), _oc(cs), n, N, 7)
    np.testing.assert_allclose(gm, om, rtol=1e-11, atol=1e-13)
    # SE from (sum_x, sum_x^2) carries a rounding floor of about |mean| sqrt(eps / (n-1))
    # (a constant estimator such as the European Rho with every path in the money)
    floor = 1e-7 * np.maximum(1.0, np.abs(om))
    assert (np.abs(gse - ose) <= 1e-6 * ose + floor).all()


@pytest.mark.parametrize("trunc", [0, 1])
@pytest.mark.parametrize("params", [BASE, PAPER], ids=["base", "paper"])
def test_estimates_fp32_match_oracle(nv, params, trunc):
    """Every estimate (Vega and Theta on the Feller-violating paper set
    included) within 3 SE and 1e-4 of the FP64 oracle: all 36 cells are
    well-conditioned at FP32 precision here (tests/conditioning.py)."""
    w = wl.multi_strike_fp32(1 << 16)
    gm, gse = _gpu_estimates(nv, params, w.contracts, w.n_paths, w.n_steps, 3, nv.HESTON_FP32, trunc)
    om, ose, delta = oracle_with_sensitivity(params, w.contracts, w.n_paths, w.n_steps, 3, trunc)
    ill = check_fp32_estimates(gm, om, ose, delta)
    assert not ill.any(), delta
    d = np.abs(gm - om)
    assert (d <= 3 * ose).all(), np.max(d / ose)
    assert (d <= 1e-4 * np.maximum(1.0, np.abs(om))).all(), np.max(d / np.maximum(1, np.abs(om)))


def test_single_european_fp64_full_size(nv):
    """2^16 paths x 100 steps, FP64, one European call: the whole estimate."""
    w = wl.single_european_fp64()
    res = nv.heston_mc_price_greeks(_gp(nv, w.params), _gc(nv, w.contracts)[0], w.n_paths,
                                    w.n_steps, w.seed)
    gm, gse = nv.results_to_arrays([res])
    om, ose = oracle.mc_price_greeks(oracle.Params(**w.params), _oc(w.contracts), w.n_paths,
                                     w.n_steps, w.seed)
    np.testing.assert_allclose(gm, om, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gse, ose, rtol=1e-6)
    assert res.status == 0 and res.n_paths == w.n_paths


def test_multi_strike_full_size_in_bench_launch(nv, torch_cuda):
    """2^22 paths x 252 steps, 6 contracts, FP32: the launch bench.py times.
    Sampled 64-path tile rows are checked against the oracle tile by tile,
    and the full estimates against the oracle's full run."""
    torch = torch_cuda
    w = wl.multi_strike_fp32()
    nc = len(w.contracts)
    ws_bytes = nv.heston_mc_workspace_bytes(nc, w.n_paths)
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device="cuda")
    off = (-ws.data_ptr()) % 256
    base = ws.data_ptr() + off
    out = torch.empty(nc * 12, dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
    nv.heston_mc_launch(_gp(nv, w.params), _gc(nv, w.contracts), w.n_paths, w.n_steps, w.seed,
                        opts, base, ws_bytes - 0, out)
    torch.cuda.synchronize()
    n_tiles = w.n_paths // 64
    rows = ws.view(torch.uint8)[off:off + n_tiles * 12 * nc * 8].view(torch.float64)
    rows = rows.view(n_tiles, 12 * nc).cpu().numpy()
    gout = out.cpu().numpy().reshape(nc, 12)

    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([[0, 1, n_tiles - 1], rng.integers(0, n_tiles, 150)]))
    P = oracle.Params(**w.params)
    oc = _oc(w.contracts)
    n_flip = 0
    for t in sample:
        idx = np.arange(t * 64, t * 64 + 64)
        rec, est = oracle.debug_paths(P, oc, idx, w.n_steps, w.seed)      # (64, C, 6)
        s, s2 = est.sum(axis=0), (est * est).sum(axis=0)
        g, g2 = rows[t, :6 * nc].reshape(nc, 6), rows[t, 6 * nc:].reshape(nc, 6)
        # per-path FP32 error <= ~1e-5 |x| bounds the tile sum error by 1e-5 sum |x|
        tol = 2e-5 * np.abs(est).sum(axis=0) + 1e-9
        tol2 = 4e-5 * s2 + 1e-9
        bad = (np.abs(g - s) > tol) | (np.abs(g2 - s2) > tol2)
        if bad.any():
            flip = _fp32_flip_mask(rec, est, w.contracts, w.params, w.n_steps)
            if not flip.any():
                rg, eg = nv.heston_mc_debug_paths(_gp(nv, w.params), _gc(nv, w.contracts),
                                                  w.n_steps, w.seed,
                                                  nv.make_options(prec=nv.HESTON_FP32), idx)
                c, j = np.argwhere(bad)[0]
                worst = np.argmax(np.abs(eg[:, c, j] - est[:, c, j]))
                pytest.fail(f"tile {t} contract {c} estimator {j}: gpu {g[c, j]!r} oracle "
                            f"{s[c, j]!r} tol {tol[c, j]!r}; worst path {idx[worst]}: gpu "
                            f"{eg[worst, c, j]!r} oracle {est[worst, c, j]!r}; record gpu "
                            f"{rg[worst].tolist()} oracle {rec[worst].tolist()}")
            n_flip += 1
    assert n_flip <= 2

    om, ose = oracle.mc_price_greeks(P, _oc(w.contracts), w.n_paths, w.n_steps, w.seed)
    gm, gse = gout[:, :6], gout[:, 6:]
    d = np.abs(gm - om)
    assert (d <= 3 * ose).all()
    assert (d <= 1e-4 * np.maximum(1.0, np.abs(om))).all()
    np.testing.assert_allclose(gse, ose, rtol=1e-3)


# ---------------------------------------------------------------------------
# Determinism, sharding, launch shape, streams
# ---------------------------------------------------------------------------

def _launch(nv, torch, params, cs, n, N, seed, prec, **opt):
    nc = len(cs)
    ws_bytes = nv.heston_mc_workspace_bytes(nc, n)
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda")
    out = torch.empty(nc * 12, dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=prec, stream=torch.cuda.current_stream(), **opt)
    nv.heston_mc_launch(_gp(nv, params), _gc(nv, cs), n, N, seed, opts, ws, ws_bytes, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_launch_shape_and_repeat_do_not_change_bits(nv, torch_cuda, prec):
    torch = torch_cuda
    cs = _contracts_for(40)
    n, N = 64 * 500 + 19, 40
    p = _prec(nv, prec)
    ref = _launch(nv, torch, BASE, cs, n, N, 9, p)
    assert np.array_equal(ref, _launch(nv, torch, BASE, cs, n, N, 9, p))
    for grid, block in ((1, 32), (7, 64), (300, 128), (0, 96)):
        got = _launch(nv, torch, BASE, cs, n, N, 9, p, grid_ctas=grid, block_threads=block)
        assert np.array_equal(ref, got), (grid, block)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_path_range_shards_reduce_to_identical_bits(nv, torch_cuda, prec):
    torch = torch_cuda
    cs = _contracts_for(30)
    n, N, seed = 64 * 1000 + 17, 30, 11
    p = _prec(nv, prec)
    ref = _launch(nv, torch, BASE, cs, n, N, seed, p)
    nc = len(cs)
    n_tiles = -(-n // 64)
    rows = torch.zeros(n_tiles * 12 * nc, dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=p, stream=torch.cuda.current_stream())
    bounds = [0, 64 * 300, 64 * 301, 64 * 700, n]
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        view = rows[(lo // 64) * 12 * nc:]
        nv.heston_mc_launch_tiles(_gp(nv, BASE), _gc(nv, cs), lo, hi - lo, N, seed, opts, view)
    ws_bytes = nv.heston_mc_workspace_bytes(nc, n)
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda")
    out = torch.empty(nc * 12, dtype=torch.float64, device="cuda")
    nv.heston_mc_reduce_tiles(rows, n_tiles, nc, n, ws, ws_bytes, out,
                              torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(ref, out.cpu().numpy())


def test_side_stream(nv, torch_cuda):
    torch = torch_cuda
    s = torch.cuda.Stream()
    cs = _contracts_for(20)
    with torch.cuda.stream(s):
        got = _launch(nv, torch, BASE, cs, 5000, 20, 4, nv.HESTON_FP64)
    om, ose = oracle.mc_price_greeks(oracle.Params(**BASE), _oc(cs), 5000, 20, 4)
    np.testing.assert_allclose(got.reshape(len(cs), 12)[:, :6], om, rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------------------
# Degenerate cases
# ---------------------------------------------------------------------------

def test_gamma_undefined_when_rho_is_one(nv):
    p = dict(BASE, rho=-1.0)
    cs = [(0, 100.0, 1.0, 0, 0)]
    res = nv.heston_mc_price_greeks_ex(_gp(nv, p), _gc(nv, cs), 4096, 16, 1,
                                       nv.make_options(prec=nv.HESTON_FP64))
    assert res[0].status == nv.HESTON_WARN_GAMMA_UNDEFINED
    gm, _ = nv.results_to_arrays(res)
    om, _ = oracle.mc_price_greeks(oracle.Params(**p), _oc(cs), 4096, 16, 1)
    assert math.isnan(gm[0, 2])
    keep = [0, 1, 3, 4, 5]
    np.testing.assert_allclose(gm[0, keep], om[0, keep], rtol=1e-9)


@pytest.mark.parametrize("change", [dict(xi=0.0), dict(rho=0.0), dict(kappa=0.0),
                                    dict(theta=0.0), dict(r=-0.01)])
def test_degenerate_parameters(nv, change):
    p = dict(BASE, **change)
    cs = [(0, 100.0, 1.0, 0, 0), (1, 0.0, 1.0, 0, 5), (0, 0.0, 1.0, 1, 0)]
    gm, _ = _gpu_estimates(nv, p, cs, 3000, 20, 5, nv.HESTON_FP64)
    om, _ = oracle.mc_price_greeks(oracle.Params(**p), _oc(cs), 3000, 20, 5)
    np.testing.assert_allclose(gm, om, rtol=1e-9, atol=1e-11)
    # K = 0 put is worthless
    assert (gm[2] == 0).all()


def test_asian_with_sparse_dates_and_odd_steps(nv):
    for N, M in ((9, 3), (128, 4), (7, 1), (7, 7)):
        cs = [(1, 100.0, 1.0, 0, M), (1, 90.0, 1.0, 1, M), (0, 100.0, 1.0, 0, 0)]
        gm, _ = _gpu_estimates(nv, PAPER, cs, 2000, N, 2, nv.HESTON_FP64)
        om, _ = oracle.mc_price_greeks(oracle.Params(**PAPER), _oc(cs), 2000, N, 2)
        np.testing.assert_allclose(gm, om, rtol=1e-9, atol=1e-11)


def test_cached_scratch_reuse_and_release(nv):
    """Repeated synchronous calls reuse the cached scratch and give the same
    bits; releasing it between calls changes nothing."""
    cs = _contracts_for(16)
    args = (_gp(nv, BASE), _gc(nv, cs), 64 * 40 + 3, 16, 5, nv.make_options(prec=nv.HESTON_FP32))
    ref = nv.results_to_arrays(nv.heston_mc_price_greeks_ex(*args))
    for release in (False, True, False):
        if release:
            nv.heston_release_cached_memory(-1)
            nv.heston_release_cached_memory(0)
        got = nv.results_to_arrays(nv.heston_mc_price_greeks_ex(*args))
        assert all(np.array_equal(a, b) for a, b in zip(ref, got))
    with pytest.raises(nv.HestonError):
        nv.heston_release_cached_memory(64)


@pytest.mark.parametrize("prec,path_begin,n,N,block,scheme", [("fp32", 0, 64 * 3 + 19, 30, 0, 0),
                                                               ("fp64", 0, 64 * 3 + 19, 30, 0, 0),
                                                               ("fp32", (1 << 32) - 128, 256 - 5, 30, 0, 0),
                                                               ("fp32", (1 << 32) - 128, 256 - 5, 67, 128, 0),
                                                               ("fp32", 64 * 7, 64 * 5 + 3, 130, 128, 0),
                                                               ("fp32", (1 << 32) - 128, 256 - 5, 67, 128, 2),
                                                               ("fp32", 0, 64 * 2 + 5, 1, 128, 0),
                                                               ("fp32", 0, 64 * 2 + 5, 2, 128, 0)])
def test_tile_rows_are_the_sums_of_the_per_path_records(nv, torch_cuda, prec, path_begin, n, N, block,
                                                        scheme):
    """The production path kernel and the per-path record kernel (the one the
    per-path parity tests check against the oracle) compute the same paths:
    each tile row equals, bit for bit, the warp's sums of the per-path
    estimators -- lane l adds paths l and l + 32 of the tile (x0 + x1 and
    fma(x0, x0, x1 * x1), zero past the last path), then a xor butterfly over
    offsets 16, 8, 4, 2, 1 -- rounded in the path precision.  The third case
    runs a path range across index 2^32, where the Philox counter's high
    word (taken per tile in the path kernel) changes.  These small launches
    take the split kernel (one path per lane); block = 128 selects the packed
    kernel, whose Philox words come from the per-warp table of 32 step pairs:
    across 2^32 (one CTA whose warps have different high words) with 33
    step pairs and an odd last step, and over 65 step pairs (three fills of
    the table); QE (scheme 2) the same way; and one step (no step pair: the
    odd step alone) and two (one step pair)."""
    from fractions import Fraction
    torch = torch_cuda
    bits = 24 if prec == "fp32" else 53
    cs = _contracts_for(N)
    nc = len(cs)
    seed = 5
    opts = nv.make_options(prec=_prec(nv, prec), stream=torch.cuda.current_stream(), block_threads=block,
                           scheme=scheme)
    n_tiles = -(-n // 64)
    rows = torch.zeros(n_tiles * 12 * nc, dtype=torch.float64, device="cuda")
    nv.heston_mc_launch_tiles(_gp(nv, BASE), _gc(nv, cs), path_begin, n, N, seed, opts, rows)
    torch.cuda.synchronize()
    rows = rows.cpu().numpy().reshape(n_tiles, 12 * nc)
    _, est = nv.heston_mc_debug_paths(_gp(nv, BASE), _gc(nv, cs), N, seed,
                                      nv.make_options(prec=_prec(nv, prec), scheme=scheme),
                                      path_begin + np.arange(n, dtype=np.uint64))
    rnd = lambda q: round_exact(q, bits)
    for t in range(n_tiles):
        for c in range(nc):
            for j in range(6):
                x = [est[t * 64 + i, c, j] if t * 64 + i < n else 0.0 for i in range(64)]
                sx = [rnd(Fraction(x[l]) + Fraction(x[l + 32])) for l in range(32)]
                sxx = [rnd(Fraction(x[l]) ** 2 + Fraction(rnd(Fraction(x[l + 32]) ** 2)))
                       for l in range(32)]
                for o in (16, 8, 4, 2, 1):
                    sx = [rnd(Fraction(sx[l]) + Fraction(sx[l ^ o])) for l in range(32)]
                    sxx = [rnd(Fraction(sxx[l]) + Fraction(sxx[l ^ o])) for l in range(32)]
                assert rows[t, c * 6 + j] == sx[0], (t, c, j)
                assert rows[t, 6 * nc + c * 6 + j] == sxx[0], (t, c, j)


def test_eight_contracts_the_widest_tile_row(nv):
    """HESTON_MAX_CONTRACTS = 8 on one set of paths: tile rows of 96 columns,
    the widest the epilogue and the fixed-order reductions handle; FP64 to
    1e-9 of the oracle (contracts on one set of paths share T and the Asian
    dates).  Nine contracts are rejected."""
    cs = [(0, 90.0, 1.0, 0, 0), (0, 100.0, 1.0, 1, 0), (1, 95.0, 1.0, 0, 0), (1, 105.0, 1.0, 1, 0),
          (0, 110.0, 1.0, 0, 0), (1, 100.0, 1.0, 0, 0), (0, 80.0, 1.0, 1, 0), (1, 120.0, 1.0, 0, 0)]
    assert len(cs) == nv.HESTON_MAX_CONTRACTS
    n, N = 64 * 40 + 3, 24
    gm, gse = _gpu_estimates(nv, BASE, cs, n, N, 77, nv.HESTON_FP64)
    om, ose = oracle.mc_price_greeks(oracle.Params(**BASE), _oc(cs), n, N, 77)
    np.testing.assert_allclose(gm, om, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gse, ose, rtol=1e-9, atol=1e-12)
    with pytest.raises(nv.HestonError) as e:
        _gpu_estimates(nv, BASE, cs + [cs[0]], n, N, 77, nv.HESTON_FP64)
    assert e.value.status == nv.HESTON_ERR_INVALID_ARG


@pytest.mark.parametrize("scheme,trunc", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0)])
@pytest.mark.parametrize("n,N,M", [(64 * 5 + 7, 9, 0), (1 << 12, 64, 4), (64 * 400 + 3, 21, 0), (3000, 50, 50)])
def test_small_launch_split_kernel_same_bits(nv, torch_cuda, scheme, trunc, n, N, M):
    """FP32 launches of fewer than 3 tiles per SM run two warps per tile, one
    path per lane (the one-path form of the step); the tile rows must be the
    packed kernel's bits, which an explicit launch shape selects -- for
    Milstein and Euler under both truncations and for QE (whose two branches
    the paper's Feller-violating set exercises)."""
    torch = torch_cuda
    cs = [(0, 100.0, 1.0, 0, 0), (1, 95.0, 1.0, 0, M), (0, 105.0, 1.0, 1, 0)]
    n_tiles = -(-n // 64)
    rows = []
    for block, grid in ((0, 0), (128, 0), (32, 7)):
        r = torch.full((n_tiles * 12 * len(cs),), float("nan"), dtype=torch.float64, device="cuda")
        opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream(), scheme=scheme,
                               trunc=trunc, block_threads=block, grid_ctas=grid)
        nv.heston_mc_launch_tiles(_gp(nv, PAPER), _gc(nv, cs), 64 * 1000, n, N, 11, opts, r)
        torch.cuda.synchronize()
        rows.append(r.cpu().numpy())
    assert np.isfinite(rows[0]).all()
    assert np.array_equal(rows[0], rows[1]) and np.array_equal(rows[0], rows[2])
