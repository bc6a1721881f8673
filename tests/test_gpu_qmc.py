"""GPU randomised-QMC variant (Sobol + digital shifts + Brownian bridge) vs
the FP64 oracle's independent implementation, through the C ABI.  Same
tolerances as the Philox parity tests (per path 1e-5 relative in FP32 plus
the measured change under the FP32 normal-error bound, here the bridge's,
branch flips counted; estimates within 3 SE and 1e-4 * max(1, |oracle|))."""
import numpy as np
import pytest

import oracle
from conditioning import check_paths, qmc_paths_with_sensitivity
from oracle import sobol
from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BASE = wl.BASE_PARAMS
PSETS = {"base": wl.BASE_PARAMS, "paper": wl.PAPER_PARAMS}


@pytest.fixture(scope="module")
def nv(cuda_lib):
    from paper_2309_10477_gb300 import native
    return native


def _oc(cs):
    return [oracle.Contract(*c) for c in cs]


def _gc(nv, cs):
    return [nv.make_contract(*c) for c in cs]


def _flips(rec, cs, params, N):
    near_zero = rec[:, 14] < 1e-5 * max(params["theta"], params["v0"])
    A_euro = params["S0"] * np.exp(rec[:, 0])
    near_k = np.zeros(len(rec), bool)
    for c in cs:
        M = c[4] or N
        A = A_euro if c[0] == 0 else rec[:, 6] / M
        near_k |= np.abs(A - c[1]) < 2e-5 * max(c[1], 1.0)
    return near_zero | near_k


@pytest.mark.parametrize("pset", ["base", "paper"])
@pytest.mark.parametrize("N,trunc", [(1, 0), (7, 0), (64, 0), (252, 0), (64, 1)])
def test_qmc_per_path(nv, pset, N, trunc):
    """Every record field and per-path estimator of chosen Sobol points against
    the oracle on its own QMC normals: |gpu - oracle| <= 1e-5 * scale + 4 *
    change, the change measured with the normals moved within the FP32
    bridge's error bound (it grows with the path's |W|, see qmc_normal_bound).
    The paper's parameter set (far from the Feller condition) drives paths
    near V = 0, where the tangents need the change term."""
    params = PSETS[pset]
    cs = [(0, 100.0, 1.0, 0, 0), (1, 95.0, 1.0, 0, 0), (0, 105.0, 1.0, 1, 0)]
    rep = 3
    pts = np.concatenate([np.arange(0, 300), [4095, 4096, 123457, 2**20 + 77, 2**31 + 5]])
    opts = nv.make_options(trunc=trunc, prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=4)
    rec_g, est_g = nv.heston_qmc_debug_paths(nv.make_params(**params), _gc(nv, cs), N, 42, opts, rep, pts)
    za, zb = sobol.qmc_normals(sobol.direction_numbers(2 * N), sobol.BridgePlan(N), 42, rep, pts)
    rec_o, est_o, drec, dest = qmc_paths_with_sensitivity(params, cs, za, zb, trunc, seed=42)
    flips = _flips(rec_o, cs, params, N)
    assert flips.sum() <= 2
    check_paths(rec_g, est_g, rec_o, est_o, drec, dest, params, cs, N, ~flips, 1e-5, (pset, N, trunc))


# N = 2048 is the largest step count; its bridge plan and Sobol rows need more
# than 48 KB of shared memory per block, which the launch opts in to.  (252,
# 2^17, 2): the bench's points per replicate and steps -- each replicate's tiles
# are those of the bench's 32-replicate launch, whatever the replicate count.
@pytest.mark.parametrize("N,P,R", [(50, 4096, 8), (252, 1024, 4), (2048, 64, 8), (252, 1 << 17, 2)])
def test_qmc_estimates_match_oracle(nv, N, P, R):
    cs = [(0, 90.0, 1.0, 0, 0), (0, 110.0, 1.0, 0, 0), (1, 100.0, 1.0, 0, 0), (1, 100.0, 1.0, 1, 0)]
    opts = nv.make_options(prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=R)
    res = nv.heston_mc_price_greeks_ex(nv.make_params(**BASE), _gc(nv, cs), R * P, N, 9, opts)
    gm, gse = nv.results_to_arrays(res)
    om, ose, _ = sobol.qmc_price_greeks(oracle.Params(**BASE), _oc(cs), R, P, N, 9)
    d = np.abs(gm - om)
    assert (d <= 3 * ose + 1e-12).all(), np.max(d / (ose + 1e-300))
    assert (d <= 1e-4 * np.maximum(1.0, np.abs(om))).all()
    np.testing.assert_allclose(gse, ose, rtol=2e-2, atol=1e-6)


def test_qmc_async_launch_matches_sync_and_full_size_runs(nv):
    import torch
    w = wl.multi_strike_fp32()
    cs = _gc(nv, w.contracts)
    R, N = 32, w.n_steps
    params = nv.make_params(**w.params)
    tb_bytes = nv.heston_qmc_tables_bytes(N)
    tables = torch.empty(tb_bytes // 8 + 1, dtype=torch.float64, device="cuda")
    nv.heston_qmc_build_tables(N, tables, tb_bytes)
    for n in (R * 2048, w.n_paths):
        ws_bytes = nv.heston_mc_workspace_bytes_qmc(len(cs), n, N, R)
        ws = torch.empty(ws_bytes // 8 + 1, dtype=torch.float64, device="cuda")
        out = torch.empty(len(cs) * 12, dtype=torch.float64, device="cuda")
        opts = nv.make_options(prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=R,
                               stream=torch.cuda.current_stream())
        nv.heston_mc_launch_qmc(params, cs, n, N, w.seed, opts, tables, ws, ws_bytes, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(len(cs), 12)
        assert np.isfinite(got).all()
        if n < w.n_paths:
            sync = nv.results_to_arrays(nv.heston_mc_price_greeks_ex(params, cs, n, N, w.seed, opts))
            assert np.array_equal(got[:, :6], sync[0]) and np.array_equal(got[:, 6:], sync[1])
    # full size: QMC and Philox MC agree within their combined standard errors
    mc = nv.results_to_arrays(nv.heston_mc_price_greeks_ex(
        params, cs, w.n_paths, N, w.seed, nv.make_options(prec=nv.HESTON_FP32)))
    d = np.abs(got[:, :6] - mc[0])
    assert (d <= 4 * np.hypot(got[:, 6:], mc[1]) + 1e-9).all()
    assert (got[:, 6] < mc[1][:, 0]).all()       # price SE: bridge-QMC below Philox MC


def test_qmc_rejections(nv):
    p = nv.make_params(**BASE)
    cs = [nv.make_contract(0, 100.0, 1.0)]
    with pytest.raises(nv.HestonError) as e:
        nv.heston_mc_price_greeks_ex(p, cs, 4096, 16, 1, nv.make_options(
            prec=nv.HESTON_FP64, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=4))
    assert e.value.status == nv.HESTON_ERR_UNSUPPORTED
    for n_paths, n_shifts in ((4096, 1), (4096 + 64, 3), (4096 * 3 + 3, 3)):
        with pytest.raises(nv.HestonError) as e:
            nv.heston_mc_price_greeks_ex(p, cs, n_paths, 16, 1, nv.make_options(
                prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=n_shifts))
        assert e.value.status == nv.HESTON_ERR_INVALID_ARG


def test_qmc_estimates_are_the_sums_of_the_per_path_records(nv):
    """The QMC path kernel (two paths per lane, packed FP32 step) and the QMC
    per-path record kernel (one path per thread, scalar step; the one the
    per-path test above checks against the oracle) compute the same paths:
    the launch's estimates equal those rebuilt on the host from the per-path
    records -- exactly rounded FP32 tile sums (lane l adds points l and
    l + 32 of its 64-point tile, then a xor butterfly), FP64 sums over each
    replicate's tiles, the mean over replicates -- to 1e-12, far below one
    FP32 rounding of any path."""
    from fractions import Fraction
    from exact_rounding import round_exact
    cs = [(0, 100.0, 1.0, 0, 0), (1, 95.0, 1.0, 0, 0), (0, 105.0, 1.0, 1, 0)]
    R, P, N, seed = 4, 128, 30, 7
    opts = nv.make_options(prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=R)
    gm, gse = nv.results_to_arrays(nv.heston_mc_price_greeks_ex(
        nv.make_params(**BASE), _gc(nv, cs), R * P, N, seed, opts))
    rnd = lambda q: round_exact(q, 24)
    rep_means = np.zeros((R, len(cs), 6))
    for r in range(R):
        _, est = nv.heston_qmc_debug_paths(nv.make_params(**BASE), _gc(nv, cs), N, seed, opts, r,
                                           np.arange(P, dtype=np.uint32))
        acc = np.zeros((len(cs), 6))
        for t in range(P // 64):
            for c in range(len(cs)):
                for j in range(6):
                    x = est[t * 64:(t + 1) * 64, c, j]
                    v = [rnd(Fraction(x[l]) + Fraction(x[l + 32])) for l in range(32)]
                    for o in (16, 8, 4, 2, 1):
                        v = [rnd(Fraction(v[l]) + Fraction(v[l ^ o])) for l in range(32)]
                    acc[c, j] += v[0]
        rep_means[r] = acc / P
    mean = rep_means.mean(axis=0)
    se = rep_means.std(axis=0, ddof=1) / np.sqrt(R)
    np.testing.assert_allclose(gm, mean, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gse, se, rtol=1e-9, atol=1e-14)


def test_qmc_launch_shape_does_not_change_bits(nv):
    """The QMC kernel stages one row of Sobol words per warp in shared memory,
    sized by the block: other grid and block shapes give the same bits."""
    cs = [(0, 100.0, 1.0, 0, 0), (1, 95.0, 1.0, 0, 0), (1, 105.0, 1.0, 1, 0)]
    R, P, N = 4, 1024, 61
    ref = None
    for grid, block in ((0, 0), (3, 64), (0, 32), (700, 128)):
        opts = nv.make_options(prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=R,
                               grid_ctas=grid, block_threads=block)
        got = np.concatenate(nv.results_to_arrays(nv.heston_mc_price_greeks_ex(
            nv.make_params(**BASE), _gc(nv, cs), R * P, N, 3, opts)), axis=1)
        if ref is None:
            ref = got
        assert np.array_equal(got, ref), (grid, block)
