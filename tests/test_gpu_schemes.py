"""Euler and QE schemes on the GPU against the FP64 oracle, on identical
Philox normals, through the C ABI.

Tolerances as for the Milstein path (tests/test_gpu_parity.py):
  * per path, FP64: every record field and estimator within 1e-12 of its
    scale (tests/conditioning.py path_scales) plus four times the oracle's
    own change when its normals move by a few ulp; paths whose branch
    decision lies within 1e-9 * max(theta, v0) of its threshold (a
    truncation sign, the QE switch psi = 1.5 or the QE zero mass) are
    counted, not compared.
  * per path, FP32: every record field (ln S_T, V_T, tangents, Asian sums,
    Gamma weights) and per-path estimator within 1e-5 of its scale plus four
    times the oracle's own change under FP32-rounded inputs and normals
    moved within the FP32 normal-error bound; paths within 1e-5 (QE) or 1e-4
    (Euler) * max(theta, v0) of a branch decision, or with A within 2e-5 K
    of the strike, are counted, not compared (at most 3 % of the sample: QE
    on a Feller-violating set meets its zero-mass threshold often).
  * estimates: FP64 within 1e-9 relative; FP32 within 3 standard errors and
    1e-4 * max(1, |oracle|) wherever the estimate is well-conditioned at FP32
    precision (tests/conditioning.py: the oracle's own change under
    FP32-sized perturbations stays below a third of the bound).
"""
import numpy as np
import pytest

import oracle
from conditioning import (check_fp32_estimates, check_paths, oracle_paths_with_sensitivity,
                          oracle_with_sensitivity)
from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BASE = wl.BASE_PARAMS
PAPER = wl.PAPER_PARAMS
SCHEMES = [("euler", 1, 0), ("euler-floor", 1, 1), ("qe", 2, 0)]
CS = [(0, 100.0, 1.0, 0, 0), (1, 95.0, 1.0, 0, 0), (0, 105.0, 1.0, 1, 0), (1, 100.0, 1.0, 1, 0)]


@pytest.fixture(scope="module")
def nv(cuda_lib):
    from paper_2309_10477_gb300 import native
    return native


def _gp(nv, d):
    return nv.make_params(**d)


def _gc(nv, cs):
    return [nv.make_contract(*c) for c in cs]


def _oc(cs):
    return [oracle.Contract(*c) for c in cs]


def _paths():
    return np.concatenate([np.arange(0, 600), 2**32 - 3 + np.arange(6),
                           2**36 + 11 * np.arange(40)]).astype(np.uint64)


def _near_strike(rec_o, cs, S0, N, tol):
    A_euro = S0 * np.exp(rec_o[:, 0])
    near = np.zeros(len(rec_o), bool)
    for c in cs:
        A = A_euro if c[0] == 0 else rec_o[:, 6] / (c[4] or N)
        near |= np.abs(A - c[1]) < tol * max(c[1], 1.0)
    return near


@pytest.mark.parametrize("name,scheme,trunc", SCHEMES)
@pytest.mark.parametrize("pname,params,N", [("base", BASE, 1), ("base", BASE, 7), ("base", BASE, 64),
                                            ("paper", PAPER, 3), ("paper", PAPER, 128)])
def test_per_path_fp64(nv, name, scheme, trunc, pname, params, N):
    paths = _paths()
    opts = nv.make_options(trunc=trunc, prec=nv.HESTON_FP64, scheme=scheme)
    rec_g, est_g = nv.heston_mc_debug_paths(_gp(nv, params), _gc(nv, CS), N, 42, opts, paths)
    rec_o, est_o, drec, dest = oracle_paths_with_sensitivity(params, CS, paths, N, 42, trunc, scheme,
                                                             prec="fp64")
    flips = rec_o[:, 14] < 1e-9 * max(params["theta"], params["v0"])
    assert flips.sum() <= 1
    check_paths(rec_g, est_g, rec_o, est_o, drec, dest, params, CS, N, ~flips, 1e-12, name)


@pytest.mark.parametrize("name,scheme,trunc", SCHEMES)
@pytest.mark.parametrize("pname,params,N", [("base", BASE, 7), ("base", BASE, 252),
                                            ("paper", PAPER, 64), ("paper", PAPER, 128)])
def test_per_path_fp32(nv, name, scheme, trunc, pname, params, N):
    paths = _paths()
    opts = nv.make_options(trunc=trunc, prec=nv.HESTON_FP32, scheme=scheme)
    rec_g, est_g = nv.heston_mc_debug_paths(_gp(nv, params), _gc(nv, CS), N, 42, opts, paths)
    rec_o, est_o, drec, dest = oracle_paths_with_sensitivity(params, CS, paths, N, 42, trunc, scheme)
    vs = max(params["theta"], params["v0"])
    # Paths near a branch decision are counted, not compared.  Euler: within
    # eps of V = 0, sqrt(V) turns an FP32 rounding error d in V into an error of
    # about xi sqrt(dt) d |Z| / (2 sqrt(eps)) in the next variance step; with
    # the paper's xi = 0.61, dt = 1/128, d ~ 2e-9 and |Z| ~ 3 that passes the
    # 1e-5 * vs tolerance for eps below about 4e-5 vs, so the band is 1e-4 vs.
    # QE's field is the distance of its branch switches (psi = 1.5, the zero
    # mass), which no square root of V amplifies: 1e-5 vs.
    band = 1e-5 if scheme == nv.HESTON_SCHEME_QE else 1e-4
    flips = (rec_o[:, 14] < band * vs) | _near_strike(rec_o, CS, params["S0"], N, 2e-5)
    assert flips.sum() <= max(2, 0.03 * len(paths)), flips.sum()
    # every record field and per-path estimator: 1e-5 of its scale plus four
    # times the oracle's own change under FP32-sized perturbations.  QE's
    # v0- and T-tangents differentiate psi = s^2 / m^2, whose derivative
    # subtracts two nearly equal terms (s^2_v / s^2 and 2 m_v / m both follow
    # V_v): the cancellation amplifies the FP32 rounding of the tangent
    # formulas themselves, which perturbing the inputs does not model; those
    # fields (X_v, V_v, X_T, V_T, the Asian tangent sums, Vega, Theta) are
    # held to 5e-5 of their scale (measured: up to 2.1e-5)
    rel = 1e-5
    if scheme == nv.HESTON_SCHEME_QE:
        rel = np.full(14, 1e-5)
        rel[[2, 3, 4, 5, 8, 9]] = 5e-5
        rel_e = np.array([1e-5, 1e-5, 1e-5, 5e-5, 1e-5, 5e-5])
        rel = (rel, rel_e)
    n_wide = check_paths(rec_g, est_g, rec_o, est_o, drec, dest, params, CS, N, ~flips, rel, name)
    assert n_wide <= 0.05 * (~flips).sum() * (14 + 6 * len(CS)), n_wide


def _gpu_estimates(nv, params, cs, n, N, seed, prec, trunc, scheme):
    res = nv.heston_mc_price_greeks_ex(_gp(nv, params), _gc(nv, cs), n, N, seed,
                                       nv.make_options(trunc=trunc, prec=prec, scheme=scheme))
    return nv.results_to_arrays(res)


@pytest.mark.parametrize("name,scheme,trunc", SCHEMES)
@pytest.mark.parametrize("n,N", [(2, 1), (65, 3), (2381, 50), ((1 << 15) + 5, 20)])
def test_estimates_fp64_match_oracle(nv, name, scheme, trunc, n, N):
    gm, gse = _gpu_estimates(nv, BASE, CS, n, N, 7, nv.HESTON_FP64, trunc, scheme)
    om, ose = oracle.mc_price_greeks(oracle.Params(**BASE), _oc(CS), n, N, 7, trunc, scheme=scheme)
    np.testing.assert_allclose(gm, om, rtol=1e-9, atol=1e-11)
    floor = 1e-7 * np.maximum(1.0, np.abs(om))
    assert (np.abs(gse - ose) <= 1e-6 * ose + floor).all()


@pytest.mark.parametrize("name,scheme,trunc", SCHEMES)
@pytest.mark.parametrize("params", [BASE, PAPER], ids=["base", "paper"])
def test_estimates_fp32_match_oracle(nv, name, scheme, trunc, params):
    """Within 3 SE and 1e-4 of the FP64 oracle wherever the estimate is
    well-conditioned at FP32 precision (tests/conditioning.py).  On the
    paper's Feller-violating set the Euler and QE Vega and Theta are not:
    the oracle's own values move by more than a third of the bound under
    FP32-sized perturbations (Euler, with no Milstein term, reaches V < 0
    often enough for its Vega to come close even on the base set).  Price,
    Delta, Gamma and Rho are well-conditioned everywhere here."""
    w = wl.multi_strike_fp32(1 << 16)
    gm, gse = _gpu_estimates(nv, params, w.contracts, w.n_paths, w.n_steps, 3, nv.HESTON_FP32,
                             trunc, scheme)
    om, ose, delta = oracle_with_sensitivity(params, w.contracts, w.n_paths, w.n_steps, 3, trunc, scheme)
    ill = check_fp32_estimates(gm, om, ose, delta, name)
    assert not ill[:, [0, 1, 2, 4]].any()            # price, Delta, Gamma, Rho always well-conditioned here


@pytest.mark.parametrize("scheme", [1, 2])
def test_full_size_sampled_paths(nv, scheme):
    """Bench-size indices (2^22 paths, 252 steps, 6 contracts, FP32): sampled
    paths up to the last one agree with the oracle."""
    w = wl.multi_strike_fp32()
    idx = np.unique(np.concatenate([[0, 1, w.n_paths - 1],
                                    np.random.default_rng(3).integers(0, w.n_paths, 300)]))
    idx = idx.astype(np.uint64)
    opts = nv.make_options(prec=nv.HESTON_FP32, scheme=scheme)
    rec_g, est_g = nv.heston_mc_debug_paths(_gp(nv, w.params), _gc(nv, w.contracts), w.n_steps,
                                            w.seed, opts, idx)
    rec_o, est_o = oracle.debug_paths(oracle.Params(**w.params), _oc(w.contracts), idx, w.n_steps,
                                      w.seed, 0, scheme)
    vs = max(w.params["theta"], w.params["v0"])
    ok = ~((rec_o[:, 14] < 1e-5 * vs) | _near_strike(rec_o, w.contracts, w.params["S0"],
                                                    w.n_steps, 2e-5))
    assert ok.sum() >= len(idx) - 3
    assert (np.abs(rec_g[ok, 0] - rec_o[ok, 0]) <= 1e-5 * np.maximum(1, np.abs(rec_o[ok, 0]))).all()
    assert (np.abs(rec_g[ok, 6] - rec_o[ok, 6]) <= 1e-5 * rec_o[ok, 6]).all()


def test_launch_shape_does_not_change_qe_bits(nv):
    import torch
    cs = CS
    n, N = 64 * 300 + 7, 30
    outs = []
    for grid, block in ((0, 0), (5, 64), (200, 128)):
        ws_bytes = nv.heston_mc_workspace_bytes(len(cs), n)
        ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda")
        out = torch.empty(len(cs) * 12, dtype=torch.float64, device="cuda")
        opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream(),
                               grid_ctas=grid, block_threads=block, scheme=nv.HESTON_SCHEME_QE)
        nv.heston_mc_launch(_gp(nv, BASE), _gc(nv, cs), n, N, 9, opts, ws, ws_bytes, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_scheme_argument_errors(nv):
    c = _gc(nv, CS[:1])
    for bad in (dict(BASE, xi=0.0), dict(BASE, kappa=0.0), dict(BASE, theta=0.0)):
        with pytest.raises(nv.HestonError) as e:
            nv.heston_mc_price_greeks_ex(_gp(nv, bad), c, 64, 4, 1,
                                         nv.make_options(scheme=nv.HESTON_SCHEME_QE))
        assert e.value.status == nv.HESTON_ERR_INVALID_ARG
    with pytest.raises(nv.HestonError) as e:
        nv.heston_mc_price_greeks_ex(_gp(nv, BASE), c, 64, 4, 1, nv.make_options(scheme=3))
    assert e.value.status == nv.HESTON_ERR_INVALID_ARG
    with pytest.raises(nv.HestonError) as e:
        nv.heston_mc_price_greeks_ex(_gp(nv, BASE), c, 1 << 10, 4, 1,
                                     nv.make_options(prec=nv.HESTON_FP32, rng=nv.HESTON_RNG_SOBOL_BB,
                                                     n_shifts=4, scheme=nv.HESTON_SCHEME_EULER))
    assert e.value.status == nv.HESTON_ERR_UNSUPPORTED
    item = nv.make_batch_item(_gp(nv, BASE), c[0], 256, 8, 1)
    with pytest.raises(nv.HestonError) as e:
        nv.heston_batch_plan_make([item], nv.make_options(prec=nv.HESTON_FP32,
                                                          scheme=nv.HESTON_SCHEME_QE))
    assert e.value.status == nv.HESTON_ERR_UNSUPPORTED
