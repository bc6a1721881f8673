"""Adjoint (reverse-mode) gradient kernels vs the oracle's forward-mode
gradient on identical normals, vs the main kernel's Greek estimators on the
same paths, and through torch.autograd."""
import numpy as np
import pytest

import oracle
from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BASE = wl.BASE_PARAMS
NAMES = ("S0", "v0", "kappa", "theta", "xi", "rho", "r")


@pytest.fixture(scope="module")
def nv(cuda_lib):
    from paper_2309_10477_gb300 import native
    return native


def _run(nv, torch, params, c, n, N, seed):
    p = nv.make_params(**params)
    ws_bytes = nv.heston_adjoint_workspace_bytes(n, N)
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    g = torch.empty(14, dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
    nv.heston_mc_adjoint_forward(p, c, n, N, seed, opts, ws, ws_bytes, out)
    nv.heston_mc_adjoint_backward(p, c, n, N, seed, opts, ws, ws_bytes, g)
    torch.cuda.synchronize()
    return out.cpu().numpy(), g.cpu().numpy()


# segments of 8 steps: N = 7 and 300 end on a short segment, 1024 is the largest N
@pytest.mark.parametrize("payoff,put,M,N,n", [(0, 0, 0, 64, 1 << 15), (1, 0, 0, 252, 1 << 14),
                                              (1, 1, 4, 32, (1 << 15) + 37), (0, 1, 0, 7, 5000),
                                              (1, 0, 0, 300, 4096 + 5), (0, 0, 0, 1024, 2048)])
def test_adjoint_matches_oracle_forward_mode(nv, payoff, put, M, N, n):
    import torch
    c = nv.make_contract(payoff, 100.0, 1.0, put, M)
    price, g = _run(nv, torch, BASE, c, n, N, 17)
    om, ose = oracle.mc_gradient(oracle.Params(**BASE), oracle.Contract(payoff, 100.0, 1.0, put, M),
                                 n, N, 17)
    gm = np.concatenate([[price[0]], g[:7]])
    d = np.abs(gm - om)
    assert (d <= 3 * ose + 1e-9).all(), (d, ose)
    assert (d <= 1e-4 * np.maximum(1.0, np.abs(om))).all(), (d, om)
    np.testing.assert_allclose(np.concatenate([[price[1]], g[7:]]), ose, rtol=2e-3, atol=1e-9)


def test_adjoint_full_size_against_the_greek_estimators(nv):
    """252-step Asian call, 2^20 paths: the S0, v0 and r components are the
    Delta, Vega and Rho of the main kernel on the same paths."""
    import torch
    c = nv.make_contract(1, 100.0, 1.0)
    n, N = 1 << 20, 252
    price, g = _run(nv, torch, BASE, c, n, N, 42)
    res = nv.heston_mc_price_greeks_ex(nv.make_params(**BASE), [c], n, N, 42,
                                       nv.make_options(prec=nv.HESTON_FP32))
    m, se = nv.results_to_arrays(res)
    for got, k in ((price[0], 0), (g[0], 1), (g[1], 3), (g[6], 4)):
        assert abs(got - m[0, k]) <= 1e-4 * max(1.0, abs(m[0, k])), (k, got, m[0, k])
    assert np.isfinite(g).all()


def test_autograd_function(nv):
    import torch
    from paper_2309_10477_gb300 import autograd as ag
    c = nv.make_contract(0, 100.0, 1.0)
    theta = torch.tensor([BASE[k] for k in NAMES], dtype=torch.float64, requires_grad=True)
    price = ag.heston_price(theta, c, 1 << 14, 50, 5)
    (grad,) = torch.autograd.grad(2.0 * price, theta)
    p, g = _run(nv, torch, BASE, c, 1 << 14, 50, 5)
    assert float(price.detach()) == p[0]
    assert np.array_equal(grad.numpy(), 2.0 * g[:7])


def test_adjoint_rejections(nv):
    import torch
    c = nv.make_contract(0, 100.0, 1.0)
    p = nv.make_params(**BASE)
    ws = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    out = torch.empty(14, dtype=torch.float64, device="cuda")
    for opts in (nv.make_options(prec=nv.HESTON_FP64), nv.make_options(prec=nv.HESTON_FP32, trunc=1)):
        with pytest.raises(nv.HestonError) as e:
            nv.heston_mc_adjoint_forward(p, c, 1024, 10, 1, opts, ws, 8 << 20, out)
        assert e.value.status == nv.HESTON_ERR_UNSUPPORTED
    for N in (1025, 2000):                       # beyond the 1024-step limit
        with pytest.raises(nv.HestonError) as e:
            nv.heston_adjoint_workspace_bytes(1024, N)
        assert e.value.status == nv.HESTON_ERR_UNSUPPORTED


@pytest.mark.parametrize("payoff,put,M,N,n", [(0, 0, 0, 64, 3000), (1, 0, 0, 252, 1500),
                                              (1, 1, 4, 32, 700 + 37), (0, 1, 0, 7, 500)])
def test_adjoint_per_path_against_the_oracle(nv, payoff, put, M, N, n):
    """The adjoint kernels' per-path payoff and its 7 derivatives (the FP32
    values the estimates sum) against the oracle's forward-mode gradient on
    the same normals: within max(1e-5, 2 N 2^-24) of each component's scale
    (max(|x|, the sample's median |x|); the payoff max(K, A)) plus four times the oracle's
    own change under FP32-rounded inputs and normals moved within the FP32
    normal-error bound.  Paths whose truncation branch or payoff indicator
    can flip between FP32 and FP64 are counted, not compared."""
    import torch
    from conditioning import oracle_gradients_with_sensitivity
    contract = (payoff, 100.0, 1.0, put, M)
    c = nv.make_contract(*contract)
    p = nv.make_params(**BASE)
    ws_bytes = nv.heston_adjoint_workspace_bytes(n, N) + 768
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device="cuda")
    per = torch.empty(n * 8, dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
    nv.heston_mc_adjoint_debug_paths(p, c, n, N, 23, opts, ws, ws_bytes, per)
    torch.cuda.synchronize()
    got = per.view(n, 8).cpu().numpy()
    paths = np.arange(n, dtype=np.uint64)
    og, dg = oracle_gradients_with_sensitivity(BASE, contract, paths, N, 23)
    rec, _ = oracle.debug_paths(oracle.Params(**BASE), [oracle.Contract(*contract)], paths, N, 23)
    A = BASE["S0"] * np.exp(rec[:, 0]) if payoff == 0 else rec[:, 6] / (M or N)
    flips = (rec[:, 14] < 1e-5 * max(BASE["theta"], BASE["v0"])) | (np.abs(A - 100.0) < 2e-5 * 100.0)
    assert flips.sum() <= max(2, n // 1000)
    ok = ~flips
    scale = np.maximum(np.abs(og), np.median(np.abs(og), axis=0))
    scale[:, 0] = np.maximum(scale[:, 0], np.maximum(A, 100.0))
    # each derivative comes out of two FP32 recursions over the N steps: the
    # adjoint state (V-bar, X-bar, carried backwards) and the running sum of its
    # contributions; their rounding bounds each grow like N u (u = 2^-24), so
    # the tolerance is 1e-5 or 2 N u, the larger
    rel = max(1e-5, 2.0 * N * 2.0 ** -24)
    lim = rel * scale + 4.0 * dg
    d = np.abs(got - og)
    assert (d[ok] <= lim[ok]).all(), ((d / lim)[ok].max(axis=0), np.argwhere((d > lim) & ok[:, None])[:5])
    assert (d[ok] > rel * scale[ok]).sum() <= 0.05 * ok.sum() * 8
