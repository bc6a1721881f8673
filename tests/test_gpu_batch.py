"""Batched persistent launch: each contract's result in the batch equals its
own launch bit for bit (same seed), the batch agrees with the oracle,
launch shape, repetition and CUDA-graph replay do not change bits, and the
cancel word stops the launch between work items."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv(cuda_lib):
    from paper_2309_10477_gb300 import native
    return native


def _items(nv, n=24, seed=3, trunc_asian_stride=True):
    g = np.random.default_rng(seed)
    items = []
    for i, d in enumerate(wl.batched_contracts(n, seed=seed)):
        n_steps = int(g.integers(1, 120))
        payoff, K, T, put, _ = d["contract"]
        M = 0
        if payoff == 1 and trunc_asian_stride and i % 3 == 0:
            M = max(1, n_steps // 3)
            n_steps = 3 * M                      # a strided Asian
        put = int(i % 4 == 1)
        items.append(nv.make_batch_item(nv.make_params(**d["params"]),
                                        nv.make_contract(payoff, K, T, put, M),
                                        int(g.integers(2, 6000)), n_steps, 1000 + 7 * i))
    return items


def _arr(results, nv):
    return np.array([[getattr(r, k) for k in nv.ESTIMATORS] + list(r.se) for r in results])


@pytest.mark.parametrize("trunc", [0, 1])
def test_batch_equals_each_contract_alone(nv, trunc):
    items = _items(nv)
    opts = nv.make_options(prec=nv.HESTON_FP32, trunc=trunc)
    got = _arr(nv.heston_mc_price_greeks_batch(items, opts), nv)
    for i, it in enumerate(items):
        alone = nv.heston_mc_price_greeks_ex(it.params, [it.contract], it.n_paths, it.n_steps,
                                             it.rng_seed, opts)
        assert np.array_equal(got[i], _arr(alone, nv)[0], equal_nan=True), i


def test_batch_matches_oracle(nv):
    items = _items(nv, n=8, seed=11)
    got = _arr(nv.heston_mc_price_greeks_batch(items, nv.make_options(prec=nv.HESTON_FP32)), nv)
    for i, it in enumerate(items):
        p = it.params
        P = oracle.Params(p.S0, p.v0, p.kappa, p.theta, p.xi, p.rho, p.r)
        c = it.contract
        om, ose = oracle.mc_price_greeks(P, [oracle.Contract(c.payoff, c.K, c.T, c.is_put, c.n_monitor)],
                                         it.n_paths, it.n_steps, it.rng_seed)
        d = np.abs(got[i, :6] - om[0])
        assert (d <= 3 * ose[0] + 1e-9).all(), i
        # 1e-4 of the FP64 oracle holds for every estimator when the variance stays
        # away from zero (Feller); otherwise the v0 / T tangents of the few paths that
        # come close to zero are ill-conditioned in FP32, and Vega and Theta are held
        # to 3 SE only
        rel = d <= 1e-4 * np.maximum(1.0, np.abs(om[0]))
        feller = 2 * p.kappa * p.theta >= p.xi**2
        check = [0, 1, 2, 4] + ([3, 5] if feller else [])
        assert rel[check].all(), (i, d, om[0])


def _prepared(nv, torch, items, opts):
    plan = nv.heston_batch_plan_make(items, opts)
    desc = torch.empty(plan.descriptor_bytes // 8 + 32, dtype=torch.float64, device="cuda")
    ws = torch.empty(plan.workspace_bytes // 8 + 32, dtype=torch.float64, device="cuda")
    nv.heston_batch_prepare(items, opts, plan, desc)
    return plan, desc, ws


def test_batch_launch_shape_repeat_and_graph_replay(nv):
    import torch
    items = _items(nv, n=40, seed=5)
    base = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
    plan, desc, ws = _prepared(nv, torch, items, base)
    out = torch.empty(len(items) * 12, dtype=torch.float64, device="cuda")
    nv.heston_mc_launch_batch(plan, desc, base, ws, out)
    torch.cuda.synchronize()
    ref = out.cpu().numpy().copy()
    for block, grid in ((32, 1), (64, 5), (128, 1000), (96, 0)):
        o = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream(),
                            block_threads=block, grid_ctas=grid)
        out.zero_()
        nv.heston_mc_launch_batch(plan, desc, o, ws, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), (block, grid)
    # capture the whole launch (memset + 3 kernels) in a CUDA graph and replay it
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    gout = torch.zeros_like(out)
    with torch.cuda.graph(graph, stream=s):
        o = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
        nv.heston_mc_launch_batch(plan, desc, o, ws, gout)
    for _ in range(2):
        gout.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(gout.cpu().numpy(), ref)


def test_batch_cancel_word(nv):
    import torch
    items = _items(nv, n=10, seed=7)
    opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
    plan, desc, ws = _prepared(nv, torch, items, opts)
    out = torch.empty(len(items) * 12, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    nv.heston_mc_launch_batch(plan, desc, opts, ws, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ok = out.cpu().numpy().copy()
    status.fill_(1)                        # cancel requested before the launch
    nv.heston_mc_launch_batch(plan, desc, opts, ws, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 2         # the kernel saw it and took no work
    status.zero_()
    nv.heston_mc_launch_batch(plan, desc, opts, ws, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and np.array_equal(out.cpu().numpy(), ok)


def test_batch_rejections(nv):
    items = _items(nv, n=3)
    with pytest.raises(nv.HestonError) as e:
        nv.heston_batch_plan_make(items, nv.make_options(prec=nv.HESTON_FP64))
    assert e.value.status == nv.HESTON_ERR_UNSUPPORTED
    bad = list(items)
    bad[1] = nv.make_batch_item(items[1].params, items[1].contract, 1, 10, 1)
    with pytest.raises(nv.HestonError) as e:
        nv.heston_batch_plan_make(bad, nv.make_options(prec=nv.HESTON_FP32))
    assert e.value.status == nv.HESTON_ERR_INVALID_ARG


def test_unstable_tangents_are_flagged(nv):
    # far from the Feller condition with many steps the v0 / T tangents blow up
    p = nv.make_params(100.0, 0.05, 5.0, 0.01, 0.9, -0.7, 0.03)
    c = [nv.make_contract(0, 100.0, 1.0)]
    lib = nv.load()
    import ctypes
    out = (nv.heston_result * 1)()
    arr = (nv.heston_contract * 1)(*c)
    opts = nv.make_options(prec=nv.HESTON_FP32)
    rc = lib.heston_mc_price_greeks_ex(ctypes.byref(p), arr, 1, 1 << 16, 400, 1, ctypes.byref(opts), out)
    r = out[0]
    finite = all(np.isfinite([r.vega, r.theta, r.se[3], r.se[5]]))
    assert (rc == nv.HESTON_WARN_TANGENT_UNSTABLE) == (not finite)
    assert np.isfinite([r.price, r.delta, r.gamma, r.rho]).all()


def test_full_batched_mix_sampled_against_the_oracle(nv):
    """The 1024-contract seeded mix of the batched benchmark (K~U[70,130],
    T in {0.25,0.5,1,2}, paths 2^14..2^20, steps 50..500, European/Asian),
    priced in one persistent launch with the benchmark's per-contract seeds.
    The four contracts with the least work are recomputed at full size by
    the FP64 oracle: every estimate within 3 SE, and price, Delta, Gamma and
    Rho (Vega/Theta too where Feller holds) within 1e-4 of the oracle."""
    w = wl.multi_strike_fp32()
    mix = wl.batched_contracts(1024)
    items = [nv.make_batch_item(nv.make_params(**d["params"]), nv.make_contract(*d["contract"]),
                                d["n_paths"], d["n_steps"], w.seed + 1000003 * i)
             for i, d in enumerate(mix)]
    got = _arr(nv.heston_mc_price_greeks_batch(items, nv.make_options(prec=nv.HESTON_FP32)), nv)
    work = [d["n_paths"] * d["n_steps"] for d in mix]
    for i in np.argsort(work)[:4]:
        it, d = items[i], mix[i]
        P = oracle.Params(**d["params"])
        om, ose = oracle.mc_price_greeks(P, [oracle.Contract(*d["contract"])], it.n_paths,
                                         it.n_steps, it.rng_seed)
        diff = np.abs(got[i, :6] - om[0])
        assert (diff <= 3 * ose[0] + 1e-9).all(), (i, diff, ose[0])
        p = d["params"]
        check = [0, 1, 2, 4] + ([3, 5] if 2 * p["kappa"] * p["theta"] >= p["xi"] ** 2 else [])
        assert (diff[check] <= 1e-4 * np.maximum(1.0, np.abs(om[0][check]))).all(), (i, diff, om[0])
