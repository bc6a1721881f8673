"""Batched persistent launch: each contract's result in the batch equals its
own launch bit for bit (same seed), the batch agrees with the oracle,
launch shape, repetition and CUDA-graph replay do not change bits, and the
cancel word stops the launch between work items."""
import ctypes

import numpy as np
import pytest

import oracle
from conditioning import WELL, check_fp32_estimates, oracle_with_sensitivity
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


def _oracle_contract(it):
    p, c = it.params, it.contract
    params = dict(S0=p.S0, v0=p.v0, kappa=p.kappa, theta=p.theta, xi=p.xi, rho=p.rho, r=p.r)
    return params, (c.payoff, c.K, c.T, c.is_put, c.n_monitor)


def test_batch_matches_oracle(nv):
    """Every estimate within 3 SE and 1e-4 of the FP64 oracle where it is
    well-conditioned at FP32 precision (the oracle's own change under FP32
    input rounding and FP32-sized normal errors, tests/conditioning.py)."""
    items = _items(nv, n=8, seed=11)
    got = _arr(nv.heston_mc_price_greeks_batch(items, nv.make_options(prec=nv.HESTON_FP32)), nv)
    for i, it in enumerate(items):
        params, c = _oracle_contract(it)
        om, ose, delta = oracle_with_sensitivity(params, [c], it.n_paths, it.n_steps, it.rng_seed)
        check_fp32_estimates(got[i, :6][None], om, ose, delta, str(i))


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
    """Far from the Feller condition with many steps the v0 / T tangents blow
    up: the GPU flags HESTON_WARN_TANGENT_UNSTABLE exactly when Vega or Theta
    (or their SE) is not finite, and the FP64 oracle on the same normals is
    itself ill-conditioned there (its Vega / Theta move by more than the
    bound under FP32-sized perturbations)."""
    params = dict(S0=100.0, v0=0.05, kappa=5.0, theta=0.01, xi=0.9, rho=-0.7, r=0.03)
    p = nv.make_params(**params)
    c = [nv.make_contract(0, 100.0, 1.0)]
    lib = nv.load()
    out = (nv.heston_result * 1)()
    arr = (nv.heston_contract * 1)(*c)
    opts = nv.make_options(prec=nv.HESTON_FP32)
    rc = lib.heston_mc_price_greeks_ex(ctypes.byref(p), arr, 1, 1 << 16, 400, 1, ctypes.byref(opts), out)
    r = out[0]
    finite = all(np.isfinite([r.vega, r.theta, r.se[3], r.se[5]]))
    assert (rc == nv.HESTON_WARN_TANGENT_UNSTABLE) == (not finite)
    assert np.isfinite([r.price, r.delta, r.gamma, r.rho]).all()
    om, ose, delta = oracle_with_sensitivity(params, [(0, 100.0, 1.0, 0, 0)], 1 << 16, 400, 1)
    gm = np.array([[r.price, r.delta, r.gamma, r.vega, r.rho, r.theta]])
    ill = check_fp32_estimates(gm, om, ose, delta, "kappa 5, theta 0.01, xi 0.9, 400 steps")
    assert ill[0, [3, 5]].all(), delta


def _mix_items(nv):
    w = wl.multi_strike_fp32()
    mix = wl.batched_contracts(1024)
    items = [nv.make_batch_item(nv.make_params(**d["params"]), nv.make_contract(*d["contract"]),
                                d["n_paths"], d["n_steps"], w.seed + 1000003 * i)
             for i, d in enumerate(mix)]
    return mix, items


def test_full_batched_mix_sampled_against_the_oracle(nv):
    """The 1024-contract seeded mix of the batched benchmark (K~U[70,130],
    T in {0.25,0.5,1,2}, paths 2^14..2^20, steps 50..500, European/Asian),
    priced in one persistent launch with the benchmark's per-contract seeds.
    The four contracts with the least work and 12 more drawn at random are
    recomputed at full size by the FP64 oracle: every well-conditioned
    estimate within 3 SE and 1e-4 of it (tests/conditioning.py)."""
    mix, items = _mix_items(nv)
    got = _arr(nv.heston_mc_price_greeks_batch(items, nv.make_options(prec=nv.HESTON_FP32)), nv)
    work = np.array([d["n_paths"] * d["n_steps"] for d in mix])
    pick = list(np.argsort(work)[:4]) + list(np.random.default_rng(5).choice(1024, 12, replace=False))
    n_ill = 0
    for i in pick:
        it, d = items[i], mix[i]
        om, ose, delta = oracle_with_sensitivity(d["params"], [d["contract"]], it.n_paths,
                                                 it.n_steps, it.rng_seed)
        n_ill += int(check_fp32_estimates(got[i, :6][None], om, ose, delta, str(i)).sum())
    assert n_ill <= 2 * 6 * len(pick) // 3          # most cells are well-conditioned


def test_flagged_contracts_of_the_mix_are_ill_conditioned(nv):
    """The contracts of the 1024 mix whose Vega or Theta estimate or SE comes
    out non-finite (the FP32 per-path tangents, or their squares in the tile
    sums, overflow): for the eight with the least work, the FP64 oracle on
    the same normals is finite, but its Vega and Theta move by more than the
    1e-4 bound -- by orders of magnitude -- under FP32-sized perturbations of
    its inputs and normals, so no FP32 path can match it there.  Their other
    estimates are held to the conditioning rule like any other cell."""
    mix, items = _mix_items(nv)
    got = _arr(nv.heston_mc_price_greeks_batch(items, nv.make_options(prec=nv.HESTON_FP32)), nv)
    flagged = np.nonzero((~np.isfinite(got[:, [3, 5, 9, 11]])).any(axis=1))[0]
    assert len(flagged) > 0
    # every flagged contract violates the Feller condition
    for i in flagged:
        p = mix[i]["params"]
        assert 2 * p["kappa"] * p["theta"] < p["xi"] ** 2, i
    work = np.array([mix[i]["n_paths"] * mix[i]["n_steps"] for i in flagged])
    for i in flagged[np.argsort(work)[:8]]:
        it, d = items[i], mix[i]
        om, ose, delta = oracle_with_sensitivity(d["params"], [d["contract"]], it.n_paths,
                                                 it.n_steps, it.rng_seed)
        assert np.isfinite(om[0, [3, 5]]).all(), i
        assert (delta[0, [3, 5]] > 100 * WELL).all(), (i, delta[0])
        check_fp32_estimates(got[i, :6][None], om, ose, delta, str(i))
