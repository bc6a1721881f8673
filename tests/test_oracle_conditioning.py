"""The oracle's sensitivity probe (oracle.mc_price_greeks_perturbed and
tests/conditioning.py), on the CPU:
  * with zero perturbation it is the oracle itself, bit for bit;
  * perturbations move the estimates in proportion to their size on a
    well-conditioned set (the base parameters, Feller satisfied);
  * the pathwise Vega and Theta of a set far from the Feller condition with
    many steps move by orders of magnitude more than the 1e-4 bound under
    FP32-sized perturbations, and far more than the price and Delta (which
    on such a set move by more than the bound too);
  * the per-path probe returns the oracle's own records on unperturbed
    normals;
  * the Brownian bridge run in time order (each W interpolated from W_k and
    the stack top W_r, the form a GPU lane uses) is the oracle's breadth-first
    bridge, and run in FP32 it stays within the per-path bound the QMC parity
    test perturbs the normals by."""
import numpy as np

import oracle
from conditioning import (BOUND, FP32_NORMAL_REL, WELL, oracle_paths_with_sensitivity, oracle_with_sensitivity,
                          qmc_normal_bound)
from oracle import sobol
from paper_2309_10477_gb300 import workloads as wl

BASE = wl.BASE_PARAMS
CS = [(0, 100.0, 1.0, 0, 0), (1, 100.0, 1.0, 0, 0)]


def test_zero_perturbation_is_the_oracle():
    P = oracle.Params(**BASE)
    cs = [oracle.Contract(*c) for c in CS]
    a = oracle.mc_price_greeks(P, cs, 3000, 40, 9)
    b = oracle.mc_price_greeks_perturbed(P, cs, 3000, 40, 9, 0.0, 0.0, 123)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_change_scales_with_the_perturbation():
    P = oracle.Params(**BASE)
    cs = [oracle.Contract(*c) for c in CS]
    a, _ = oracle.mc_price_greeks(P, cs, 4096, 40, 9)
    d = []
    for eps in (1e-9, 1e-8, 1e-7):
        b, _ = oracle.mc_price_greeks_perturbed(P, cs, 4096, 40, 9, 0.0, eps, 1)
        d.append(np.abs(b - a).max())
    assert d[0] > 0
    assert 3 < d[1] / d[0] < 30 and 3 < d[2] / d[1] < 30     # about linear in eps


def test_base_set_well_conditioned():
    om, ose, delta = oracle_with_sensitivity(BASE, CS, 1 << 13, 100, 3)
    assert (delta <= WELL).all(), delta
    assert (delta < 1e-5).all()


def test_far_from_feller_tangents_ill_conditioned():
    params = dict(S0=100.0, v0=0.05, kappa=5.0, theta=0.01, xi=0.9, rho=-0.7, r=0.03)
    om, ose, delta = oracle_with_sensitivity(params, [(0, 100.0, 1.0, 0, 0)], 1 << 14, 400, 1)
    assert np.isfinite(om).all()
    assert (delta[0, [3, 5]] > 100 * BOUND).all(), delta      # Vega, Theta
    assert delta[0, [3, 5]].min() > 1e4 * delta[0, [0, 1]].max(), delta


def test_per_path_probe_returns_the_oracle_records():
    paths = np.arange(40, dtype=np.uint64)
    rec, est, drec, dest = oracle_paths_with_sensitivity(BASE, CS, paths, 30, 5)
    rec_d, est_d = oracle.debug_paths(oracle.Params(**BASE), [oracle.Contract(*c) for c in CS],
                                      paths, 30, 5)
    assert np.array_equal(rec, rec_d) and np.array_equal(est, est_d)
    assert (drec[:, :14] > 0).any() and np.isfinite(drec).all()
    assert (drec[:, 0] < 1e-5 * np.maximum(1.0, np.abs(rec[:, 0]))).all()


def _time_ordered_bridge(z, N, dtype, rel_noise=0.0, seed=0):
    """Step normals (n, N) of the bridge on node normals z (n, N), built in
    time order with a stack of right ends: entering step k with W_k known, push
    W_m = W_k + (m-k)/(r-k) (W_r - W_k) + sqrt((m-k)(r-m)/(r-k)) z_m for the
    midpoints m of [k, r] down to [k, k+1], pop W_{k+1}.  In FP32 each
    multiply-add is rounded once (an FMA: exact product, one rounding) and the
    node normals carry a relative error up to rel_noise (the inverse normal's)."""
    plan = sobol.BridgePlan(N)
    node = {m: j for j, (m, l, r) in enumerate(plan.nodes)}
    rng = np.random.default_rng(seed)
    zz = z * (1.0 + rel_noise * rng.uniform(-1, 1, z.shape))
    zz = zz.astype(dtype)

    def fma(a, b, c):
        return (np.float64(a) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(dtype)

    n = z.shape[0]
    Wk = np.zeros(n, dtype)
    stack, right = [], []
    out = np.zeros((n, N), dtype)
    for k in range(N):
        if k == 0:
            stack.append(fma(dtype(np.sqrt(N)), zz[:, 0], np.zeros(n, dtype)))
            right.append(N)
        while right[-1] - k >= 2:
            r = right[-1]
            m = k + (r - k) // 2
            assert plan.nodes[node[m]][1:] == (k, r)      # the node's interval starts at k
            d = fma(-1.0, Wk, stack[-1])
            stack.append(fma(dtype(np.sqrt((m - k) * (r - m) / (r - k))), zz[:, node[m]],
                             fma(dtype((m - k) / (r - k)), d, Wk)))
            right.append(m)
        w = stack.pop()
        right.pop()
        out[:, k] = fma(-1.0, Wk, w)
        Wk = w
    return out.astype(np.float64)


def test_time_ordered_bridge_is_the_bisection_bridge_and_fp32_stays_in_bound():
    for N in (1, 7, 64, 252, 1024):
        V = sobol.direction_numbers(2 * N)
        y = sobol.points(V, np.arange(512)) ^ sobol.shifts(42, 1, V.shape[0])[None, :]
        z = sobol.ndtri(sobol.uniforms(y))[:, 0:2 * N:2]
        ref = sobol.BridgePlan(N).step_normals(z)
        np.testing.assert_allclose(_time_ordered_bridge(z, N, np.float64), ref, rtol=0, atol=1e-12)
        # FP32, with the node normals off by up to 2e-7 relative (the inverse
        # normal's fit and the lg2 approximation)
        err = np.abs(_time_ordered_bridge(z, N, np.float32, 2e-7, N) - ref)
        lim = qmc_normal_bound(ref, ref) + FP32_NORMAL_REL * np.abs(ref)
        assert (err <= lim).all(), (N, (err / lim).max())
        # the Box-Muller-sized bound alone does not cover the bridge at many steps
        if N >= 64:
            assert (err > 1e-7 + FP32_NORMAL_REL * np.abs(ref)).any()
