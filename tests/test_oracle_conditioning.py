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
    normals."""
import numpy as np

import oracle
from conditioning import (BOUND, WELL, oracle_paths_with_sensitivity, oracle_with_sensitivity)
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
