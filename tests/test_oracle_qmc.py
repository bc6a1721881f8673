"""Pins for the oracle's quasi-Monte Carlo normals (Sec. 2.7 Sobol
sequences; Brownian bridge), and the library's host-built direction table
checked against the oracle's independent construction."""
import math

import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from oracle import Contract, Params
from oracle import closed_form as cf
from oracle import sobol


def _euler_phi(n):
    out, m, p = n, n, 2
    while p * p <= m:
        if m % p == 0:
            out -= out // p
            while m % p == 0:
                m //= p
        p += 1
    if m > 1:
        out -= out // m
    return out


def test_primitive_polynomial_counts_match_number_theory():
    # the number of primitive polynomials of degree s over GF(2) is phi(2^s - 1) / s
    polys = sobol.primitive_polynomials(1000)
    degs = [p.bit_length() - 1 for p in polys]
    for s in range(1, max(degs)):
        assert degs.count(s) == _euler_phi(2**s - 1) // s, s
    # ordered by degree, then value; each one irreducible (no factor of degree <= s/2)
    assert polys == sorted(polys)
    for p in polys[:60]:
        s = p.bit_length() - 1
        for q in range(2, 1 << (s // 2 + 1)):
            if q.bit_length() - 1 >= 1:
                # polynomial remainder of p by q over GF(2)
                r = p
                while r.bit_length() >= q.bit_length():
                    r ^= q << (r.bit_length() - q.bit_length())
                assert r != 0, (p, q)


@pytest.fixture(scope="module")
def V():
    return sobol.direction_numbers(504)


def test_every_dimension_is_stratified(V):
    # each aligned block of 2^m points puts one point in each dyadic interval of length 2^-m
    x = sobol.points(V, np.arange(1 << 10))
    y = x ^ sobol.shifts(42, 3, V.shape[0])[None, :]
    for arr in (x, y):
        for m in (1, 4, 10):
            cells = (arr >> np.uint32(32 - m)).astype(np.int64)
            for blk in range(0, 1 << 10, 1 << m):
                c = cells[blk:blk + (1 << m)]
                assert (np.sort(c, axis=0) == np.arange(1 << m)[:, None]).all(), m


@pytest.mark.parametrize("d", [2, 5, 9, 13])
def test_property_a(V, d):
    # 2^d points, one in each of the 2^d subcubes of the half-split unit cube
    pts = sobol.points(V, np.arange(1 << d))[:, :d]
    code = np.zeros(len(pts), dtype=np.int64)
    for i in range(d):
        code |= (pts[:, i] >> np.uint32(31)).astype(np.int64) << i
    assert len(np.unique(code)) == 1 << d


def test_property_a_leading_minors_up_to_32(V):
    # first-digit matrix of dims 0..31 over index bits 1..32 is non-singular
    rows = [sum(((int(V[j, k]) >> 31) & 1) << k for k in range(32)) for j in range(32)]
    basis = {}
    for r in rows:
        for bit in range(32):
            if r >> bit & 1:
                if bit in basis:
                    r ^= basis[bit]
                else:
                    basis[bit] = r
                    break
        else:
            pytest.fail("dependent row")


def test_first_dimension_is_van_der_corput(V):
    n = np.arange(1 << 12)
    x = sobol.points(V, n)[:, 0]
    rev = np.array([int(format(int(i), "032b")[::-1], 2) for i in n], dtype=np.uint32)
    assert np.array_equal(x, rev)


@pytest.mark.parametrize("N", [1, 2, 7, 64, 252])
def test_brownian_bridge_covariance_is_min(N):
    plan = sobol.BridgePlan(N)
    L = plan.build(np.eye(N))                  # column j: W on the grid for z = e_j
    cov = L.T @ L                               # (N+1) x (N+1)
    t = np.arange(N + 1)
    np.testing.assert_allclose(cov, np.minimum.outer(t, t), atol=1e-12)
    # step normals are an orthonormal image of z
    dW = np.diff(L, axis=1)
    np.testing.assert_allclose(dW.T @ dW, np.eye(N), atol=1e-12)


def test_uniforms_and_inverse_normal(V):
    y = np.array([0, 255, 256, 2**31, 2**32 - 1], dtype=np.uint32)
    u = sobol.uniforms(y)
    assert (u > 0).all() and (u < 1).all()
    assert u[0] == 0.5 * 2**-24 and u[-1] == 1 - 0.5 * 2**-24
    from scipy.special import ndtri
    np.testing.assert_allclose(ndtr(ndtri(u)), u, rtol=1e-12)


def test_qmc_estimates_agree_with_closed_form_and_beat_mc():
    p = Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)
    cs = [Contract(0, 100.0, 1.0)]
    N, R, P = 32, 16, 1 << 12
    m, se, _ = sobol.qmc_price_greeks(p, cs, R, P, N, 42)
    ref = cf.heston_price_greeks(100.0, 100.0, 1.0, 0.05, 0.04, 2.0, 0.04, 0.3, -0.7)
    # Milstein bias at N = 32 is well below the slack
    for j, k in enumerate(oracle.ESTIMATORS):
        assert abs(m[0, j] - ref[k]) < 4 * se[0, j] + 0.01 * max(1.0, abs(ref[k])), k
    mm, mse = oracle.mc_price_greeks(p, cs, R * P, N, 42)
    assert se[0, 0] < 0.5 * mse[0, 0]        # the bridge-QMC price is far less noisy


def test_replicate_se_matches_the_spread_of_independent_estimates():
    """The randomised-QMC SE (Sec. 2.7's randomisation): each seed draws
    independent digital shifts, so the estimates of different seeds scatter
    by the SE each one reports -- the spread of 60 estimates over the RMS of
    their SEs is 1 up to sampling noise (about 9 % for 60 seeds), for all six
    estimators."""
    p = Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)
    cs = [Contract(0, 100.0, 1.0)]
    means, ses = [], []
    for seed in range(1, 61):
        m, se, _ = sobol.qmc_price_greeks(p, cs, 8, 256, 8, seed)
        means.append(m[0])
        ses.append(se[0])
    means, ses = np.array(means), np.array(ses)
    ratio = means.std(axis=0, ddof=1) / np.sqrt((ses ** 2).mean(axis=0))
    assert ((ratio > 0.7) & (ratio < 1.4)).all(), ratio


def test_library_direction_table_matches_oracle():
    from paper_2309_10477_gb300 import build, native
    build.build()
    for D in (1, 2, 31, 33, 504, 1000):
        assert np.array_equal(native.heston_sobol_directions(D), sobol.direction_numbers(D)), D
