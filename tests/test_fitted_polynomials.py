"""The two fitted polynomials of the FP32 device code, read from
heston_device.cuh and evaluated here in FP32 steps (with exact log / sqrt),
meet the error bounds the code documents:

* the Box-Muller radius near u1 = 1, r2 = w P(w) for w = 1 - u1 in [0, 0.1]:
  relative error of P below 8.4e-9 against -2 ln(1 - w) / w with exact
  arithmetic, below 1e-7 evaluated in FP32;
* the QMC inverse normal, z = v P(w) with v = 2u - 1, w = -ln(1 - v^2):
  relative error below 3e-7 (central branch) and 2.5e-7 (tail branch)
  against scipy's ndtri over all 2^24 values of u = (k + 1/2) 2^-24, each
  FMA rounded once as on the GPU.
"""
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2309_10477_gb300", "csrc", "heston_device.cuh")


def _source():
    return open(SRC).read()


def _fma32(a, b, c):
    """FP32 fused multiply-add: the exact product-sum rounded once (float64
    holds the product of two floats exactly; the sum is then rounded to
    float32, which for these magnitudes is the single FP32 rounding)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_box_muller_radius_polynomial():
    src = _source()
    c = [np.float32(float(re.search(rf"kBmP{i} = ([-0-9.e]+)f", src).group(1))) for i in range(5)]
    w = np.linspace(0.0, 0.1, 200001)[1:].astype(np.float32)
    p = _fma32(w, np.full_like(w, c[4]), np.full_like(w, c[3]))
    for k in (2, 1, 0):
        p = _fma32(w, p, np.full_like(w, c[k]))
    ref = -2.0 * np.log1p(-w.astype(np.float64)) / w.astype(np.float64)
    # FP32 evaluation adds a few roundings (6.8e-8 at most here) to the 8.4e-9 of the polynomial
    assert np.max(np.abs(p.astype(np.float64) / ref - 1.0)) < 1e-7


def _qmc_coefficients(src):
    body = src[src.index("__device__ __forceinline__ float qmc_normal(uint32_t y)"):]
    body = body[:body.index("\n}\n")]
    central = body[body.index("const float t = add_(w, -3.125f);"):body.index("const float t = add_(sqrt_approx(w), -3.0f);")]
    tail = body[body.index("const float t = add_(sqrt_approx(w), -3.0f);"):]
    num = r"(-?[0-9.]+(?:e-?[0-9]+)?)f"

    def horner_coefs(part):
        first = re.search(rf"fma_\(t, {num}, {num}\)", part)
        rest = re.findall(rf"fma_\(t, p2?, {num}\)", part)
        return [float(first.group(1)), float(first.group(2))] + [float(v) for v in rest]

    return horner_coefs(central), horner_coefs(tail)


def _horner32(t, coefs):
    p = np.full_like(t, np.float32(coefs[0]))
    for a in coefs[1:]:
        p = _fma32(t, p, np.full_like(t, np.float32(a)))
    return p


def test_qmc_inverse_normal_all_24_bit_inputs():
    scipy_special = pytest.importorskip("scipy.special")
    cc, ct = _qmc_coefficients(_source())
    assert len(cc) == 10 and len(ct) == 10
    k = np.arange(1 << 24, dtype=np.int64)
    v = ((2 * k + 1 - (1 << 24)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    one_minus = _fma32(-v, v, np.ones_like(v))
    w = (-np.log(one_minus.astype(np.float64))).astype(np.float32)
    pc = _horner32((w - np.float32(3.125)).astype(np.float32), cc)
    pt = _horner32((np.sqrt(w.astype(np.float64)).astype(np.float32) - np.float32(3.0)).astype(np.float32), ct)
    central = w <= np.float32(6.25)
    z = (v * np.where(central, pc, pt)).astype(np.float32)
    ref = scipy_special.ndtri((k + 0.5) * 2.0 ** -24)
    err = np.abs(z.astype(np.float64) - ref) / np.abs(ref)
    # measured: 2.83e-7 (central branch) and 2.08e-7 (tail, 16202 inputs), FP32 rounding included
    assert err[central].max() < 3e-7
    assert err[~central].max() < 2.5e-7
