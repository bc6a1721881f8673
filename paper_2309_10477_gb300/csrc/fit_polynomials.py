"""Fit the two polynomials the FP32 device code evaluates, and print their
coefficients (rounded to FP32, as written in heston_device.cuh) with their
maximum relative error on a dense grid.

* Box-Muller radius near u1 = 1: P(w) ~ -2 ln(1 - w) / w on [0, 0.1], so
  that r2 = -2 ln u1 = w P(w) in the exact w = 1 - u1.  Degree 4.
* Inverse normal of the QMC kernel: Phi^-1(u) = sqrt(2) erfinv(v) with
  v = 2u - 1, written as v P(w), w = -ln(1 - v^2) -- the two-branch
  structure of M. Giles, "Approximating the erfinv function" (GPU Computing
  Gems Jade, 2011).  P is a degree-9 polynomial in w - 3.125 for
  w <= 6.25 and a degree-9 polynomial in sqrt(w) - 3 above, up to the
  largest w of a 24-bit uniform, -ln(2^-23 - 2^-48).

Each polynomial minimises the maximum relative error: weighted least
squares on Chebyshev nodes, reweighted by the error (Lawson's iteration).
The references are mpmath evaluations at 40 digits.  Run:

    python paper_2309_10477_gb300/csrc/fit_polynomials.py
"""
import numpy as np
from mpmath import erfinv, exp, log, mp, mpf, sqrt

mp.dps = 40


def lawson_fit(f, a, b, deg, var, n=3000, iters=300):
    x = (a + b) / 2 + (b - a) / 2 * np.cos(np.pi * (np.arange(n) + 0.5) / n)
    y = np.array([f(v) for v in x])
    V = np.vander(var(x), deg + 1, increasing=True)
    W = np.ones(n)
    for _ in range(iters):
        A = V / y[:, None] * np.sqrt(W)[:, None]
        c, *_ = np.linalg.lstsq(A, np.sqrt(W), rcond=None)
        err = np.abs(V @ c / y - 1)
        W = W * err
        W /= W.sum()
    return np.float32(c)


def max_rel_err(c32, f, a, b, var, n=20001):
    x = np.linspace(a, b, n)
    y = np.array([f(v) for v in x])
    p = np.polyval(c32.astype(np.float64)[::-1], var(x))
    return float(np.max(np.abs(p / y - 1)))


def radius_ratio(w):
    w = mpf(w)
    return 2.0 if w == 0 else float(-2 * log(1 - w) / w)


def invnorm_ratio(w):
    w = mpf(w)
    if w == 0:
        return float(sqrt(mp.pi / 2))
    v = sqrt(1 - exp(-w))
    return float(sqrt(2) * erfinv(v) / v)


def main():
    c = lawson_fit(radius_ratio, 0.0, 0.1, 4, lambda x: x)
    print("Box-Muller radius, P(w), w in [0, 0.1]:", [repr(float(v)) for v in c],
          "max rel err %.2e" % max_rel_err(c, radius_ratio, 0.0, 0.1, lambda x: x, 4001))
    wc = 6.25
    wmax = float(-log(2 * mpf(2) ** -24 - mpf(2) ** -48))
    cc = lawson_fit(invnorm_ratio, 0.0, wc, 9, lambda x: x - wc / 2)
    ct = lawson_fit(invnorm_ratio, wc, wmax, 9, lambda x: np.sqrt(x) - 3.0)
    print("inverse normal, central P(w - 3.125):", [repr(float(v)) for v in cc],
          "max rel err %.2e" % max_rel_err(cc, invnorm_ratio, 0.0, wc, lambda x: x - wc / 2, 2001))
    print("inverse normal, tail P(sqrt(w) - 3):", [repr(float(v)) for v in ct],
          "max rel err %.2e" % max_rel_err(ct, invnorm_ratio, wc, wmax, lambda x: np.sqrt(x) - 3.0, 2001))


if __name__ == "__main__":
    main()
