"""The exact-rounding helper the GPU tests use to rebuild the kernels' sums
agrees with numpy's IEEE float32 / float64 arithmetic."""
from fractions import Fraction

import numpy as np

from exact_rounding import round_exact


def test_round_exact_matches_ieee_add_and_multiply():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        a = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-3, 4))
        b = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-3, 4))
        assert round_exact(Fraction(float(a)) + Fraction(float(b)), 24) == float(a + b)
        assert round_exact(Fraction(float(a)) * Fraction(float(b)), 24) == float(a * b)
        x, y = rng.standard_normal(2) * 10.0 ** rng.integers(-3, 4, 2)
        assert round_exact(Fraction(x) + Fraction(y), 53) == x + y
        assert round_exact(Fraction(x) * Fraction(y), 53) == x * y


def test_round_exact_ties_to_even():
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 23)
    assert round_exact(one + ulp / 2, 24) == 1.0                 # tie, even mantissa below
    assert round_exact(one + ulp + ulp / 2, 24) == float(one + 2 * ulp)   # tie, odd below: up
    assert round_exact(-(one + ulp / 2), 24) == -1.0
