"""Exact rounding of rationals to a float format, for tests that rebuild the
GPU's FP32 / FP64 sums operation by operation on the host."""
from fractions import Fraction


def round_exact(q, bits):
    """Round the exact rational q to the nearest float with `bits` significant
    bits (ties to even): the rounding of one IEEE add, multiply or fma.
    Normal range only (no subnormals or overflow)."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(Fraction(q))
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    scaled = q / Fraction(2) ** (e - bits + 1)          # in [2^(bits-1), 2^bits)
    m, r = divmod(scaled.numerator, scaled.denominator)
    if 2 * r > scaled.denominator or (2 * r == scaled.denominator and m % 2 == 1):
        m += 1
    return sign * float(Fraction(m) * Fraction(2) ** (e - bits + 1))
