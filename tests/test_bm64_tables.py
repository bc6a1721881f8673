"""The constant tables of the FP64 Box-Muller's table-driven logarithm and
sine/cosine (paper_2309_10477_gb300/csrc/bm64_tables.h) equal the values its
generator computes at 60 digits, rounded once to FP64; the ln 2 entry of the
logarithm table is the exact negative of the E = -1 entry, so that the two
cancel exactly near u1 = 1; and the entries are the mathematical values
(checked against mpmath independently of the generator's rounding helper)."""
import importlib.util
import math
import os
import re

import pytest

mpmath = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2309_10477_gb300", "csrc")


def _header_tables():
    text = open(os.path.join(CSRC, "bm64_tables.h")).read()
    out = {}
    for name, body in re.findall(r"const double (\w+)\[\d+\] = \{([^}]*)\};", text):
        out[name] = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-fA-F.]+p[+-]\d+", body)]
    return out


def _generator():
    spec = importlib.util.spec_from_file_location("gen_bm64_tables", os.path.join(CSRC, "gen_bm64_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _within_half_ulp(x: float, exact) -> bool:
    """x is exact rounded to the nearest FP64."""
    return abs(mpmath.mpf(x) - exact) <= mpmath.mpf(math.ulp(x)) / 2


def test_header_is_the_generator_output():
    h = _header_tables()
    t = _generator().tables()
    names = {"kBmLnHi": "ln_hi", "kBmLnLo": "ln_lo", "kBmLnInv": "ln_inv", "kBmELn2Hi": "e_hi",
             "kBmELn2Lo": "e_lo", "kBmSinT": "sin_t", "kBmCosT": "cos_t"}
    assert set(h) == set(names)
    for k, v in names.items():
        assert h[k] == t[v], k
    assert len(h["kBmLnHi"]) == 257 and len(h["kBmELn2Hi"]) == 25 and len(h["kBmSinT"]) == 65


def test_entries_are_the_mathematical_values():
    from mpmath import cos, log, mp, mpf, pi, sin
    mp.dps = 50
    h = _header_tables()
    for j in range(257):
        v = log(1 + mpf(j) / 256)
        # hi + lo carries ln c_j to well below FP64 resolution
        assert abs(mpf(h["kBmLnHi"][j]) + mpf(h["kBmLnLo"][j]) - v) < mpf(2) ** -100
        assert _within_half_ulp(h["kBmLnHi"][j], v)
        assert _within_half_ulp(h["kBmLnInv"][j], 1 / (1 + mpf(j) / 256))
    for i, E in enumerate(range(-24, 1)):
        assert abs(mpf(h["kBmELn2Hi"][i]) + mpf(h["kBmELn2Lo"][i]) - E * log(2)) < mpf(2) ** -95
    assert h["kBmLnHi"][256] == -h["kBmELn2Hi"][23] and h["kBmLnLo"][256] == -h["kBmELn2Lo"][23]
    for t in range(65):
        a = pi / 4 * t / 64
        assert _within_half_ulp(h["kBmSinT"][t], sin(a))
        assert _within_half_ulp(h["kBmCosT"][t], cos(a))
