"""Write bm64_tables.h: the constant tables of the FP64 Box-Muller's
table-driven logarithm and sine/cosine (heston_device.cuh, bm_ln_u1 and
bm_sincos_2pi), from 60-digit mpmath values rounded once to FP64.

* ln(c_j), c_j = 1 + j/256, j = 0..256, as a pair hi + lo (hi = RN(ln c_j),
  lo = RN(ln c_j - hi)), and 1/c_j rounded to FP64.  The entry j = 256
  (c = 2) is the exact negative of the E = -1 entry below, so that
  -ln 2 + ln 2 cancels exactly when u1 is close to 1.
* E ln 2 for E = -24..0 as pairs hi + lo.
* sin and cos of theta_t = (pi/4) t/64, t = 0..64, rounded to FP64.

The reduction is the table-driven method of P. T. P. Tang, "Table-driven
implementation of the logarithm function in IEEE floating-point arithmetic"
(ACM TOMS 16(4), 1990), and the same split theta = theta_t + beta for sine
and cosine.  Run:

    python paper_2309_10477_gb300/csrc/gen_bm64_tables.py
"""
import os

from mpmath import cos, log, mp, mpf, pi, sin

mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "bm64_tables.h")


def rn(x) -> float:
    """Round an mpmath value to the nearest FP64 (ties to even): rounded to
    53 bits at the working precision's nearest rounding, then converted
    exactly."""
    with mp.workprec(53):
        y = +mpf(x)
    return float(y)


def pair(x):
    hi = rn(x)
    lo = rn(x - mpf(hi))
    return hi, lo


def tables():
    ln_hi, ln_lo, inv = [], [], []
    for j in range(257):
        c = 1 + mpf(j) / 256
        h, l = pair(log(c))
        ln_hi.append(h)
        ln_lo.append(l)
        inv.append(rn(1 / c))
    e_hi, e_lo = [], []
    for E in range(-24, 1):
        h, l = pair(E * log(2))
        e_hi.append(h)
        e_lo.append(l)
    # j = 256 is ln 2: make it the exact negative of E = -1 (both are RN of the same value)
    assert (ln_hi[256], ln_lo[256]) == (-e_hi[23], -e_lo[23])
    sin_t = [rn(sin(pi / 4 * t / 64)) for t in range(65)]
    cos_t = [rn(cos(pi / 4 * t / 64)) for t in range(65)]
    return dict(ln_hi=ln_hi, ln_lo=ln_lo, ln_inv=inv, e_hi=e_hi, e_lo=e_lo, sin_t=sin_t, cos_t=cos_t)


def emit(name, values, comment):
    lines = [f"// {comment}", f"__device__ const double {name}[{len(values)}] = {{"]
    for i in range(0, len(values), 3):
        lines.append("    " + " ".join(f"{v.hex()}," for v in values[i:i + 3]))
    lines.append("};")
    return "\n".join(lines)


def main():
    t = tables()
    parts = [
        "// Generated by gen_bm64_tables.py: do not edit.  Constant tables of the FP64",
        "// Box-Muller's table-driven logarithm and sine/cosine (60-digit values rounded",
        "// once to FP64; hexadecimal floating-point literals).",
        "#pragma once",
        "",
        emit("kBmLnHi", t["ln_hi"], "ln(1 + j/256), high part, j = 0..256"),
        emit("kBmLnLo", t["ln_lo"], "ln(1 + j/256) - kBmLnHi[j], rounded"),
        emit("kBmLnInv", t["ln_inv"], "1 / (1 + j/256), rounded"),
        emit("kBmELn2Hi", t["e_hi"], "E ln 2, high part, E = -24..0 (index E + 24)"),
        emit("kBmELn2Lo", t["e_lo"], "E ln 2 - kBmELn2Hi, rounded"),
        emit("kBmSinT", t["sin_t"], "sin((pi/4) t/64), t = 0..64"),
        emit("kBmCosT", t["cos_t"], "cos((pi/4) t/64), t = 0..64"),
        "",
    ]
    with open(OUT, "w") as f:
        f.write("\n".join(parts))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
