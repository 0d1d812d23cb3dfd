"""Write fv_erfcx_table.h: piecewise polynomial coefficients of the scaled
complementary error function erfcx(z) = exp(z^2) erfc(z) on 0 <= z < 128.

The normalised Black function of Section 2.2 is evaluated as a difference of
two erfcx values, so erfcx is the most frequent FP64 special function of the
solvers.  On this GPU an FP64 operation costs as much issue time as ~70 FP32
ones, so the kernels evaluate erfcx from a small table instead of a general
library routine: Chebyshev interpolation (Trefethen, Approximation Theory and
Approximation Practice, ch. 4) of erfcx on short pieces, the piecewise scheme
used by S. G. Johnson's Faddeeva package, with the pieces laid out so that the
piece index comes from the bits of z:

  piece k = 0..3:    [k/8, (k+1)/8)                (uniform below 1/2)
  piece 4 + 8e' + j: [2^e (1 + j/8), 2^e (1 + (j+1)/8)),  e = e' - 1 = -1..6

Each piece stores its centre c and the degree-10 polynomial in v = z - c that
interpolates erfcx at the 11 Chebyshev points of the piece.  v is exact where
z and c lie within a factor of two of each other (Sterbenz), which is every
piece but the first below z = 1/32; there its rounding error is below 2^-58.
Beyond z = 128 the kernels use the asymptotic series (Abramowitz & Stegun
7.1.23) instead.

Run:  python gen_erfcx_table.py [samples per piece]
(needs mpmath; prints the worst error of the FP64 Horner evaluation, emulated
with exactly rounded fused multiply-adds, against mpmath on a dense sample of
every piece).
"""
import os
import sys

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "fv_erfcx_table.h")

DEGREE = 10
STRIDE = 16         # doubles per piece: centre + 11 coefficients + padding (128 bytes)
UNIFORM = 4         # pieces of width 1/8 on [0, 1/2)
SUB = 8             # pieces per binade on [1/2, 128)
BINADES = range(-1, 7)
Z_TABLE_END = 128.0

mp.mp.dps = 50


def erfcx(z):
    return mp.exp(z * z) * mp.erfc(z)


def pieces():
    out = [(mp.mpf(k) / 8, mp.mpf(k + 1) / 8) for k in range(UNIFORM)]
    for e in BINADES:
        for j in range(SUB):
            a = mp.mpf(2) ** e * (1 + mp.mpf(j) / SUB)
            b = mp.mpf(2) ** e * (1 + mp.mpf(j + 1) / SUB)
            out.append((a, b))
    return out


def fit(a, b):
    """Monomial coefficients in v = z - c of the Chebyshev interpolant."""
    c = (a + b) / 2
    half = (b - a) / 2
    n = DEGREE + 1
    nodes = [half * mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n)]
    A = mp.matrix([[v ** j for j in range(n)] for v in nodes])
    y = mp.matrix([erfcx(c + v) for v in nodes])
    coef = mp.lu_solve(A, y)
    return float(c), [float(coef[j]) for j in range(n)]


def fma(x, y, z):
    """FP64 fused multiply-add, exactly rounded (what the GPU's DFMA does)."""
    return float(mp.mpf(x) * mp.mpf(y) + mp.mpf(z))


def horner(coefs, v):
    p = coefs[-1]
    for cj in reversed(coefs[:-1]):
        p = fma(p, v, cj)
    return p


def worst_error(table, samples=64):
    worst = (0.0, None)
    for (a, b), (c, coefs) in zip(pieces(), table):
        for i in range(samples + 1):
            z = float(a + (b - a) * i / samples)
            if z >= float(b):
                z = float(b) - float(b) * 2.0 ** -52
            v = z - c
            got = horner(coefs, v)
            ref = erfcx(mp.mpf(z))
            err = abs(float((got - ref) / ref))
            if err > worst[0]:
                worst = (err, z)
    return worst


def write(table, out=OUT):
    lines = [
        "// Generated by gen_erfcx_table.py (beside this file); do not edit.",
        "// Piecewise Chebyshev interpolants of erfcx(z) on 0 <= z < %g: piece k holds" % Z_TABLE_END,
        "// its centre c_k and the degree-%d polynomial in v = z - c_k (lowest order" % DEGREE,
        "// first), padded to %d doubles (%d bytes) per piece." % (STRIDE, STRIDE * 8),
        "#pragma once",
        "#define FV_ERFCX_PIECES %d" % len(table),
        "#define FV_ERFCX_STRIDE %d" % STRIDE,
        "#define FV_ERFCX_TABLE_END %.1f" % Z_TABLE_END,
        "static __device__ __align__(128) const double kErfcxTable[FV_ERFCX_PIECES * FV_ERFCX_STRIDE] = {",
    ]
    for c, coefs in table:
        row = [c] + coefs + [0.0] * (STRIDE - 1 - len(coefs))
        lines.append("    " + ", ".join(repr(x) for x in row) + ",")
    lines.append("};")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


def main(out=OUT, samples=64):
    table = [fit(a, b) for a, b in pieces()]
    write(table, out)
    err, z = worst_error(table, samples)
    print("%s: %d pieces, worst relative error %.3e (%.2f ulp of 2^-52) at z = %r"
          % (out, len(table), err, err / 2.0 ** -52, z))
    return err


if __name__ == "__main__":
    main(samples=int(sys.argv[1]) if len(sys.argv) > 1 else 64)
