"""Write fv_fp64_tables.h: the tables of the kernels' own FP64 erfcx, log and exp.

On this GPU an FP64 operation costs as much issue time as ~70 FP32 ones, and
the solvers of Section 2.2 spend most of their FP64 work in two functions: the
scaled complementary error function erfcx(z) = exp(z^2) erfc(z) (the
normalised Black function is a difference of two erfcx values) and the
logarithm (the lowest- and highest-region objectives work with ln b), and
every evaluation takes one exponential.  The kernels evaluate all three from
small tables instead of general library routines.

erfcx on 0 <= z < 128: Chebyshev interpolation (Trefethen, Approximation
Theory and Approximation Practice, ch. 4) on short pieces, the piecewise
scheme of S. G. Johnson's Faddeeva package, with pieces laid out so that the
piece index comes from the bits of z:

  piece k = 0..7:     [k/16, (k+1)/16)                  (uniform below 1/2)
  piece 8 + 16e' + j: [2^e (1 + j/16), 2^e (1 + (j+1)/16)),  e = e' - 1 = -1..6

Each piece stores its centre c and the degree-8 polynomial in v = z - c that
interpolates erfcx at the 9 Chebyshev points of the piece.  v is exact where
z and c lie within a factor of two of each other (Sterbenz), which is every
piece but the first below z = 1/64; there its rounding error is below 2^-59.
Beyond z = 128 the kernels use the asymptotic series (Abramowitz & Stegun
7.1.23) instead.

log: the table-driven method of P. T. P. Tang (ACM TOMS 16(4), 1990).  With
y = 2^m f, f in [1/sqrt2, sqrt2), and F_j = 1 + j/256 the grid point nearest
f (j = -75..106), the kernels form r = f c_j - 1 with one fused multiply-add,
c_j = 1/F_j rounded to FP64, and return
    (m ln2_hi + L_hi[j]) + (m ln2_lo + L_lo[j] + log1p(r)),
where L_j = -ln(c_j) for the rounded c_j (so the rounding of c_j costs
nothing), split so that m ln2_hi + L_hi[j] is exact (both on a 2^-42 grid),
and log1p(r), |r| <= 0.0028, is its Taylor polynomial to r^6.  c_0 = 1, so
next to y = 1 the result is log1p(y - 1) with y - 1 exact.

exp: the table-driven method of P. T. P. Tang (ACM TOMS 15(2), 1989).  With
k = round(v 128/ln2), r = v - k ln2/128 (ln2/128 split into a 35-bit head, so
k ln2_128_hi is exact, and a tail) and j = k mod 128, m = floor(k/128):
    exp(v) = 2^m (T_hi[j] + (T_hi[j] expm1(r) + T_lo[j])),
T_hi + T_lo = 2^(j/128) to 2^-106 and expm1(r), |r| <= ln2/256, its Taylor
polynomial to r^5.

Run:  python gen_fp64_tables.py [samples per piece]
(needs mpmath; prints the worst error of the FP64 erfcx Horner evaluation,
emulated with exactly rounded fused multiply-adds, against mpmath on a dense
sample of every piece).
"""
import os
import sys

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "fv_fp64_tables.h")

DEGREE = 8
STRIDE = 10         # doubles per erfcx piece: centre + 9 coefficients (80 bytes, five 16-byte loads)
UNIFORM = 8         # pieces of width 1/16 on [0, 1/2)
SUB = 16            # pieces per binade on [1/2, 128)
BINADES = range(-1, 7)
Z_TABLE_END = 128.0

LOG_J = range(-75, 107)  # F_j = 1 + j/256 covers [1/sqrt2, sqrt2)
EXP_N = 128
LOG_GRID = 2.0 ** -42    # m ln2_hi and L_hi are multiples of this

mp.mp.dps = 50


def erfcx(z):
    return mp.exp(z * z) * mp.erfc(z)


def pieces():
    out = [(mp.mpf(k) / (2 * UNIFORM), mp.mpf(k + 1) / (2 * UNIFORM)) for k in range(UNIFORM)]
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


def on_grid(v):
    """Round v to the nearest multiple of LOG_GRID (exact in FP64)."""
    return float(mp.nint(mp.mpf(v) / LOG_GRID) * LOG_GRID)


def log_table():
    ln2 = mp.log(2)
    ln2_hi = on_grid(ln2)
    ln2_lo = float(ln2 - ln2_hi)
    rows = []
    for j in LOG_J:
        c = 1.0 if j == 0 else float(1 / (1 + mp.mpf(j) / 256))
        L = -mp.log(mp.mpf(c))
        L_hi = on_grid(L)
        rows.append((c, L_hi, float(L - L_hi)))
    return ln2_hi, ln2_lo, rows


def exp_table():
    ln2_64 = mp.log(2) / EXP_N
    e = int(mp.floor(mp.log(ln2_64, 2)))
    q = mp.mpf(2) ** (e - 34)               # 35 significant bits
    hi = float(mp.nint(ln2_64 / q) * q)
    lo = float(ln2_64 - hi)
    rows = []
    for j in range(EXP_N):
        t = mp.mpf(2) ** (mp.mpf(j) / EXP_N)
        t_hi = float(t)
        rows.append((t_hi, float(t - t_hi)))
    return float(EXP_N / mp.log(2)), hi, lo, rows


def write(table, out=OUT):
    ln2_hi, ln2_lo, lrows = log_table()
    inv, e_hi, e_lo, erows = exp_table()
    lines = [
        "// Generated by gen_fp64_tables.py (beside this file); do not edit.",
        "#pragma once",
        "",
        "// erfcx: piecewise Chebyshev interpolants on 0 <= z < %g; piece k holds its" % Z_TABLE_END,
        "// centre c_k and the degree-%d polynomial in v = z - c_k (lowest order first)," % DEGREE,
        "// %d doubles (%d bytes) per piece." % (STRIDE, STRIDE * 8),
        "#define FV_ERFCX_PIECES %d" % len(table),
        "#define FV_ERFCX_DEGREE %d" % DEGREE,
        "#define FV_ERFCX_STRIDE %d" % STRIDE,
        "#define FV_ERFCX_TABLE_END %.1f" % Z_TABLE_END,
        "static __device__ __align__(128) const double kErfcxTable[FV_ERFCX_PIECES * FV_ERFCX_STRIDE] = {",
    ]
    for c, coefs in table:
        row = [c] + coefs + [0.0] * (STRIDE - 1 - len(coefs))
        lines.append("    " + ", ".join(repr(x) for x in row) + ",")
    lines += [
        "};",
        "",
        "// log: row j + %d holds c_j = 1/(1 + j/256) (rounded; c_0 = 1), L_hi[j] and" % -LOG_J[0],
        "// L_lo[j] with L_hi + L_lo = -ln(c_j), L_hi and ln2_hi on a 2^-42 grid, and a pad.",
        "#define FV_LOG_J0 %d" % LOG_J[0],
        "#define FV_LOG_ROWS %d" % len(lrows),
        "#define FV_LN2_HI %r" % ln2_hi,
        "#define FV_LN2_LO %r" % ln2_lo,
        "static __device__ __align__(32) const double kLogTable[FV_LOG_ROWS * 4] = {",
    ]
    for c, hi, lo in lrows:
        lines.append("    %r, %r, %r, 0.0," % (c, hi, lo))
    lines += [
        "};",
        "",
        "// exp: row j holds T_hi[j], T_lo[j] with T_hi + T_lo = 2^(j/128); ln2/128 = LN2_N_HI +",
        "// LN2_N_LO with a 35-bit head.",
        "#define FV_EXP_N %d" % EXP_N,
        "#define FV_EXP_INV_LN2_N %r" % inv,
        "#define FV_EXP_LN2_N_HI %r" % e_hi,
        "#define FV_EXP_LN2_N_LO %r" % e_lo,
        "static __device__ __align__(16) const double kExpTable[%d * 2] = {" % EXP_N,
    ]
    for hi, lo in erows:
        lines.append("    %r, %r," % (hi, lo))
    lines.append("};")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


def main(out=OUT, samples=64):
    table = [fit(a, b) for a, b in pieces()]
    write(table, out)
    err, z = worst_error(table, samples)
    print("%s: %d erfcx pieces, worst relative error %.3e (%.2f ulp of 2^-52) at z = %r"
          % (out, len(table), err, err / 2.0 ** -52, z))
    return err


if __name__ == "__main__":
    main(samples=int(sys.argv[1]) if len(sys.argv) > 1 else 64)
