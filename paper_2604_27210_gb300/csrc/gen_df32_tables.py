"""Write fv_df32_tables.h: the tables of the kernels' double-float (df32) erfcx, exp and log.

A double-float number is an unevaluated sum hi + lo of two FP32 numbers with
|lo| <= ulp(hi)/2: 48 significant bits from FP32 arithmetic (T. J. Dekker, "A
floating-point technique for extending the available precision", Numer. Math.
18, 1971).  On this GPU an FP64 instruction holds its pipe ~64 times as long
as an FP32 one issues, so the mixed solver's one Householder(3) correction
(Section 2.2: the FP64 step after the FP32 iterations) evaluates its
normalised Black residual in double-float instead of FP64 wherever the quote's
scales fit FP32's exponent range.

erfcx on 0 <= z < 128: the pieces of the FP64 table (gen_fp64_tables.py:
8 uniform pieces of width 1/16 below 1/2, 16 per binade above), each with its
centre c (exact in FP32: a dyadic rational with few bits) and the degree-8
Chebyshev interpolant in v = z - c.  |v| <= z/32 (and <= 1/32 below 1/2), so
the term of degree k is below 2^-5k of the value relative to the leading one:
the coefficients of degree 0..4 are stored as double-float pairs, those of
degree 5..8 as FP32 (their rounding is below 2^-49 of the value).

exp: Tang's table-driven reduction (ACM TOMS 15(2), 1989) as in the FP64
table, k = round(v 128/ln2), r = v - k ln2/128 with ln2/128 split into four
FP32 parts of 10, 10, 24 and 24 significant bits (k ln2_1 and k ln2_2 are
exact for |k| < 2^14), 2^(j/128) stored as a double-float pair.

log: Tang's table-driven method (ACM TOMS 16(4), 1990) on a 1/128 grid:
y = 2^m f, f in [1/sqrt2, sqrt2), F_j = 1 + j/128 nearest f (j = -38..53),
c_j = 1/F_j rounded to FP32, r = f c_j - 1 (f_hi c_j exact as a two-product),
    ln y = m ln2 + L_j + log1p(r),   L_j = -ln(c_j) as a double-float pair,
|r| <= 2^-7.5; ln2 in three FP32 parts of 12, 12 and 24 bits.  log1p(u) for
u in [-1/2, 1] takes the same rows (j = -64..128) with r = (c_j - 1) + c_j u,
c_j - 1 exact (Sterbenz), so that 1 + u is never rounded.

Run:  python gen_df32_tables.py   (needs mpmath)
"""
import importlib.util
import os
import struct

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "fv_df32_tables.h")
mp.mp.dps = 60

DF_TERMS = 5      # coefficients of degree 0..4 as double-float pairs
STRIDE = 16       # floats per erfcx piece: c, 5 pairs, 4 singles, pad (64 bytes)
EXP_N = 128
LOG_N = 128
LOG_J = range(-64, 129)   # [1/sqrt2, sqrt2) for log, 1 + u on [1/2, 2] for log1p


def f32(v):
    """v rounded to the nearest FP32 number."""
    return struct.unpack("<f", struct.pack("<f", float(v)))[0]


def split(v):
    """hi + lo, both FP32, hi = fl32(v), lo = fl32(v - hi)."""
    hi = f32(v)
    return hi, f32(mp.mpf(v) - hi)


def bits_split(v, bits):
    """v rounded to `bits` significant bits (a number exact in FP32)."""
    e = int(mp.floor(mp.log(abs(v), 2)))
    q = mp.mpf(2) ** (e - bits + 1)
    return float(mp.nint(mp.mpf(v) / q) * q)


def _fp64_gen():
    spec = importlib.util.spec_from_file_location("gen_fp64_tables",
                                                  os.path.join(HERE, "gen_fp64_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def erfcx(z):
    return mp.exp(z * z) * mp.erfc(z)


def fit(a, b, degree):
    """Monomial coefficients in v = z - c of the Chebyshev interpolant, in mpmath."""
    c = (a + b) / 2
    half = (b - a) / 2
    n = degree + 1
    nodes = [half * mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n)]
    A = mp.matrix([[v ** j for j in range(n)] for v in nodes])
    y = mp.matrix([erfcx(c + v) for v in nodes])
    coef = mp.lu_solve(A, y)
    return c, [coef[j] for j in range(n)]


def erfcx_rows():
    g = _fp64_gen()
    rows = []
    for a, b in g.pieces():
        c, coefs = fit(a, b, g.DEGREE)
        assert f32(c) == float(c), "piece centre not exact in FP32"
        row = [f32(c)]
        for k in range(DF_TERMS):
            row += list(split(coefs[k]))
        row += [f32(cf) for cf in coefs[DF_TERMS:]]
        row += [0.0] * (STRIDE - len(row))
        rows.append(row)
    return rows


def exp_rows():
    rows = []
    for j in range(EXP_N):
        rows.append(split(mp.mpf(2) ** (mp.mpf(j) / EXP_N)))
    return rows


def log_rows():
    rows = []
    for j in LOG_J:
        c = 1.0 if j == 0 else f32(1 / (1 + mp.mpf(j) / LOG_N))
        hi, lo = (0.0, 0.0) if j == 0 else split(-mp.log(mp.mpf(c)))
        rows.append((c, hi, lo))
    return rows


def three_parts(v, b1, b2):
    p1 = bits_split(v, b1)
    p2 = bits_split(mp.mpf(v) - p1, b2)
    p3 = f32(mp.mpf(v) - p1 - p2)
    return p1, p2, p3


def four_parts(v, b1, b2):
    p1, p2, p3 = three_parts(v, b1, b2)
    return p1, p2, p3, f32(mp.mpf(v) - p1 - p2 - p3)


def consts():
    ln2 = mp.log(2)
    out = {}
    out["FV_DF_LN2_1"], out["FV_DF_LN2_2"], out["FV_DF_LN2_3"] = three_parts(ln2, 12, 12)
    (out["FV_DF_EXP_L1"], out["FV_DF_EXP_L2"], out["FV_DF_EXP_L3"],
     out["FV_DF_EXP_L4"]) = four_parts(ln2 / EXP_N, 10, 10)
    out["FV_DF_EXP_INV"] = f32(EXP_N / ln2)
    pairs = {
        "INV_SQRT2": 1 / mp.sqrt(2),
        "SQRT2PI": mp.sqrt(2 * mp.pi),
        "INV_SQRT2PI": 1 / mp.sqrt(2 * mp.pi),
        "SQRT_PI_2": mp.sqrt(mp.pi / 2),
        "SQRT_2_PI": mp.sqrt(2 / mp.pi),
        "INV_SQRTPI": 1 / mp.sqrt(mp.pi),
        "THIRD": mp.mpf(1) / 3,
        "SIXTH": mp.mpf(1) / 6,
        "INV120": mp.mpf(1) / 120,
        "INV5040": mp.mpf(1) / 5040,
    }
    for k, v in pairs.items():
        out["FV_DF_%s_HI" % k], out["FV_DF_%s_LO" % k] = split(v)
    return out


def _lit(v):
    r = repr(float(v))
    if "e" not in r and "." not in r and "inf" not in r:
        r += ".0"
    return r + "f"


def write(out=OUT):
    er, ex, lg, cs = erfcx_rows(), exp_rows(), log_rows(), consts()
    lines = [
        "// Generated by gen_df32_tables.py (beside this file); do not edit.",
        "#pragma once",
        "",
        "// FV_DF_TABLE is __device__ in CUDA builds and empty in host builds of the",
        "// double-float functions (fv_df32.cuh).",
        "#ifndef FV_DF_TABLE",
        "#define FV_DF_TABLE",
        "#endif",
        "",
        "// erfcx: piece k (the pieces of the FP64 table) holds its centre c_k, the",
        "// coefficients of degree 0..%d of the polynomial in v = z - c_k as (hi, lo)" % (DF_TERMS - 1),
        "// pairs, those of degree %d..8 as FP32, and a pad: %d floats." % (DF_TERMS, STRIDE),
        "#define FV_DF_ERFCX_PIECES %d" % len(er),
        "#define FV_DF_ERFCX_STRIDE %d" % STRIDE,
        "static FV_DF_TABLE __align__(64) const float kErfcxDf[FV_DF_ERFCX_PIECES * FV_DF_ERFCX_STRIDE] = {",
    ]
    for row in er:
        lines.append("    " + ", ".join(_lit(v) for v in row) + ",")
    lines += [
        "};",
        "",
        "// exp: row j holds 2^(j/128) as (hi, lo).",
        "#define FV_DF_EXP_N %d" % EXP_N,
        "static FV_DF_TABLE __align__(8) const float kExpDf[FV_DF_EXP_N * 2] = {",
    ]
    for hi, lo in ex:
        lines.append("    %s, %s," % (_lit(hi), _lit(lo)))
    lines += [
        "};",
        "",
        "// log: row j + %d holds c_j = 1/(1 + j/128) rounded to FP32 (c_0 = 1) and" % -LOG_J[0],
        "// -ln(c_j) as (hi, lo), and a pad.",
        "#define FV_DF_LOG_J0 %d" % LOG_J[0],
        "#define FV_DF_LOG_ROWS %d" % len(lg),
        "static FV_DF_TABLE __align__(16) const float kLogDf[FV_DF_LOG_ROWS * 4] = {",
    ]
    for c, hi, lo in lg:
        lines.append("    %s, %s, %s, 0.0f," % (_lit(c), _lit(hi), _lit(lo)))
    lines += ["};", ""]
    for k, v in cs.items():
        lines.append("#define %s %s" % (k, _lit(v)))
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    return out


if __name__ == "__main__":
    print(write())
