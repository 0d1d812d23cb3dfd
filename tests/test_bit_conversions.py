"""The integer-unit helpers of the kernels' hot loops (csrc/fv_device.cuh),
step by step on the CPU: the FP64 <-> FP32 conversions f32_trunc and f64_of
against numpy's (truncation within 2^-23 relative, exact widening, the stated
handling of zeros, FP32 range limits, infinities and NaN), the reciprocal
recip64 and Markstein's division div64 against the rounded quotient, the
exponent-field halving half64, and the convergence test |ds| > tol s on the
bit patterns against the FP64 comparison."""
import struct

import numpy as np


def _hi_lo(d):
    b = struct.unpack("<Q", struct.pack("<d", d))[0]
    return b >> 32, b & 0xffffffff


def f32_trunc(d):
    hi, lo = _hi_lo(d)
    e = ((hi >> 20) & 0x7ff) - 896
    sign = hi & 0x80000000
    frac = ((hi & 0xfffff) << 3) | (lo >> 29)
    bits = sign if e <= 0 else (sign | 0x7f800000 if e >= 255 else sign | (e << 23) | frac)
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def f64_of(f):
    b = struct.unpack("<I", struct.pack("<f", f))[0]
    e = (b >> 23) & 0xff
    sign = b & 0x80000000
    normal = e not in (0, 255)
    e64 = 0 if e == 0 else (0x7ff if e == 255 else e + 896)
    frac = b & 0x7fffff if normal else 0
    hi = sign | (e64 << 20) | (frac >> 3)
    lo = (frac << 29) & 0xffffffff
    return struct.unpack("<d", struct.pack("<Q", (hi << 32) | lo))[0]


def test_truncation_within_fp32_resolution():
    g = np.random.default_rng(1)
    d = np.concatenate([np.exp(g.uniform(np.log(1.2e-38), np.log(3.3e38), 20000)) * g.choice([-1, 1], 20000),
                        [1.0, -1.0, 0.1, 3.4028234663852886e38, 1.1754943508222875e-38]])
    for v in d:
        t = f32_trunc(float(v))
        assert abs(t) <= abs(v) and np.sign(t) == np.sign(v)
        assert abs(t - v) <= abs(v) * 2.0 ** -23, v
        # truncation is one of the two FP32 neighbours of v
        r = float(np.float32(v))
        assert t == r or t == float(np.nextafter(np.float32(r), np.float32(0)))


def test_truncation_special_values():
    assert f32_trunc(0.0) == 0.0 and str(f32_trunc(-0.0)) == "-0.0"
    assert f32_trunc(1e-40) == 0.0 and f32_trunc(-1e-300) == 0.0
    assert f32_trunc(1e39) == np.inf and f32_trunc(-1e300) == -np.inf
    assert f32_trunc(np.inf) == np.inf and f32_trunc(-np.inf) == -np.inf
    assert f32_trunc(np.nan) in (np.inf, -np.inf)


def test_widening_is_exact():
    g = np.random.default_rng(2)
    f = np.concatenate([np.exp(g.uniform(np.log(1.2e-38), np.log(3.3e38), 20000)).astype(np.float32),
                        np.float32([1, -1, 0.1, 3.4028235e38, 1.1754944e-38, -2.5])])
    for v in f:
        assert f64_of(float(v)) == float(v)
    assert f64_of(0.0) == 0.0 and str(f64_of(-0.0)) == "-0.0"
    assert f64_of(float(np.float32(1e-40))) == 0.0  # FP32 subnormal
    assert f64_of(np.inf) == np.inf and f64_of(-np.inf) == -np.inf
    assert f64_of(float("nan")) in (np.inf, -np.inf)



def _fma(x, y, z):
    """x*y + z rounded once (what the GPU's FMA does)."""
    from fractions import Fraction
    return float(Fraction(x) * Fraction(y) + Fraction(z))


def _recip64(s):
    """The kernels' recip64 for s in FP32's normal range: the FP32 reciprocal of
    the truncated s (correctly rounded, as __frcp_rn), then two Newton steps."""
    r = f64_of(float(np.float32(1.0) / np.float32(f32_trunc(s))))
    r = _fma(r, _fma(-s, r, 1.0), r)
    return _fma(r, _fma(-s, r, 1.0), r)


def _div64(a, b):
    r = _recip64(b)
    q = a * r
    return _fma(_fma(-q, b, a), r, q)


def test_reciprocal_and_markstein_division():
    # the reciprocal within an ulp; the quotient the rounded one but for rare
    # last-place misses
    g = np.random.default_rng(3)
    b = np.exp(g.uniform(np.log(1e-30), np.log(1e30), 5000))
    a = np.exp(g.uniform(np.log(1e-30), np.log(1e30), 5000)) * g.choice([-1, 1], 5000)
    miss = 0
    for ai, bi in zip(a, b):
        r = _recip64(float(bi))
        assert abs(r - 1.0 / float(bi)) <= abs(np.spacing(1.0 / float(bi)))
        q = _div64(float(ai), float(bi))
        exact = float(ai) / float(bi)
        if q != exact:
            miss += 1
            assert abs(q - exact) <= abs(np.spacing(exact)), (ai, bi)
    assert miss <= len(a) * 2e-3, miss


def _half64(v):
    """The kernels' half64: v/2 on the bit pattern."""
    b = struct.unpack("<q", struct.pack("<d", v))[0]
    e = (b >> 52) & 0x7ff
    sign = b & -0x8000000000000000
    if e >= 2:
        r = b if e == 0x7ff else b - (1 << 52)
    else:
        r = sign | ((b & 0x7fffffffffffffff) >> 1)
    return struct.unpack("<d", struct.pack("<q", r))[0]


def test_half_on_the_exponent_field():
    g = np.random.default_rng(4)
    v = np.concatenate([np.exp(g.uniform(np.log(1e-307), np.log(1e307), 5000)) * g.choice([-1, 1], 5000),
                        [1.0, -3.0, 2.2250738585072014e-308 * 2, 2.2250738585072014e-308, 1.7976931348623157e308]])
    for x in v:
        assert _half64(float(x)) == float(x) / 2, x
    # subnormals: truncated halving (within one subnormal step)
    for x in (5e-324, 1e-310, -3e-320):
        assert abs(_half64(x) - x / 2) <= 5e-324
    assert _half64(0.0) == 0.0 and str(_half64(-0.0)) == "-0.0"
    assert _half64(np.inf) == np.inf and _half64(-np.inf) == -np.inf and np.isnan(_half64(np.nan))


def _moved_more(ds, s, tol):
    """The kernels' |ds| > tol s for a power-of-two tol, on the patterns."""
    q = lambda d: struct.unpack("<q", struct.pack("<d", d))[0]
    bt, bs = q(tol), q(s)
    if (bt & 0xfffffffffffff) != 0 or bs < (64 << 52) or bt <= 0:
        return abs(ds) > tol * s
    return (q(ds) & 0x7fffffffffffffff) > bs + (bt - (1023 << 52))


def test_convergence_test_on_the_patterns():
    g = np.random.default_rng(5)
    tol = 2.0 ** -17
    s = np.exp(g.uniform(np.log(1e-250), np.log(1e250), 3000))
    for si in s:
        si = float(si)
        lim = tol * si
        for ds in (lim, -lim, np.nextafter(lim, 0), np.nextafter(lim, np.inf), -np.nextafter(lim, np.inf),
                   lim * g.uniform(0.5, 2.0), 0.0):
            assert _moved_more(float(ds), si, tol) == (abs(float(ds)) > lim), (ds, si)
