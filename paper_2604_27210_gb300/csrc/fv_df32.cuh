// fv_df32.cuh -- double-float (df32) arithmetic and the mixed solver's
// Householder(3) correction evaluated in it.
//
// A double-float number is an unevaluated sum h + l of two FP32 numbers,
// |l| <= ulp(h)/2: 48 significant bits from FP32 arithmetic, built from the
// error-free transformations of Dekker (Numer. Math. 18, 1971) and Knuth
// (TAOCP vol. 2, 4.2.2): a + b = s + e exactly (two_sum) and a b = p + e
// exactly with one fused multiply-add (two_prod).
//
// Why: on this GPU an FP64 instruction holds its SM sub-partition's pipe for
// ~64 cycles, against one cycle of issue for an FP32 one.  The mixed solver
// (Section 2.2's LBR, FP32 iterations, then one Householder(3) correction at
// FP64 accuracy) spent most of its time in the FP64 evaluation of the
// normalised Black residual for that correction.  Here the residual is
// evaluated in double-float: the correction step needs the residual to
// ~2^-47 relative, which moves sigma by ~2^-47 times the objective's
// conditioning (O(1) for the LBR's three-branch objective), far inside
// 1e-12.  Quotes whose scales leave FP32's exponent range return false and
// the caller takes the FP64 correction.
//
// The header compiles as CUDA device code and as plain C++ (the CPU tests
// build it with the host compiler and compare every function with mpmath):
// the error-free transformations use the non-contracting intrinsics on the
// device and plain operations on the host (built with -ffp-contract=off), and
// the special functions use nothing but +, -, *, fma, the correctly rounded
// reciprocal and square root, and their own tables (fv_df32_tables.h, written
// by gen_df32_tables.py), so both builds give the same bits.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define FV_DF_FN __device__ __forceinline__
#define FV_DF_TABLE __device__
#else
#define FV_DF_FN inline
#ifndef __align__
#define __align__(n) __attribute__((aligned(n)))
#endif
#endif

#include "fv_df32_tables.h"

namespace fvdf {

struct df {
  float h, l;
};

// ---------------------------------------------------------------------------
// FP32 operations that are never contracted, bit access
// ---------------------------------------------------------------------------
FV_DF_FN float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
FV_DF_FN float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
FV_DF_FN float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
FV_DF_FN float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
// correctly rounded reciprocal and square root
FV_DF_FN float rcp(float a) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(a);
#else
  return 1.0f / a;
#endif
}
FV_DF_FN float sqrt_(float a) {
#ifdef __CUDA_ARCH__
  return __fsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}
FV_DF_FN uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
FV_DF_FN float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}
FV_DF_FN uint64_t dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
#endif
}
FV_DF_FN double bitsd(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}
// unsigned integer to FP32, rounded to nearest
FV_DF_FN float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(u);
#else
  return (float)u;
#endif
}
// 2^e as FP32 for -126 <= e <= 127
FV_DF_FN float pow2f(int e) { return bitsf((uint32_t)(e + 127) << 23); }

struct f4 {
  float x, y, z, w;
};
FV_DF_FN f4 ld4(const float* p) {
#ifdef __CUDA_ARCH__
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {v.x, v.y, v.z, v.w};
#else
  return {p[0], p[1], p[2], p[3]};
#endif
}
FV_DF_FN df ld2(const float* p) {
#ifdef __CUDA_ARCH__
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
#else
  return {p[0], p[1]};
#endif
}

// ---------------------------------------------------------------------------
// error-free transformations and double-float arithmetic
// ---------------------------------------------------------------------------
// a + b = s + e exactly (Knuth)
FV_DF_FN df two_sum(float a, float b) {
  const float s = add(a, b);
  const float bb = sub(s, a);
  return {s, add(sub(a, sub(s, bb)), sub(b, bb))};
}
// a + b = s + e exactly where a == 0 or exponent(a) >= exponent(b) (Dekker)
FV_DF_FN df fast_two_sum(float a, float b) {
  const float s = add(a, b);
  return {s, sub(b, sub(s, a))};
}
// a b = p + e exactly (one fused multiply-add)
FV_DF_FN df two_prod(float a, float b) {
  const float p = mul(a, b);
  return {p, fma_(a, b, -p)};
}
FV_DF_FN df mk(float h) { return {h, 0.0f}; }
FV_DF_FN df neg(df a) { return {-a.h, -a.l}; }
// x + y for any signs and magnitudes (cancellation included): relative error
// ~2^-47 of max(|x|, |y|)
FV_DF_FN df dadd(df x, df y) {
  const df s = two_sum(x.h, y.h);
  return two_sum(s.h, add(add(s.l, x.l), y.l));
}
FV_DF_FN df dsub(df x, df y) { return dadd(x, neg(y)); }
// c + y where |y| is well below |c| (Horner steps of convergent series)
FV_DF_FN df dadd_fast(df c, df y) {
  const df s = fast_two_sum(c.h, y.h);
  return fast_two_sum(s.h, add(add(s.l, c.l), y.l));
}
FV_DF_FN df dmul(df x, df y) {
  const df p = two_prod(x.h, y.h);
  return fast_two_sum(p.h, fma_(x.l, y.h, fma_(x.h, y.l, p.l)));
}
FV_DF_FN df dmulf(df x, float f) {
  const df p = two_prod(x.h, f);
  return fast_two_sum(p.h, fma_(x.l, f, p.l));
}
FV_DF_FN df dsqr(df x) {
  const df p = two_prod(x.h, x.h);
  return fast_two_sum(p.h, fma_(add(x.h, x.h), x.l, p.l));
}
// exact scaling by a power of two (no underflow of the tail assumed)
FV_DF_FN df dscale(df x, float p2) { return {mul(x.h, p2), mul(x.l, p2)}; }
// 1/y: the FP32 reciprocal r and one Newton correction r (1 - y r), whose
// head 1 - y_h r is exact by one FMA
FV_DF_FN df drcp(df y) {
  const float r = rcp(y.h);
  float e = fma_(-y.h, r, 1.0f);
  e = fma_(-y.l, r, e);
  return fast_two_sum(r, mul(r, e));
}
// 1/sqrt(y) for y > 0: the correctly rounded FP32 seed r = 1/sqrt(y_h) and one
// Newton step r + r (1 - y r^2)/2, the residual formed in double-float
FV_DF_FN df drsqrt(df y) {
  const float r = rcp(sqrt_(y.h));
  const df r2 = two_prod(r, r);
  const df e = dsub(mk(1.0f), dmul(y, r2));  // ~2^-23: the head cancels
  return fast_two_sum(r, mul(mul(r, e.h), 0.5f));
}

// ---------------------------------------------------------------------------
// conversions with FP64 on the integer unit (an FP64 conversion issues on the
// FP64 pipe on this GPU)
// ---------------------------------------------------------------------------
// A double-float within 2^-47 of d (the head truncated to FP32, the tail the
// next bits rounded), for 2^-100 <= |d| < 2^127; false outside that range
// (and for zero, subnormals, infinities and NaN).
FV_DF_FN bool df_of(double d, df& out) {
  const uint64_t b = dbits(d);
  const int E = (int)((b >> 52) & 0x7ff) - 1023;
  if (E < -100 || E > 126) return false;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint32_t frac23 = (uint32_t)((b >> 29) & 0x7fffffu);
  const float hi = bitsf(sign | ((uint32_t)(E + 127) << 23) | frac23);
  // the 29 bits below the head: m29 2^(E - 52) = (m29 2^-29) 2^(E - 23)
  const float m = mul(u2f((uint32_t)(b & 0x1fffffffu)), 1.862645149230957e-09f);  // 2^-29
  const float lo = mul(m, pow2f(E - 23));  // E - 23 in [-123, 103]
  out = {hi, sign ? -lo : lo};
  return true;
}
// the double h + l (exact: 48 bits fit FP64's 53), widening on the integer unit
FV_DF_FN double widen(float f) {
  const uint32_t b = fbits(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u) return bitsd((uint64_t)(b & 0x80000000u) << 32);  // zero (subnormals flushed)
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const uint64_t e64 = e == 255u ? 0x7ffu : (uint64_t)(e + 896u);
  return bitsd(sign | (e64 << 52) | ((uint64_t)(b & 0x7fffffu) << 29));
}
FV_DF_FN double to_double(df a) { return widen(a.h) + widen(a.l); }

// ---------------------------------------------------------------------------
// exp, log, erfcx in double-float
// ---------------------------------------------------------------------------
// e^a for -70 <= a_h <= 87 (the result and its tail stay normal FP32 numbers):
// k = round(a 128/ln2), r = a - k ln2/128 (ln2/128 in four parts: k ln2_1 and
// k ln2_2 exact and both subtractions exact, k ln2_3 a two-product, k ln2_4
// rounded), e^a = 2^(k>>7) 2^(j/128) (1 + expm1(r)), j = k & 127,
// expm1(r) = r + r^2/2 in double-float plus r^3/6 + r^4/24 + r^5/120 in FP32
// (|r| <= ln2/256: the FP32 tail's rounding is below 2^-52).  ~2^-46.
FV_DF_FN df dexp(df a) {
  const float t = fma_(a.h, FV_DF_EXP_INV, 12582912.0f);  // 1.5 2^23: round to integer
  const int k = (int)(fbits(t) - fbits(12582912.0f));
  const float kd = sub(t, 12582912.0f);
  const float r1 = fma_(-kd, FV_DF_EXP_L2, fma_(-kd, FV_DF_EXP_L1, a.h));
  const df r = dadd(dsub(two_sum(r1, a.l), two_prod(kd, FV_DF_EXP_L3)), mk(mul(-kd, FV_DF_EXP_L4)));
  const df r2 = dsqr(r);
  const float rh = r.h;
  const float tail = mul(mul(mul(rh, rh), rh),
                         fma_(fma_(rh, 1.0f / 120.0f, 1.0f / 24.0f), rh, 1.0f / 6.0f));
  const df em1 = dadd(r, dadd_fast(dscale(r2, 0.5f), mk(tail)));
  const df T = ld2(kExpDf + 2 * (k & (FV_DF_EXP_N - 1)));
  const df e = dadd_fast(T, dmul(T, em1));
  return dscale(e, pow2f(k >> 7));
}

// e^a and expm1(a) for -70 <= a <= 0 from one reduction, e^a to ~2^-46 and
// expm1(a) to ~2^-44 relative (the table's pair holds 2^(j/128) to 2^-48,
// against an expm1 down to ~1/200 of it): expm1(r) = r + r^2/2 + r^3/6 in
// double-float plus r^4/24 + r^5/120
// + r^6/720 in FP32 (below 2^-28 of r), and
//   expm1(a) = (2^m T_h - 1) + 2^m (T_l + T expm1(r)),
// the first term exact for m = 0, -1 (Sterbenz) and the two never cancelling
// by more than a factor ~1.3; below |a| = 1/200 the reduction is skipped
// (k = 0, expm1(a) = expm1(r)).
FV_DF_FN df dexp_em1(df a, df& em1_out) {
  const bool tiny = fabsf(a.h) < 0.005f;
  const float t = fma_(a.h, FV_DF_EXP_INV, 12582912.0f);
  const int k = tiny ? 0 : (int)(fbits(t) - fbits(12582912.0f));
  const float kd = tiny ? 0.0f : sub(t, 12582912.0f);
  const float r1 = fma_(-kd, FV_DF_EXP_L2, fma_(-kd, FV_DF_EXP_L1, a.h));
  const df r = dadd(dsub(two_sum(r1, a.l), two_prod(kd, FV_DF_EXP_L3)), mk(mul(-kd, FV_DF_EXP_L4)));
  const df r2 = dsqr(r);
  const df r3 = dmul(r2, r);
  const float rh = r.h;
  const float tail = mul(mul(r2.h, r2.h), fma_(fma_(rh, 1.0f / 720.0f, 1.0f / 120.0f), rh, 1.0f / 24.0f));
  const df em1 = dadd(r, dadd_fast(dscale(r2, 0.5f), dadd_fast(dmul(r3, df{FV_DF_SIXTH_HI, FV_DF_SIXTH_LO}), mk(tail))));
  const df T = ld2(kExpDf + 2 * (k & (FV_DF_EXP_N - 1)));
  const float p2 = pow2f(k >> 7);
  const df Tem1 = dadd(dmul(T, em1), mk(T.l));
  em1_out = dadd(two_sum(mul(T.h, p2), -1.0f), dscale(Tem1, p2));
  return dscale(dadd_fast(mk(T.h), Tem1), p2);
}

// ln(2^m f) for f = fh + fl in [1/sqrt2, sqrt2) (fh with 24 bits): Tang's
// table-driven method on a 1/128 grid, r = f c_j - 1 exact as a double-float
// (f_h c_j a two-product, its head minus one exact by Sterbenz), log1p(r) =
// r - r^2/2 in double-float plus r^3/3 - ... - r^6/6 in FP32 (|r| <= 2^-8:
// absolute error below 2^-49), m ln2 from three parts (the first two
// products exact for |m| < 2^11).
// log1p(r) for |r| <= 2^-7: r - r^2/2 + r^3/3 in double-float, -r^4/4 + r^5/5 -
// r^6/6 in FP32 (below 2^-30 of r: their rounding is below 2^-54 of the
// result, which stays within 2^-47 relative for any such r)
FV_DF_FN df log1p_small(df r) {
  const df r2 = dsqr(r);
  const df r3 = dmul(r2, r);
  const float rh = r.h;
  const float poly = fma_(fma_(rh, -1.0f / 6.0f, 0.2f), rh, -0.25f);
  const float tail = mul(mul(r2.h, r2.h), poly);
  const df t3 = dmul(r3, df{FV_DF_THIRD_HI, FV_DF_THIRD_LO});
  return dadd(r, dadd_fast(dscale(neg(r2), 0.5f), dadd_fast(t3, mk(tail))));
}
FV_DF_FN df dlog_core(int m, float fh, float fl) {
  const float jf = sub(fma_(fh, 128.0f, 12582784.0f), 12582912.0f);  // round((f - 1) 128)
  const int j = (int)jf;
  const f4 row = ld4(kLogDf + 4 * (j - FV_DF_LOG_J0));
  const df p = two_prod(fh, row.x);
  const df r = two_sum(sub(p.h, 1.0f), fma_(fl, row.x, p.l));
  const df l1p = log1p_small(r);
  const float mf = (float)m;
  const df mln2 = dadd(two_sum(mul(mf, FV_DF_LN2_1), mul(mf, FV_DF_LN2_2)), mk(mul(mf, FV_DF_LN2_3)));
  return dadd(dadd(mln2, df{row.y, row.z}), l1p);
}
// The exponent m and significand f = fh + fl in [1/sqrt2, sqrt2) of a
// double-float y with 2^-126 <= y_h < 2^127 (ln y = dlog_core(m, fh, fl))
FV_DF_FN void log_arg(df y, int& m, float& fh, float& fl) {
  const uint32_t b = fbits(y.h);
  m = (int)(b >> 23) - 127;
  uint32_t fb = (b & 0x7fffffu) | 0x3f800000u;
  if (fb >= 0x3fb504f3u) {  // f >= sqrt2: f/2, m + 1
    fb -= 0x800000u;
    m += 1;
  }
  fh = bitsf(fb);
  // y_l 2^-m: two exact power-of-two scalings (2^-m may leave FP32's range)
  fl = mul(mul(y.l, pow2f(-(m / 2))), pow2f(-(m - m / 2)));
}
// the same for any positive normal double d, from its bit pattern: the head
// of the significand and its 29 low bits (each weighing 2^-52)
FV_DF_FN void log_arg_of(double d, int& m, float& fh, float& fl) {
  const uint64_t b = dbits(d);
  m = (int)((b >> 52) & 0x7ff) - 1023;
  uint32_t fb = 0x3f800000u | (uint32_t)((b >> 29) & 0x7fffffu);
  fl = mul(u2f((uint32_t)(b & 0x1fffffffu)), 2.220446049250313e-16f);
  if (fb >= 0x3fb504f3u) {
    fb -= 0x800000u;
    fl = mul(fl, 0.5f);
    m += 1;
  }
  fh = bitsf(fb);
}
FV_DF_FN df dlog(df y) {
  int m;
  float fh, fl;
  log_arg(y, m, fh, fl);
  return dlog_core(m, fh, fl);
}
FV_DF_FN df dlog_of(double d) {
  int m;
  float fh, fl;
  log_arg_of(d, m, fh, fl);
  return dlog_core(m, fh, fl);
}

// log1p(u) for -1/2 <= u <= 1 (a double-float u) with the error of u's own
// precision (~2^-47 relative): the table row j = round(128 u) gives
// ln(1 + u) = -ln c_j + log1p(r), r = c_j (1 + u) - 1 = (c_j - 1) + c_j u with
// c_j - 1 exact (Sterbenz) and c_j u_h a two-product, so 1 + u is never
// rounded; j = 0 (|u| < 1/256) leaves r = u.
FV_DF_FN df dlog1p(df u) {
  const int j = (int)sub(fma_(u.h, 128.0f, 12582912.0f), 12582912.0f);
  const f4 row = ld4(kLogDf + 4 * (j - FV_DF_LOG_J0));
  const df a = two_prod(row.x, u.h);
  const df s = two_sum(sub(row.x, 1.0f), a.h);
  const df r = two_sum(s.h, add(add(s.l, a.l), mul(row.x, u.l)));
  return dadd(df{row.y, row.z}, log1p_small(r));
}

// erfcx(z) = exp(z^2) erfc(z) for z >= 0.  Below 128: the piecewise Chebyshev
// interpolants of the FP64 table (the piece from the bits of z_h), Horner in
// v = z - c_k with the terms of degree 5..8 in FP32 and 0..4 in double-float:
// |v| <= z/32, so the FP32 terms weigh below 2^-25 of the value.  Beyond: the
// asymptotic series (Abramowitz & Stegun 7.1.23) to z^-8.  ~2^-46.
FV_DF_FN df derfcx(df z) {
  const uint32_t b = fbits(z.h);
  if (b < 0x43000000u) {  // z < 128
    const int e = (int)(b >> 23) - 127;
    int k;
    if (e >= -1) {
      k = 8 + ((e + 1) << 4) + (int)((b >> 19) & 15u);
    } else {
      // floor(16 z) = (1.f x 2^23) >> (19 - e) for e = -4..-2, else 0
      k = e >= -4 ? (int)(((b & 0x7fffffu) | 0x800000u) >> (19 - e)) : 0;
    }
    const float* row = kErfcxDf + FV_DF_ERFCX_STRIDE * k;
    const f4 a = ld4(row), bb = ld4(row + 4), c = ld4(row + 8), d = ld4(row + 12);
    // a = (c_k, c0h, c0l, c1h), bb = (c1l, c2h, c2l, c3h), c = (c3l, c4h, c4l, c5),
    // d = (c6, c7, c8, pad)
    const df v = dadd(z, mk(-a.x));
    const float T = fma_(fma_(fma_(d.z, v.h, d.y), v.h, d.x), v.h, c.w);
    df p = dadd_fast(df{c.y, c.z}, dmulf(v, T));
    p = dadd_fast(df{bb.w, c.x}, dmul(v, p));
    p = dadd_fast(df{bb.y, bb.z}, dmul(v, p));
    p = dadd_fast(df{a.w, bb.x}, dmul(v, p));
    return dadd_fast(df{a.y, a.z}, dmul(v, p));
  }
  const df r = drcp(z);
  const df w = dsqr(r);
  const float wh = w.h;
  const float tail = mul(mul(wh, wh), fma_(fma_(wh, 6.5625f, -1.875f), wh, 0.75f));
  const df sum = dadd_fast(mk(1.0f), dadd_fast(dscale(neg(w), 0.5f), mk(tail)));
  return dmul(df{FV_DF_INV_SQRTPI_HI, FV_DF_INV_SQRTPI_LO}, dmul(r, sum));
}

// ---------------------------------------------------------------------------
// normalised Black function in double-float (the forms of fv_device.cuh's
// FP64 nb_eval: erfcx difference, complement, small-t series, asymptote)
// ---------------------------------------------------------------------------
// integer-coefficient polynomial in u (highest degree first) in double-float
template <int N>
FV_DF_FN df dpoly_int(df u, const float (&c)[N]) {
  df p = mk(c[0]);
  for (int i = 1; i < N; i++) p = dadd(dmul(p, u), mk(c[i]));
  return p;
}

// t (A + h R C): the FP64 solver's small-t series (the odd part of
// R(h+t) - R(h-t), R the Mills ratio), u = h^2, w = t^2, A = sum_k w^k
// P_{2k+1}(u)/(2k+1)!, C = sum_k w^k Q_{2k+1}(u)/(2k+1)!, k = 0..5.  The terms
// k <= 3 in double-float, k = 4, 5 in FP32: with u w = x^2/4 below 1/4 where
// the series is used, those weigh below 1.1e-8 (their rounding below 2^-50).
// |h| < 1000 keeps u^5 inside FP32's range.
FV_DF_FN df series_df(df h, float t, df R) {
  const df u = dsqr(h);
  const df w = two_prod(t, t);
  const float uf = u.h, wf = w.h;
  const float p9 = (384.0f + uf * (975.0f + uf * (345.0f + uf * (35.0f + uf)))) * (1.0f / 362880.0f);
  const float q9 = (945.0f + uf * (1260.0f + uf * (378.0f + uf * (36.0f + uf)))) * (1.0f / 362880.0f);
  const float p11 = (3840.0f + uf * (12645.0f + uf * (6090.0f + uf * (938.0f + uf * (54.0f + uf))))) *
                    (1.0f / 39916800.0f);
  const float q11 = (10395.0f + uf * (17325.0f + uf * (6930.0f + uf * (990.0f + uf * (55.0f + uf))))) *
                    (1.0f / 39916800.0f);
  const float a45 = p9 + wf * p11, c45 = q9 + wf * q11;
  const df i6 = {FV_DF_SIXTH_HI, FV_DF_SIXTH_LO}, i120 = {FV_DF_INV120_HI, FV_DF_INV120_LO},
           i5040 = {FV_DF_INV5040_HI, FV_DF_INV5040_LO};
  const float P7[4] = {1.0f, 20.0f, 87.0f, 48.0f}, Q7[4] = {1.0f, 21.0f, 105.0f, 105.0f};
  const float P5[3] = {1.0f, 9.0f, 8.0f}, Q5[3] = {1.0f, 10.0f, 15.0f};
  const float P3[2] = {1.0f, 2.0f}, Q3[2] = {1.0f, 3.0f};
  const df p7 = dmul(dpoly_int(u, P7), i5040), q7 = dmul(dpoly_int(u, Q7), i5040);
  const df p5 = dmul(dpoly_int(u, P5), i120), q5 = dmul(dpoly_int(u, Q5), i120);
  const df p3 = dmul(dpoly_int(u, P3), i6), q3 = dmul(dpoly_int(u, Q3), i6);
  df A = dadd(p7, dmulf(w, a45));
  A = dadd(p5, dmul(w, A));
  A = dadd(p3, dmul(w, A));
  A = dadd(mk(1.0f), dmul(w, A));
  df C = dadd(q7, dmulf(w, c45));
  C = dadd(q5, dmul(w, C));
  C = dadd(q3, dmul(w, C));
  C = dadd(mk(1.0f), dmul(w, C));
  return dmulf(dadd(A, dmul(dmul(h, R), C)), t);
}

// The normalised Black evaluation at (x, s) for a correction step:
//   E = (h^2 + t^2)/2 (so that e = exp(-E) and b = e B), and
//   B = b/e, or C = (b_max - b)/e where `comp` (the highest region) or where
//   the middle regions' value is taken past the inflection point (via_comp).
struct NBdf {
  df h, E, B;
  bool via_comp;
};
//
// The one to three evaluations of erfcx run through a single loop body (one
// copy of the function's code instead of one per call): the correction is
// bound by instruction fetch rather than arithmetic once it leaves FP64.
FV_DF_FN bool nb_df(df x, float s, int reg, NBdf& o) {
  const df inv_s = drcp(mk(s));
  const df h = dmul(x, inv_s);
  const float t = mul(s, 0.5f);
  o.h = h;
  o.E = dscale(dadd(dsqr(h), two_prod(t, t)), 0.5f);
  const bool comp = reg == 3, middle = reg == 1 || reg == 2;
  const bool log_space = reg == 0;
  // the FP64 solver's branch rules: small t (t < 0.1) takes the series, in
  // the lowest region only where |x| < 1 or |x|/s^2 is beyond 1e12
  const bool small = t < 0.1f && !comp && (!log_space || !(x.h <= -1.0f && -x.h < 1e12f * s * s));
  // |h| >= 1000 with small t (lowest region only): the two-term asymptote of
  // the Mills-ratio difference, exact to ~15/h^4 relative, which moves s by
  // ~15/h^6 in log space; it needs no erfcx
  const bool asym = small && !(-h.h < 1000.0f);
  const df ht = dadd(h, mk(t));
  o.via_comp = !small && middle && ht.h > 0.0f;
  const bool csum = comp || o.via_comp;
  // the arguments of erfcx are non-negative: -h for the series, h + t for the
  // complement, -(h + t) and t - h for the direct difference
  if (!small && (csum ? !(ht.h >= 0.0f) : !(ht.h <= 0.0f))) return false;
  const df isq2 = {FV_DF_INV_SQRT2_HI, FV_DF_INV_SQRT2_LO};
  const df z0 = dmul(small ? neg(h) : (csum ? ht : neg(ht)), isq2);
  const df z1 = dmul(dsub(mk(t), h), isq2);
  const int n = asym ? 0 : (small ? 1 : 2);
  df Y0 = mk(0.0f), Y1 = mk(0.0f);
#pragma unroll 1
  for (int i = 0; i < n; i++) {
    const df y = derfcx(i == 0 ? z0 : z1);
    if (i == 0) Y0 = y;
    else Y1 = y;
  }
  const df s2p = {FV_DF_SQRT_2_PI_HI, FV_DF_SQRT_2_PI_LO};
  if (asym) {
    // (t/D)(1 - (3h^2 + t^2)/D^2), D = h^2 - t^2
    const df D = dsub(dsqr(h), two_prod(t, t));
    const df tD = dmulf(drcp(D), t);
    const float corr = (3.0f * h.h * h.h + t * t) / (D.h * D.h);
    o.B = dmul(s2p, dsub(tD, dmulf(tD, corr)));
  } else if (small) {
    o.B = dmul(s2p, series_df(h, t, dmul(df{FV_DF_SQRT_PI_2_HI, FV_DF_SQRT_PI_2_LO}, Y0)));
  } else {
    o.B = dscale(csum ? dadd(Y0, Y1) : dsub(Y0, Y1), 0.5f);
  }
  return true;
}

// The mixed solver's Householder(3) correction of the FP32 iterate s (exact
// in FP32) of region reg, with the residual and the Newton step in
// double-float and the second-order ratios in FP32, the form of the FP64
// solver's hh3_ds_mixed:
//   regions 1, 2: nu = (beta - b)/b'  = sqrt(2 pi) (beta e^E - B), or past the
//                 inflection point sqrt(2 pi) (C - c_beta e^E)
//   region 0:     nu = (ln beta - ln b) ln b / ln beta * b/b',  ln b = ln B - E
//   region 3:     nu = -(ln c_beta - ln(b_max - b)) (b_max - b)/b'
// on the reduced quote as double-float numbers: beta, c_beta = b_max - beta,
// x <= 0, T, and ln beta where has_ln (beta below the double-float range,
// given as 0).  Writes sigma = (s + ds)/sqrt(T) and returns true; returns
// false, writing nothing, where the quote's scales leave the range this
// evaluation covers (the caller then takes the FP64 correction).
FV_DF_FN bool hh3_correction_dfv(df beta, df c_beta, df xd, df ln_beta, bool has_ln, df Td, float s,
                                 int reg, double& sigma) {
  if (!(s > 1e-30f && s < 1e30f) || !(Td.h > 1e-30f && Td.h < 1e30f)) return false;
  NBdf v;
  if (!nb_df(xd, s, reg, v)) return false;
  df nu;
  float qf = 0.0f, iLf = 0.0f;
  const df s2pi = {FV_DF_SQRT2PI_HI, FV_DF_SQRT2PI_LO};
  if (reg == 1 || reg == 2) {
    // e^E times the reduced price (or its distance to the bound); E <= 80
    // keeps e^E and the products normal FP32 numbers
    const df p = v.via_comp ? c_beta : beta;
    if (!(v.E.h <= 80.0f) || !(p.h > 1e-26f)) return false;
    const df pe = dmul(p, dexp(v.E));
    nu = dmul(s2pi, v.via_comp ? dsub(v.B, pe) : dsub(pe, v.B));
  } else {
    if (!(v.B.h > 1e-30f) || !(v.E.h < 1e30f)) return false;
    // ln B (or ln C), and ln beta (region 0, unless given) or ln c_beta
    // (region 3), through one loop body of the logarithm
    const df d = reg == 0 ? beta : c_beta;
    const bool given = reg == 0 && has_ln;
    if (!given && !(d.h > 1e-37f)) return false;
    df L1 = given ? ln_beta : mk(0.0f);
    int m0, m1;
    float fh0, fl0, fh1, fl1;
    log_arg(v.B, m0, fh0, fl0);
    log_arg(given ? v.B : d, m1, fh1, fl1);
    df L0 = mk(0.0f);
#pragma unroll 1
    for (int i = 0; i < (given ? 1 : 2); i++) {
      const df l = dlog_core(i == 0 ? m0 : m1, i == 0 ? fh0 : fh1, i == 0 ? fl0 : fl1);
      if (i == 0) L0 = l;
      else L1 = l;
    }
    const df lnX = dsub(L0, v.E);
    const df bq = dmul(v.B, s2pi);  // b/b' (region 0) or (b_max - b)/b' (region 3)
    qf = 1.0f / bq.h;
    iLf = 1.0f / lnX.h;
    if (reg == 0) {
      nu = dmul(dmul(dmul(dsub(L1, lnX), lnX), drcp(L1)), bq);
    } else {
      nu = dmul(neg(dsub(L1, lnX)), bq);
    }
  }
  // second-order ratios in FP32 (they shape the correction factor at O(nu))
  const float hf = v.h.h, sf = s;
  const float hh = hf * hf, is = 1.0f / sf;
  const float u = hh * is - 0.25f * sf;
  const float du = -3.0f * hh * is * is - 0.25f;
  float h2, h3;
  if (reg == 1 || reg == 2) {
    h2 = u;
    h3 = u * u + du;
  } else if (reg == 0) {
    const float k1 = 1.0f + 2.0f * iLf;
    h2 = u - qf * k1;
    h3 = h2 * h2 + du - (qf * u - qf * qf) * k1 + 2.0f * qf * qf * iLf * iLf;
  } else {
    h2 = u + qf;
    h3 = h2 * h2 + du + qf * h2;
  }
  const float nf = nu.h;
  const float phi = nf * (-0.5f * h2 - h3 * nf * (1.0f / 6.0f)) / (1.0f + nf * (h2 + h3 * nf * (1.0f / 6.0f)));
  df ds = (phi - phi == 0.0f) ? dadd(nu, dmulf(nu, phi)) : nu;
  if (!(ds.h - ds.h == 0.0f)) ds = mk(0.0f);
  // the guard of the FP64 solver: a step to s/4 or below stops at s/4
  df sn = dadd(mk(s), ds);
  if (sn.h <= 0.25f * s) sn = mk(0.25f * s);
  sigma = to_double(dmul(sn, drsqrt(Td)));
  return true;
}

// the same from the FP64 reduced quote (ln_beta its preset logarithm or 0)
FV_DF_FN bool hh3_correction_df(double beta, double c_beta, double x, double ln_beta, double T,
                                float s, int reg, double& sigma) {
  df xd, Td, bd = mk(0.0f), cd = mk(0.0f), lb = mk(0.0f);
  if (x == 0.0) {
    xd = mk(0.0f);
  } else if (!df_of(x, xd)) {
    return false;
  }
  if (!df_of(T, Td)) return false;
  bool has_ln = ln_beta != 0.0;
  if (has_ln && !df_of(ln_beta, lb)) return false;
  if (!has_ln && beta > 0.0 && !df_of(beta, bd)) {
    // beta below the double-float range: the lowest region works with ln beta
    if (reg != 0) return false;
    lb = dlog_of(beta);
    has_ln = true;
  }
  if (c_beta > 0.0 && !df_of(c_beta, cd)) return false;
  return hh3_correction_dfv(bd, cd, xd, lb, has_ln, Td, s, reg, sigma);
}

// ---------------------------------------------------------------------------
// The status rule and the reduction to an out-of-the-money call (Section
// 2.2's shared preprocessing) in double-float, for the mixed solver
// ---------------------------------------------------------------------------
// Status codes of the FP64 rule (fv.h's fv_quote_status)
enum { DF_Q_OK = 0, DF_Q_BELOW = 1, DF_Q_ABOVE = 2, DF_Q_INVALID = 3 };

struct NormDF {
  int status;     // the FP64 rule's status (when !fp64)
  bool solve;     // a positive root exists
  bool fp64;      // not decided here: the quote takes the FP64 rule
  bool tiny;      // beta below the double-float range; ln_beta holds ln beta
  df beta, x, bmax, c_beta, ln_beta;  // x = -|ln(F/K)|, c_beta = b_max - beta
};

FV_DF_FN bool finite64(double v) {
  return (dbits(v) & 0x7fffffffffffffffULL) < 0x7ff0000000000000ULL;
}
FV_DF_FN bool pos_finite64(double v) {
  const uint64_t b = dbits(v);
  return b != 0 && b < 0x7ff0000000000000ULL;  // sign clear, nonzero, finite
}
FV_DF_FN double dsub64(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}
// a double-float for d = 0 or 2^-100 <= |d| < 2^127
FV_DF_FN bool df_of0(double d, df& out) {
  if (d == 0.0) {
    out = mk(0.0f);
    return true;
  }
  return df_of(d, out);
}
// within [2^-60, 2^60]: products and quotients of two such stay normal FP32
FV_DF_FN bool mid_range(float v) { return v >= 8.673617379884035e-19f && v <= 1.152921504606847e18f; }

// The decision and the reduced quote of one quote, where the double-float
// evaluation can take them with certainty; otherwise fp64 = true and the
// caller applies the FP64 rule (its status then decides).
//  - Validity: the FP64 rule's tests (non-finite inputs, F, K, T <= 0, flag
//    not +-1: INVALID).
//  - x = ln(F/K): near the money (K/2 <= F <= 2K) log1p((F - K)/K) with F - K
//    exact in FP64 (Sterbenz) and log1p on the unrounded 1 + u; else ln of
//    the ratio.  Black-Scholes / BSM add (r - q) T; where that sum cancels to
//    below 1/8 of its terms the quote takes the FP64 rule (x's error, ~2^-46
//    of the larger term, moves sigma by about that error over max(|x|, s):
//    below 2^-43 relative with the guard).
//  - BELOW where beta < iota (1 - 2^-46) (out of the money iota = 0: exactly
//    where P < 0), ABOVE where the reduced price beta - iota >= b_max
//    (1 - 2^-46): each decided here only farther than 2^-42 of iota or
//    b_max from its threshold (the evaluations carry ~2^-45 and the FP64
//    rule's roundings a few ulp), else the FP64 rule.
//  - In the money (theta x > 0) the reduced price beta - iota cancels: taken
//    here where it keeps at least half of beta, else the FP64 rule.
//  - beta = P e^{rate}/sqrt(F K) (rate = r T, or (r + q) T/2 with S); below
//    2^-90 the reduced price is carried as ln beta = ln P + rate - ln(F K)/2
//    (FP64 keeps beta itself down to its subnormals: quotes where it would
//    underflow take the FP64 rule).
// Scales outside the double-float range take the FP64 rule.
FV_DF_FN NormDF decide_df(int model, double P, double SF, double K, double T, double r,
                          double q, int flag) {
  NormDF o;
  o.status = DF_Q_INVALID;
  o.solve = false;
  o.fp64 = false;
  o.tiny = false;
  o.beta = o.x = o.c_beta = o.ln_beta = mk(0.0f);
  o.bmax = mk(1.0f);
  const bool bsm = model == 2;
  if (!(flag == 1 || flag == -1) || !finite64(P) || !pos_finite64(SF) || !pos_finite64(K) ||
      !pos_finite64(T) || !finite64(r) || (bsm && !finite64(q)))
    return o;
  const double qq = bsm ? q : 0.0;
  df Sd, Kd, Td, rd, qd;
  if (!df_of(SF, Sd) || !df_of(K, Kd) || !df_of(T, Td) || !df_of0(r, rd) || !df_of0(qq, qd) ||
      !mid_range(Sd.h) || !mid_range(Kd.h) || !mid_range(Td.h) || !(rd.h <= 1e6f && rd.h >= -1e6f) ||
      !(qd.h <= 1e6f && qd.h >= -1e6f)) {
    o.fp64 = true;
    return o;
  }
  // x = ln(F/K) (+ (r - q) T)
  df x;
  const uint64_t bs = dbits(SF), bk = dbits(K), one = 1ULL << 52;
  const bool near = bs + one >= bk && bs <= bk + one;  // K/2 <= SF <= 2K (normal SF, K)
  if (near) {
    const double d = dsub64(SF, K);  // exact
    df dd;
    if (!df_of0(d, dd)) {
      o.fp64 = true;
      return o;
    }
    x = dlog1p(dmul(dd, drcp(Kd)));
  } else {
    x = dlog(dmul(Sd, drcp(Kd)));
  }
  if (model != 0) {
    const df g = dmul(dsub(rd, qd), Td);
    const float big = fmaxf(fabsf(x.h), fabsf(g.h));
    x = dadd(x, g);
    if (fabsf(x.h) < 0.125f * big) {
      o.fp64 = true;
      return o;
    }
  }
  const df rate = model == 0 ? dmul(rd, Td) : dscale(dmul(dadd(rd, qd), Td), 0.5f);
  // scales beyond the exponentials' range: the FP64 rule
  if (!(fabsf(x.h) <= 120.0f) || !(fabsf(rate.h) <= 60.0f)) {
    o.fp64 = true;
    return o;
  }
  const bool itm = flag > 0 ? x.h > 0.0f : x.h < 0.0f;
  const df xo = x.h > 0.0f ? neg(x) : x;
  o.x = xo;
  df E;  // expm1(-|x|/2)
  o.bmax = dexp_em1(dscale(xo, 0.5f), E);
  if (P < 0.0) {
    o.status = DF_Q_BELOW;
    return o;
  }
  df Pd;
  df beta = mk(0.0f);
  if (P != 0.0 && df_of(P, Pd)) beta = dmul(dmul(Pd, dexp(rate)), drsqrt(dmul(Sd, Kd)));
  if (itm) {
    // iota = e^{|x|/2} - e^{-|x|/2} = -E (1 + b_max)/b_max, the FP64 rule's
    // form; BELOW where beta < iota (1 - 2^-46), with the guard band 2^-42 iota
    const df iota = dmul(dmul(neg(E), dadd(mk(1.0f), o.bmax)), drcp(o.bmax));
    if (P == 0.0) {
      o.status = DF_Q_BELOW;
      return o;
    }
    if (!(beta.h >= 8.077935669463161e-28f) || !(iota.h > 0.0f)) {
      o.fp64 = true;
      return o;
    }
    const df tb = dsub(beta, dsub(iota, dscale(iota, 1.4210854715202004e-14f)));
    if (fabsf(tb.h) <= 2.2737367544323206e-13f * iota.h) {
      o.fp64 = true;
      return o;
    }
    if (tb.h < 0.0f) {
      o.status = DF_Q_BELOW;
      return o;
    }
    // the reduced price beta - iota, where it keeps at least half of beta
    // (its error is then below 3 2^-46 of it); deeper: the FP64 rule
    const df bo = dsub(beta, iota);
    if (!(bo.h >= 0.5f * beta.h)) {
      o.fp64 = true;
      return o;
    }
    beta = bo;
  }
  o.status = DF_Q_OK;
  if (P == 0.0) return o;  // beta = 0 out of the money: at the intrinsic value, sigma = 0
  if (beta.h >= 8.077935669463161e-28f) {  // 2^-90
    // ABOVE: beta >= b_max (1 - 2^-46), with a guard band of 2^-42 b_max
    const df lim = dsub(o.bmax, dscale(o.bmax, 1.4210854715202004e-14f));
    const df t = dsub(beta, lim);
    if (fabsf(t.h) <= 2.2737367544323206e-13f * o.bmax.h) {
      o.fp64 = true;
      return o;
    }
    if (t.h >= 0.0f) {
      o.status = DF_Q_ABOVE;
      return o;
    }
    o.solve = true;
    o.beta = beta;
    o.c_beta = dsub(o.bmax, beta);
    return o;
  }
  // beta below 2^-90: ln beta from the logarithms of P, F and K
  if (P < 2.2250738585072014e-308 || P > 1e30) {
    o.fp64 = true;
    return o;
  }
  const df lnb = dsub(dadd(dlog_of(P), rate), dscale(dadd(dlog_of(SF), dlog_of(K)), 0.5f));
  // FP64 beta stays normal (its own rule then solves), and far below b_max
  if (!(lnb.h > -700.0f) || !(lnb.h < 0.5f * xo.h - 1.0f)) {
    o.fp64 = true;
    return o;
  }
  o.solve = true;
  o.tiny = true;
  o.ln_beta = lnb;
  o.c_beta = o.bmax;
  return o;
}

}  // namespace fvdf
