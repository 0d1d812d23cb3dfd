// fv_device.cuh -- device math of the GB300 implied-volatility library.
//
// Notation (fast-vollib paper, Section 2.2 and Section 2.4):
//   theta = +1 call / -1 put, x = ln(F/K), s = sigma sqrt(T),
//   beta = P e^{rT} / sqrt(F K)  (normalised, undiscounted price),
//   b(x, s) = e^{x/2} Phi(x/s + s/2) - e^{-x/2} Phi(x/s - s/2)  for the call,
//   h = x/s, t = s/2.
// Every quote is reduced to an out-of-the-money call with x <= 0 (intrinsic
// value subtracted, put/call symmetry b(x,s,theta) = b(-x,s,-theta)).
//
// The normalised Black value is computed as b = e * B with
//   e = exp(-(h^2 + t^2)/2)   (sqrt(2 pi) times the normalised vega b'),
// so that ln b = -(h^2+t^2)/2 + ln B never underflows.  B comes from one of
// two evaluations (Section 2.2 lists erfcx, asymptotic, small-t and CDF-direct
// branches; two suffice here, because the erfcx form below carries the
// CDF-direct and asymptotic regimes without overflow for the arguments the
// solvers reach):
//   erfcx form:  B = [erfcx(-(h+t)/sqrt2) - erfcx((t-h)/sqrt2)] / 2
//   complement:  (b_max - b)/e = [erfcx((h+t)/sqrt2) + erfcx((t-h)/sqrt2)] / 2
//   small t:     B = sqrt(2/pi) sum_k R^{(2k+1)}(h) t^{2k+1} / (2k+1)!
// where R(h) = Phi(h)/phi(h) = sqrt(pi/2) erfcx(-h/sqrt2) is the Mills ratio,
// whose derivatives satisfy R' = 1 + h R, so R^{(n)} = P_n(h) + Q_n(h) R with
// integer polynomials (P_{n+1} = P_n' + Q_n, Q_{n+1} = Q_n' + h Q_n).  The
// series is the odd part of R(h+t) - R(h-t), i.e. the cancellation-free form
// of the erfcx difference when t is small.  Past the inflection point
// (h + t > 0) the value itself is b_max - e (b_max - b)/e: the complement
// needs no reflected erfcx, hence no second exponential.
//
// Every lane of a warp calls the same special functions with lane-selected
// arguments (region-selected coefficients instead of region branches), so the
// four LBR regions do not serialise the FP64 pipe.
#pragma once

#include <cstdint>
#include <type_traits>

#include "fv_df32.cuh"
#include "fv_fp64_tables.h"

namespace fvd {

// mathematical constants
constexpr double kInvSqrt2Pi = 0.398942280401432677939946059934381868;  // 1/sqrt(2 pi)
constexpr double kSqrt2Pi = 2.50662827463100050241576528481104525;      // sqrt(2 pi)
constexpr double kInvSqrt2 = 0.707106781186547524400844362104849039;    // 1/sqrt(2)
constexpr double kSqrtPiOver2 = 1.25331413731550025120788264240552263;  // sqrt(pi/2)
constexpr double kSqrt2OverPi = 0.797884560802865355879892119868763737;  // sqrt(2/pi)
constexpr double kInvSqrt3 = 0.577350269189625764509148780501957456;    // 1/sqrt(3)
constexpr double kInvSqrtPi = 0.564189583547756286948079451560772586;   // 1/sqrt(pi)
constexpr double kLn2Pi = 1.83787706640934548356065947281123527;        // ln(2 pi)
// relative slack band of the three bound tests of the status rule:
// 64 * 2^-52, wider than the few-ulp spread of a price that equals the
// intrinsic value up to rounding, so libm differences cannot flip a decision
constexpr double kEpsS = 1.42108547152020037174224853515625e-14;

enum { Q_OK = 0, Q_BELOW = 1, Q_ABOVE = 2, Q_INVALID = 3 };
enum { M_BLACK76 = 0, M_BS = 1, M_BSM = 2 };

// ---------------------------------------------------------------------------
// precision traits and special-function wrappers (FP64: this file's table-driven
// functions; FP32: CUDA's math library)
// ---------------------------------------------------------------------------
template <typename T>
struct Prec;
template <>
struct Prec<double> {
  // the small-t series is used below t_small with `terms` odd terms; its
  // truncation error is below 1e-17 t there
  static constexpr double t_small = 0.1;
  static constexpr int terms = 6;
  // beyond |h| = h_asym the series' cancellation A + hRC costs eps h^2 and the
  // two-term asymptote of the Mills-ratio difference is exact to 1/h^4
  static constexpr double h_asym = 1e6;
  // ln p below which the inverse normal CDF takes its tail asymptote
  static constexpr double ln_p_floor = -700.0;
};
template <>
struct Prec<float> {
  static constexpr float t_small = 0.3f;
  static constexpr int terms = 4;
  static constexpr float h_asym = 300.0f;
  static constexpr float ln_p_floor = -80.0f;
};

// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversions and FP64 sign / range tests on the integer unit.
// On this GPU a conversion between FP64 and FP32 and an FP64 comparison issue
// on the FP64 pipe like an FMA; the hot loops take them from the bit
// patterns instead, where the integer pipe has room to spare.
// ---------------------------------------------------------------------------
// FP64 -> FP32 with the fraction truncated (relative error below 2^-23).
// Magnitudes below FP32's normal range give a signed zero; beyond it, and
// infinities and NaN, a signed infinity.
__device__ __forceinline__ float f32_trunc(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // FP32 exponent field
  const unsigned sign = hi & 0x80000000u;
  const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned bits =
      e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : (sign | ((unsigned)e << 23) | frac));
  return __uint_as_float(bits);
}

// FP32 -> FP64, exact for normal numbers, zeros and infinities (FP32
// subnormals give zero, NaN an infinity).
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned sign = b & 0x80000000u;
  const bool normal = e != 0u && e != 255u;
  const unsigned e64 = e == 0u ? 0u : (e == 255u ? 0x7ffu : e + 896u);
  const unsigned frac = normal ? (b & 0x7fffffu) : 0u;
  return __hiloint2double((int)(sign | (e64 << 20) | (frac >> 3)), (int)(frac << 29));
}

// v > 0 (or +NaN): positive doubles are exactly the positive 64-bit patterns
__device__ __forceinline__ bool positive64(double v) { return __double_as_longlong(v) > 0; }

// v/2 on the pattern: one less in the exponent field for normal numbers from
// 2^-1021 up, the magnitude bits shifted right below (truncating a subnormal's
// last bit); zero, infinity and NaN pass through
__device__ __forceinline__ double half64(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const long long sign = b & (long long)0x8000000000000000ULL;
  return __longlong_as_double(e >= 2 ? (e == 0x7ff ? b : b - (1LL << 52))
                                     : (sign | ((b & 0x7fffffffffffffffLL) >> 1)));
}

// Rare paths of the FP64 functions below, out of line: a warp whose lanes all
// take the common path pays one untaken branch for them, where inlined code
// of a short rare path can be predicated into every call and take FP64 issue
// slots with no lane active.
static __device__ __noinline__ double recip_rare(double s) { return 1.0 / s; }
static __device__ __noinline__ double exp_rare(double v) { return v < -745.2 ? 0.0 : exp(v); }
static __device__ __noinline__ double exp_expm1_rare(double v, double* em1) {
  *em1 = v < 0.0 ? -1.0 : expm1(v);  // +inf, or NaN
  return v < -745.2 ? 0.0 : exp(v);
}
static __device__ __noinline__ double log_rare(double y) { return log(y); }

// 1/s for s in FP32's normal range (else the FP64 division): the FP32
// reciprocal (relative error ~2^-23 after the truncation) and two Newton
// steps r += r (1 - s r), the error squaring each time; within an ulp.
__device__ __forceinline__ double recip64(double s) {
  const unsigned ah = (unsigned)__double2hiint(s) & 0x7fffffffu;
  if (ah - 0x38200000u >= 0x0fb00000u) return recip_rare(s);  // |s| outside [2^-125, 2^126)
  double r = f64_of(__frcp_rn(f32_trunc(s)));
  r = fma(r, fma(-s, r, 1.0), r);
  return fma(r, fma(-s, r, 1.0), r);
}

// a/b from that reciprocal with Markstein's correction q + (a - q b)/b, the
// remainder a - q b exact by one FMA: the rounded quotient up to a last-place
// difference in rare cases (a non-finite quotient gives NaN or inf)
__device__ __forceinline__ double div64(double a, double b) {
  const double r = recip64(b);
  const double q = a * r;
  return fma(fma(-q, b, a), r, q);
}

__device__ __forceinline__ float f_exp(float v) { return expf(v); }
__device__ __forceinline__ float f_log(float v) { return logf(v); }
// FP64 exponential, the table-driven method of P. T. P. Tang (ACM TOMS
// 15(2), 1989): k = round(v 128/ln2), r = v - k ln2/128 (35-bit head, exact
// product), j = k mod 128, m = floor(k/128),
//   exp(v) = 2^m (T_hi[j] + (T_hi[j] expm1(r) + T_lo[j])),
// T_hi + T_lo = 2^(j/128), expm1(r) to r^5 for |r| <= ln2/256.  Arguments whose
// result is subnormal, infinite or NaN take the library routine; below
// -745.2 the result is 0.
// -708.3 < v < 709.7 (the table's range) on the high word, an integer test
// that keeps the FP64 pipe free; NaN fails it
__device__ __forceinline__ bool exp_table_range(double v) {
  const int hv = __double2hiint(v), ah = hv & 0x7fffffff;
  return ah < (hv >= 0 ? 0x40862d99 : 0x40862266);
}

__device__ __forceinline__ double exp64(double v) {
  if (!exp_table_range(v)) return exp_rare(v);
  const double t = fma(v, FV_EXP_INV_LN2_N, 6755399441055744.0);  // 1.5 * 2^52: round to integer
  const int k = __double2loint(t);
  const double kd = t - 6755399441055744.0;
  double r = fma(kd, -FV_EXP_LN2_N_HI, v);
  r = fma(kd, -FV_EXP_LN2_N_LO, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(r * r, q, r);  // expm1(r)
  const double2 tj = __ldg(reinterpret_cast<const double2*>(kExpTable) + (k & (FV_EXP_N - 1)));
  // times 2^m by adding m to the exponent field (the result is normal here)
  const double r1 = tj.x + fma(tj.x, p, tj.y);
  return __longlong_as_double(__double_as_longlong(r1) + ((long long)(k >> 7) << 52));
}

// exp(v) and expm1(v) from one reduction of the method above (the polynomial
// taken to r^6, so that expm1(r) = p holds to 2^-60 relative):
//   expm1(v) = (2^m T_hi[j] - 1) + 2^m (T_hi[j] p + T_lo[j]).
// 2^m T_hi - 1 is exact for m = 0, -1 (Sterbenz: 2^m T_hi in [1/2, 2)) and
// otherwise below half an ulp of a result beyond 1/2 in magnitude; the second
// term is at most 2^m T_hi ln2/256.  Below |v| = 1/200 the reduction is
// skipped (k = 0, expm1 = p; the polynomial's truncation stays below 2^-60
// there), so that the two terms never cancel by more than a factor ~1.3.
// Within ~1 ulp for both.
__device__ __forceinline__ double exp_expm1_64(double v, double& em1) {
  if (!exp_table_range(v)) return exp_expm1_rare(v, &em1);
  const double t = fma(v, FV_EXP_INV_LN2_N, 6755399441055744.0);
  const bool tiny = (__double2hiint(v) & 0x7fffffff) < 0x3f747ae1;  // |v| < 0.005
  const int k = tiny ? 0 : __double2loint(t);
  const double kd = tiny ? 0.0 : t - 6755399441055744.0;
  double r = fma(kd, -FV_EXP_LN2_N_HI, v);
  r = fma(kd, -FV_EXP_LN2_N_LO, r);
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(r * r, q, r);
  const double2 tj = __ldg(reinterpret_cast<const double2*>(kExpTable) + (k & (FV_EXP_N - 1)));
  const double sc = __hiloint2double(((k >> 7) + 1023) << 20, 0);
  const double th = tj.x * sc;  // exact: a power-of-two scaling of a normal number
  const double tl = tj.y * sc;
  em1 = (th - 1.0) + fma(th, p, tl);
  return th + fma(th, p, tl);
}

// FP64 erfcx(z) = exp(z^2) erfc(z).  FP64 is the scarce unit of this GPU, and
// the solvers evaluate erfcx more often than any other FP64 function, so it
// is not the general library routine: for 0 <= z < 128 a degree-8 piecewise
// Chebyshev interpolant (fv_fp64_tables.h, 136 pieces located from the bits of
// z, within 1.2 ulp); beyond, the asymptotic series (Abramowitz & Stegun
// 7.1.23) to the term in z^-8, whose first omitted term is below 2^-55 there.
//
// The piece index comes from the high word of z alone (integer operations,
// which leave the FP64 pipe to the arithmetic): for z >= 0 the integer order
// of the high words is the numeric order.
// The interpolant of piece k at v = make_v(c_k), the caller's form of
// z - c_k (c_k the piece's centre, the row's first entry).
template <typename MakeV>
__device__ __forceinline__ double erfcx_piece(int k, const MakeV& make_v) {
  // row k: centre, then the coefficients of v^0 .. v^8
  const double2* c = reinterpret_cast<const double2*>(kErfcxTable + k * FV_ERFCX_STRIDE);
  const double2 c0 = __ldg(c), c1 = __ldg(c + 1), c2 = __ldg(c + 2), c3 = __ldg(c + 3),
                c4 = __ldg(c + 4);
  const double v = make_v(c0.x);
  double p = fma(c4.y, v, c4.x);
  p = fma(p, v, c3.y);
  p = fma(p, v, c3.x);
  p = fma(p, v, c2.y);
  p = fma(p, v, c2.x);
  p = fma(p, v, c1.y);
  p = fma(p, v, c1.x);
  return fma(p, v, c0.y);
}

// z >= 128, +inf (gives 0) or NaN (gives NaN); out of line (rare)
static __device__ __noinline__ double erfcx_asymptotic(double z) {
  const double r = 1.0 / z, w = r * r;
  const double sum = fma(w, fma(w, fma(w, fma(w, 6.5625, -1.875), 0.75), -0.5), 1.0);
  return kInvSqrtPi * r * sum;
}

__device__ __forceinline__ double erfcx_nonneg(double z) {
  const int hi = __double2hiint(z);
  if (hi < 0x40600000) {  // z < 128 (FV_ERFCX_TABLE_END)
    const int e = (hi >> 20) - 1023;  // binade 2^e
    int k;
    if (e >= -1) {
      // e = -1..6 and the top four fraction bits: k in 8..135
      k = 8 + ((e + 1) << 4) + ((hi >> 16) & 15);
    } else {
      // floor(16 z) = (1.f x 2^20) >> (16 - e) for e = -4..-2, else 0: k in 0..7
      k = e >= -4 ? ((hi & 0xfffff) | 0x100000) >> (16 - e) : 0;
    }
    return erfcx_piece(k, [&](double c) { return z - c; });  // exact
  }
  return erfcx_asymptotic(z);
}

// erfcx(w/sqrt2) for w >= 0, the form the kernels call (their arguments come
// as h + t, t - h, h, |d|): v = w/sqrt2 - c_k is one FMA, and the piece index
// comes from the FP32 view of z = w/sqrt2 on the integer unit.  That view may
// place z in the neighbouring piece next to an edge (it is within 2^-22 of
// z), where the piece's interpolant, evaluated that little outside its
// interval, keeps its accuracy.
__device__ __forceinline__ double erfcx_nonneg_w(double w) {
  const unsigned b = __float_as_uint(f32_trunc(w) * 0.70710677f);
  if (b < 0x43000000u) {  // z < 128 in FP32
    const int e = (int)(b >> 23) - 127;
    int k;
    if (e >= -1) {
      k = 8 + ((e + 1) << 4) + (int)((b >> 19) & 15u);
    } else {
      // floor(16 z) = (1.f x 2^23) >> (19 - e) for e = -4..-2, else 0
      k = e >= -4 ? (int)(((b & 0x7fffffu) | 0x800000u) >> (19 - e)) : 0;
    }
    return erfcx_piece(k, [&](double c) { return fma(w, kInvSqrt2, -c); });
  }
  return erfcx_asymptotic(w * kInvSqrt2);
}

// erfcx for any z: below zero by reflection, erfcx(z) = 2 exp(z^2) - erfcx(-z),
// with z^2 split exactly into zz + zl so that exp(z^2) = exp(zz) (1 + zl)
// keeps its relative accuracy up to the overflow at z^2 ~ 709.8.
__device__ __forceinline__ double erfcx64(double z) {
  const double p = erfcx_nonneg(fabs(z));
  if (__double2hiint(z) >= 0) return p;  // sign bit clear
  const double zz = z * z, zl = fma(z, z, -zz);
  const double e2 = 2.0 * exp64(zz);
  return isinf(e2) ? e2 : fma(e2, zl, e2) - p;
}

// erfcx(w/sqrt2) for any w, by the same reflection; z^2 = w^2/2 is split
// exactly from w (the halving is exact)
static __device__ __noinline__ double erfcx_w_reflected(double w, double p) {
  const double ww = w * w, wl = fma(w, w, -ww);
  const double e2 = 2.0 * exp64(0.5 * ww);
  return isinf(e2) ? e2 : fma(e2, 0.5 * wl, e2) - p;
}
__device__ __forceinline__ double erfcx64_w(double w) {
  const double p = erfcx_nonneg_w(fabs(w));
  if (__double2hiint(w) >= 0) return p;
  return erfcx_w_reflected(w, p);  // below zero: rare on the solvers' paths
}

// FP64 natural logarithm, the table-driven method of P. T. P. Tang (ACM TOMS
// 16(4), 1990): y = 2^m f with f in [1/sqrt2, sqrt2), F_j = 1 + j/256 the grid
// point nearest f, r = f c_j - 1 (one rounding; c_j = 1/F_j in FP64, c_0 = 1),
//   ln y = (m ln2_hi + L_hi[j]) + (m ln2_lo + L_lo[j] + log1p(r))
// with L_hi + L_lo = -ln(c_j) for the rounded c_j, the first sum exact (both
// terms on a 2^-42 grid) and log1p(r), |r| <= 0.0028, its Taylor polynomial to
// r^6 (truncation below 2^-58 relative).  Zero, negative, subnormal, infinite
// and NaN arguments take the library routine.  With c (|c| below half an ulp
// of y) the result is ln(y + c): c/y = 2^-m c / f enters r as 2^-m c c_j (its
// relative error, |r| <= 0.0028, does not show).
template <bool kWithC>
__device__ __forceinline__ double log64_core(double y, double c) {
  const int hi = __double2hiint(y), lo = __double2loint(y);
  // positive, normal and finite: exponent field 1..2046 with the sign clear
  if ((unsigned)hi - 0x00100000u >= 0x7fe00000u) return log_rare(y);
  const int mant = hi & 0xfffff;
  int m = (hi >> 20) - 1023, j, ehi;
  if (mant >= 0x6a09e) {  // f >= sqrt2: take f/2 in [1/sqrt2, 1), j in -75..0
    m += 1;
    j = ((mant + (1 << 12)) >> 13) - 128;
    ehi = 0x3fe00000;
  } else {                // f in [1, sqrt2), j in 0..106
    j = (mant + (1 << 11)) >> 12;
    ehi = 0x3ff00000;
  }
  const double f = __hiloint2double(ehi | mant, lo);
  const double2* t = reinterpret_cast<const double2*>(kLogTable + (j - FV_LOG_J0) * 4);
  const double2 t0 = __ldg(t), t1 = __ldg(t + 1);  // (c_j, L_hi), (L_lo, pad)
  double r = fma(f, t0.x, -1.0);
  if (kWithC) r = fma(__dmul_rn(c, __hiloint2double((1023 - m) << 20, 0)), t0.x, r);
  double q = fma(r, -1.0 / 6.0, 0.2);
  q = fma(q, r, -0.25);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double p = fma(r * r, q, r);  // log1p(r)
  // m as a double without an int -> FP64 conversion: 2^52 + 2^31 + m is exact
  // in the low word of a double with high word 0x43300000
  const double md = __hiloint2double(0x43300000, m ^ (int)0x80000000) - 4503601774854144.0;
  return fma(md, FV_LN2_HI, t0.y) + (fma(md, FV_LN2_LO, t1.x) + p);
}
__device__ __forceinline__ double log64(double y) { return log64_core<false>(y, 0.0); }
__device__ __forceinline__ double log64(double y, double c) { return log64_core<true>(y, c); }

// ln(1 + u) = ln(y + c), (y, c) the exact sum 1 + u (Knuth's TwoSum)
__device__ __forceinline__ double log1p64(double u) {
  const double y = 1.0 + u, bu = y - 1.0;
  const double c = (1.0 - (y - bu)) + (u - bu);
  return log64(y, c);
}

__device__ __forceinline__ double f_erfcx(double v) { return erfcx64(v); }
__device__ __forceinline__ double f_exp(double v) { return exp64(v); }
__device__ __forceinline__ double f_log(double v) { return log64(v); }
__device__ __forceinline__ float f_erfcx(float v) { return erfcxf(v); }
// erfcx(w/sqrt2)
__device__ __forceinline__ double f_erfcx_w(double w) { return erfcx64_w(w); }
__device__ __forceinline__ float f_erfcx_w(float w) { return erfcxf(w * float(kInvSqrt2)); }
__device__ __forceinline__ double f_half(double v) { return half64(v); }
__device__ __forceinline__ float f_half(float v) { return 0.5f * v; }
__device__ __forceinline__ double f_ncdf(double v) { return normcdf(v); }
__device__ __forceinline__ float f_ncdf(float v) { return normcdff(v); }
__device__ __forceinline__ double f_ncdfinv(double v) { return normcdfinv(v); }
__device__ __forceinline__ float f_ncdfinv(float v) { return normcdfinvf(v); }
__device__ __forceinline__ double f_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float f_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double f_abs(double v) { return fabs(v); }
__device__ __forceinline__ float f_abs(float v) { return fabsf(v); }
__device__ __forceinline__ bool f_finite(double v) { return isfinite(v); }
__device__ __forceinline__ bool f_finite(float v) { return isfinite(v); }

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000LL); }

// ---------------------------------------------------------------------------
// normalisation and the per-quote status decision (always FP64)
// ---------------------------------------------------------------------------
struct Norm {
  int status;       // Q_*
  bool solve;       // OK and strictly above intrinsic: a positive root exists
  double x;         // ln(F/K)
  double beta;      // full normalised price
  double iota;      // normalised intrinsic value
  double beta_otm;  // beta - iota for in-the-money quotes, else beta
  double x_otm;     // -|x|
  double bmax;      // e^{x_otm/2}: upper bound of the reduced call
  double c_beta;    // bmax - beta_otm (the reduced price's distance to its bound)
  double ln_beta;   // ln beta when beta < 1e-280 (else 0: take log(beta_otm))
};

// ln(F/K): near the money F - K is exact (Sterbenz) and log1p keeps x accurate
// relative to itself; log(F/K) would carry one ulp of 1 in absolute error.
// K/2 <= SF <= 2K for positive finite SF, K, on the bit patterns where K's
// exponent field is neither the lowest two nor the highest: there the integer
// order of positive doubles is their numeric order and K/2, 2K differ from K
// by one in the exponent field.
__device__ __forceinline__ bool within_factor_two(double SF, double K) {
  const long long bs = __double_as_longlong(SF), bk = __double_as_longlong(K);
  const long long one = 1LL << 52;
  if (bk >= 2 * one && bk < 0x7fe0000000000000LL) return bs >= bk - one && bs <= bk + one;
  return SF >= 0.5 * K && SF <= 2.0 * K;
}

// One division and one logarithm for both cases: near the money
// log1p(u) = ln(y + c) with y = 1 + u rounded and c = u - (y - 1) its exact
// rounding error (|u| <= 1).
__device__ __forceinline__ double log_moneyness(double SF, double K) {
  const bool near = within_factor_two(SF, K);
  const double u = div64(near ? __dsub_rn(SF, K) : SF, K);
  const double y = near ? __dadd_rn(1.0, u) : u;
  return log64(y, near ? __dsub_rn(u, __dsub_rn(y, 1.0)) : 0.0);
}

// finiteness tests on the bit pattern (integer unit, not the FP64 pipe)
__device__ __forceinline__ bool bits_finite(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool pos_finite(double v) {
  const long long b = __double_as_longlong(v);  // > 0: positive, nonzero; below +inf: finite
  return b > 0 && b < 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool inputs_valid(int model, double SF, double K, double T, double r,
                                             double q, int flag) {
  if (!(flag == 1 || flag == -1)) return false;
  if (!pos_finite(SF) || !pos_finite(K) || !pos_finite(T) || !bits_finite(r)) return false;
  if (model == M_BSM && !bits_finite(q)) return false;
  return true;
}

// x = ln(F/K) for the model (Black-Scholes / BSM: F = S e^{(r-q)T})
__device__ __forceinline__ double model_x(int model, double SF, double K, double T, double r,
                                          double q) {
  const double lm = log_moneyness(SF, K);
  if (model == M_BLACK76) return lm;
  const double qq = model == M_BSM ? q : 0.0;
  return __dadd_rn(lm, __dmul_rn(__dsub_rn(r, qq), T));
}

// The status rule: every product and sum rounded as written (no contraction),
// so the decision matches an FP64 evaluation of the same expressions up to the
// last-place differences of exp / expm1 / log1p / log implementations and of
// the divisions' rare last-place misses, which the 64-ulp band of the bound
// tests absorbs.
__device__ __forceinline__ Norm decide(int model, double P, double SF, double K, double T,
                                       double r, double q, int flag) {
  Norm o;
  o.status = Q_INVALID;
  o.solve = false;
  o.x = o.beta = o.iota = o.beta_otm = o.x_otm = o.ln_beta = 0.0;
  o.bmax = 1.0;
  o.c_beta = 1.0;
  if (!bits_finite(P) || !inputs_valid(model, SF, K, T, r, q, flag)) return o;
  const double qq = model == M_BSM ? q : 0.0;
  const double x = model_x(model, SF, K, T, r, qq);
  double beta;
  const double rate = model == M_BLACK76 ? __dmul_rn(r, T)
                                         : __dmul_rn(half64(__dadd_rn(r, qq)), T);
  // P e^{rate} / sqrt(F K) as a product with the reciprocal square root (one
  // FP64 step instead of a square root and a division; within 1.5 ulp)
  beta = __dmul_rn(__dmul_rn(P, exp64(rate)), rsqrt(__dmul_rn(SF, K)));
  // beta of a price near the bottom of the FP64 range has lost digits to
  // subnormal rounding; its logarithm is taken from P directly
  // (beta < 1e-280 and P > 0 on the bit patterns: beta and P are finite here)
  o.ln_beta = (__double_as_longlong(beta) < __double_as_longlong(1e-280) && __double_as_longlong(P) > 0)
                  ? log64(P) + rate - 0.5 * log64(__dmul_rn(SF, K))
                  : 0.0;
  if (!bits_finite(x) || !bits_finite(beta)) return o;
  // Em = e^{-|x|/2} is the reduced call's bound; with E = Em - 1 (from expm1,
  // accurate near the money) an in-the-money quote's intrinsic value is
  // e^{|x|/2} - e^{-|x|/2} = -E (1 + Em) / Em, accurate for every x
  double E;
  const double Em = exp_expm1_64(-half64(fabs(x)), E);
  // in the money: x > 0 for a call, x < 0 for a put (sign tests on the bits)
  const long long bx = __double_as_longlong(x);
  const bool itm = flag > 0 ? bx > 0 : (bx < 0 && bx != (long long)0x8000000000000000ULL);
  double iota = 0.0;
  if (itm) iota = div64(__dmul_rn(-E, __dadd_rn(1.0, Em)), Em);
  o.x = x;
  o.beta = beta;
  o.iota = iota;
  if (beta < __dmul_rn(iota, 1.0 - kEpsS)) {
    o.status = Q_BELOW;
    return o;
  }
  const double beta_otm = itm ? __dsub_rn(beta, iota) : beta;
  const double bmax = Em;
  if (beta_otm >= __dmul_rn(bmax, 1.0 - kEpsS)) {
    o.status = Q_ABOVE;
    return o;
  }
  o.status = Q_OK;
  o.beta_otm = beta_otm;
  o.x_otm = -fabs(x);
  o.bmax = bmax;
  o.c_beta = __dsub_rn(bmax, beta_otm);
  o.solve = beta_otm > __dmul_rn(iota, kEpsS);
  return o;
}

// ---------------------------------------------------------------------------
// Double-double refinement of the reduced price of ill-conditioned quotes
//
// The inputs are FP64 numbers and the implied volatility is the exact root
// for them, but beta, the intrinsic value iota and the bound b_max above each
// carry a few ulp.  In the money beta_otm = beta - iota cancels, and near the
// upper bound b_max - beta_otm does: sigma moves by ~eps beta/beta_otm (or
// eps b_max/(b_max - beta_otm)) times the quote's own sensitivity, far beyond
// 1e-12 for deep quotes whose normalised vega still exceeds 1e-8.  Both are
// differences of undiscounted prices divided by sqrt(F K):
//   beta_otm sqrt(F K)          = p - theta (F - K)    (in the money),
//   (b_max - beta_otm) sqrt(F K) = bound - p,  bound = F (call) or K (put),
// with p = P e^{rT} and F = S e^{(r-q)T} (Black-76: F given).  Those two
// products are taken in double-double (head + tail), the differences formed
// exactly, and only the final division by sqrt(F K) rounds.
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};
// a + b = s + e exactly (Knuth)
__device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
// a * b = p + e exactly (one FMA)
__device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = __dmul_rn(a, b);
  return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd dd_norm(double hi, double lo) {
  const double s = __dadd_rn(hi, lo);
  return {s, __dsub_rn(lo, __dsub_rn(s, hi))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  dd u = dd_norm(s.hi, __dadd_rn(s.lo, t.hi));
  return dd_norm(u.hi, __dadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const dd p = two_prod(a.hi, b.hi);
  return dd_norm(p.hi, fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo)));
}

// e^a for a double-double a (|a| < 700): the table reduction of exp64,
// a = k ln2/128 + r with |r| <= ln2/256 (k ln2_hi exact, a_hi - k ln2_hi
// exact), expm1(r) = r + r^2/2 in double-double plus the rest of its Taylor
// series (below 3.3e-9 of the result) in FP64, then 2^m (T_hi + T_lo)(1 +
// expm1(r)): relative error ~1e-25, limited by ln2/128's two-part constant.
__device__ __forceinline__ dd exp_dd(dd a) {
  const double t = fma(a.hi, FV_EXP_INV_LN2_N, 6755399441055744.0);
  const int k = __double2loint(t);
  const double kd = t - 6755399441055744.0;
  const double r0 = fma(kd, -FV_EXP_LN2_N_HI, a.hi);
  const dd r = two_sum(r0, fma(kd, -FV_EXP_LN2_N_LO, a.lo));
  const dd r2 = dd_mul(r, r);
  const double rh = r.hi;
  double tail = fma(rh, 1.0 / 40320.0, 1.0 / 5040.0);
  tail = fma(tail, rh, 1.0 / 720.0);
  tail = fma(tail, rh, 1.0 / 120.0);
  tail = fma(tail, rh, 1.0 / 24.0);
  tail = fma(tail, rh, 1.0 / 6.0);
  tail = tail * rh * r2.hi;  // r^3/6 + r^4/24 + ... + r^10/10!
  const dd em1 = dd_add(r, dd_add({0.5 * r2.hi, 0.5 * r2.lo}, {tail, 0.0}));
  const double2 tj = __ldg(reinterpret_cast<const double2*>(kExpTable) + (k & (FV_EXP_N - 1)));
  const dd T = {tj.x, tj.y};
  const dd e = dd_add(T, dd_mul(T, em1));
  const double sc = __hiloint2double(((k >> 7) + 1023) << 20, 0);  // 2^m, exact scaling
  return {e.hi * sc, e.lo * sc};
}

// The reduced quote needs the refinement where the cancellation costs more
// than a factor 64: in the money with beta_otm < beta / 64, or any quote with
// b_max - beta_otm < b_max / 64.  The test takes FP32 views (integer unit,
// FP32 compares): the factor is a threshold, not a result.
__device__ __forceinline__ bool needs_refine(const Norm& n) {
  if (!n.solve) return false;
  const bool itm = positive64(n.iota);
  return (itm && f32_trunc(n.beta_otm) < 0.015625f * f32_trunc(n.beta)) ||
         f32_trunc(n.c_beta) < 0.015625f * f32_trunc(n.bmax);
}
// Status bit of a quote the large-batch LBR kernels (flat and chains) leave
// to their refinement kernel (set between the two launches only).
constexpr uint8_t kRefineMark = 0x80;

// beta_otm (in the money) and c_beta of a quote that needs_refine, from its
// inputs (model, flag as in decide)
__device__ __forceinline__ void refine_reduced_inline(int model, double P, double SF, double K,
                                                      double T, double r, double q, int flag,
                                                      bool itm, double& beta_otm, double& c_beta) {
  // p = P e^{rT}; F and 1/sqrt(F K)
  const dd p = dd_mul(exp_dd(two_prod(r, T)), {P, 0.0});
  dd F = {SF, 0.0};
  double inv_sqrt_fk;
  if (model == M_BLACK76) {
    inv_sqrt_fk = rsqrt(__dmul_rn(SF, K));
  } else {
    const double qq = model == M_BSM ? q : 0.0;
    const dd rq = two_sum(r, -qq);                       // r - q exactly
    const dd g = dd_add(two_prod(rq.hi, T), two_prod(rq.lo, T));  // (r - q) T
    F = dd_mul(exp_dd(g), {SF, 0.0});
    inv_sqrt_fk = __dmul_rn(rsqrt(__dmul_rn(SF, K)), exp64(-half64(g.hi)));
  }
  // A refined value replaces the FP64 one only where it is positive: a quote
  // the FP64 status rule keeps (within a few ulp of a threshold) may be
  // exactly at its bound or at its intrinsic value, and then keeps the FP64
  // values it was decided with.
  const dd mK = {-K, 0.0};
  if (itm) {
    // p - theta (F - K)
    const dd fk = dd_add(F, mK);
    const dd num = dd_add(p, flag > 0 ? dd{-fk.hi, -fk.lo} : fk);
    const double b = __dmul_rn(num.hi + num.lo, inv_sqrt_fk);
    if (b > 0.0) beta_otm = b;
  }
  // bound - p
  const dd bound = flag > 0 ? F : dd{K, 0.0};
  const dd cnum = dd_add(bound, dd{-p.hi, -p.lo});
  const double c = __dmul_rn(cnum.hi + cnum.lo, inv_sqrt_fk);
  if (c > 0.0) c_beta = c;
}
// the same as a call: kernels whose registers are tight keep the call's
// spills out of their hot loop
static __device__ __noinline__ void refine_reduced(int model, double P, double SF, double K, double T,
                                            double r, double q, int flag, bool itm,
                                            double& beta_otm, double& c_beta) {
  refine_reduced_inline(model, P, SF, K, T, r, q, flag, itm, beta_otm, c_beta);
}

// decide, then the refinement where the quote needs it (INLINE: in the
// kernel's own code instead of a call)
template <bool INLINE = false>
__device__ __forceinline__ void refine_if_needed(int model, double P, double SF, double K,
                                                 double T, double r, double q, int flag, Norm& n) {
  if (needs_refine(n)) {
    if (INLINE)
      refine_reduced_inline(model, P, SF, K, T, r, q, flag, n.iota > 0.0, n.beta_otm, n.c_beta);
    else
      refine_reduced(model, P, SF, K, T, r, q, flag, n.iota > 0.0, n.beta_otm, n.c_beta);
  }
}

// ---------------------------------------------------------------------------
// normalised Black function
// ---------------------------------------------------------------------------
template <typename T>
struct NB {
  T e;      // exp(-(h^2+t^2)/2)
  T B;      // b/e (or (b_max - b)/e for the complement)
  T b;      // b itself (value mode of nb_eval only)
  T h, t, inv_s;
};

// Odd part of R(h+t) - R(h-t) divided by 2: sum_k R^{(2k+1)}(h) t^{2k+1}/(2k+1)!
// with R^{(n)} = P_n(h) + Q_n(h) R.  P_{2k+1} is even in h, Q_{2k+1} odd; the
// coefficients below are P_{2k+1}(h) and Q_{2k+1}(h)/h as polynomials in h^2,
// each divided by (2k+1)!.
template <typename T>
__device__ __forceinline__ T small_t_series(T h, T t, T R) {
  const T u = h * h, w = t * t;
  // k = 0: P1 = 1, Q1/h = 1
  // k = 1: P3 = 2 + u, Q3/h = 3 + u                       (/3!)
  // k = 2: P5 = 8 + 9u + u^2, Q5/h = 15 + 10u + u^2       (/5!)
  // k = 3: P7 = 48 + 87u + 20u^2 + u^3,
  //        Q7/h = 105 + 105u + 21u^2 + u^3                (/7!)
  // k = 4: P9 = 384 + 975u + 345u^2 + 35u^3 + u^4,
  //        Q9/h = 945 + 1260u + 378u^2 + 36u^3 + u^4      (/9!)
  // k = 5: P11 = 3840 + 12645u + 6090u^2 + 938u^3 + 54u^4 + u^5,
  //        Q11/h = 10395 + 17325u + 6930u^2 + 990u^3 + 55u^4 + u^5   (/11!)
  const T p1 = T(1), q1 = T(1);
  const T p3 = (T(2) + u) * T(1.0 / 6.0), q3 = (T(3) + u) * T(1.0 / 6.0);
  const T p5 = (T(8) + u * (T(9) + u)) * T(1.0 / 120.0);
  const T q5 = (T(15) + u * (T(10) + u)) * T(1.0 / 120.0);
  const T p7 = (T(48) + u * (T(87) + u * (T(20) + u))) * T(1.0 / 5040.0);
  const T q7 = (T(105) + u * (T(105) + u * (T(21) + u))) * T(1.0 / 5040.0);
  T A, C;
  if (Prec<T>::terms >= 6) {
    const T p9 = (T(384) + u * (T(975) + u * (T(345) + u * (T(35) + u)))) * T(1.0 / 362880.0);
    const T q9 = (T(945) + u * (T(1260) + u * (T(378) + u * (T(36) + u)))) * T(1.0 / 362880.0);
    const T p11 = (T(3840) + u * (T(12645) + u * (T(6090) + u * (T(938) + u * (T(54) + u))))) *
                  T(1.0 / 39916800.0);
    const T q11 = (T(10395) + u * (T(17325) + u * (T(6930) + u * (T(990) + u * (T(55) + u))))) *
                  T(1.0 / 39916800.0);
    A = p1 + w * (p3 + w * (p5 + w * (p7 + w * (p9 + w * p11))));
    C = q1 + w * (q3 + w * (q5 + w * (q7 + w * (q9 + w * q11))));
  } else {
    A = p1 + w * (p3 + w * (p5 + w * p7));
    C = q1 + w * (q3 + w * (q5 + w * q7));
  }
  return t * (A + h * R * C);
}

// b(x, s) for x <= 0 (or its complement b_max - b when comp), scaled by e.
// with_e = false leaves o.e unset: the wing objectives use only B and ln b.
//
// Value mode (with_e, a bound bmax = e^{x/2} >= 0 passed in, not comp): o.b
// is b itself.  Past the inflection point (h + t > 0) the erfcx form would
// reflect a negative argument, erfcx(-a) = 2 exp(a^2) - erfcx(a), at the cost
// of one more exponential; but e exp((h+t)^2/2) = e^{ht} = e^{x/2} = b_max, so
// there b = b_max - e [erfcx((h+t)/sqrt2) + erfcx((t-h)/sqrt2)]/2 instead,
// with the same error relative to b_max and no exponential (o.B then holds
// the complement, (b_max - b)/e).
//
// log_space: the caller's objective is ln b (the lowest region).  B's
// relative error is then an absolute error of ln b, which moves s by that
// error over s (ln b)' ~ h^2.  For small t the erfcx difference loses a factor
// ~|h|/(2t) = |x|/s^2 to cancellation, so its effect on s is ~eps/|x|: within
// an ulp for |x| >= 1, where the two erfcx evaluations replace the small-t
// series (while |x|/s^2 < 1e12 leaves the difference four digits or more).
// t < t_small and b_max >= 0 (b_max < 0 means no bound was passed), for
// t, b_max of either type; the FP64 forms test the bits
__device__ __forceinline__ bool small_t(double t) { return __double2hiint(t) < 0x3fb9999a; }  // 0.1
__device__ __forceinline__ bool small_t(float t) { return t < Prec<float>::t_small; }
// small_t with a preferred side near the threshold.  Over 0.09 <= t < 0.11
// both forms are accurate (the series' truncation grows as t^12, 3x at 0.11;
// the erfcx difference's cancellation as 1/t, 1.1x at 0.09), so there a quote
// keeps the side its guess took (pref = 1: series, 0: erfcx; pref < 0: no
// preference).  The binned solvers sort a tile's quotes by that side, and
// the lanes of a warp then stay on one branch while their iterations cross
// t_small instead of running both.
__device__ __forceinline__ bool small_t_pref(double t, int pref) {
  const int hi = __double2hiint(t);
  if (pref >= 0 && hi >= 0x3fb70a3d && hi < 0x3fbc28f5) return pref != 0;  // [0.09, 0.11)
  return hi < 0x3fb9999a;
}
__device__ __forceinline__ bool small_t_pref(float t, int) { return small_t(t); }
__device__ __forceinline__ bool has_bound(double b) { return __double2hiint(b) >= 0; }
__device__ __forceinline__ bool has_bound(float b) { return b >= 0.0f; }
__device__ __forceinline__ bool positive(double v) { return positive64(v); }
__device__ __forceinline__ bool positive(float v) { return v > 0.0f; }
__device__ __forceinline__ double recip(double s) { return recip64(s); }
__device__ __forceinline__ float recip(float s) { return 1.0f / s; }

template <typename T>
__device__ __forceinline__ bool series_in_log_space(T x, T s) {
  return !(x <= T(-1) && -x < T(1e12) * s * s);
}

//
// kIntHalf: the exact halvings on the exponent field (integer operations,
// FP64 issue slots saved) or as multiplications by 1/2 (fewer instructions:
// faster in the divergent Halley kernels, which are bound by issue rather than
// by the FP64 pipe); the values are the same.
template <typename T, bool kIntHalf = true>
__device__ __forceinline__ T halved(T v) {
  if constexpr (kIntHalf) return f_half(v);
  return T(0.5) * v;
}

// R(z) ~ 1/|z| - 1/|z|^3 for z -> -inf: with a = |h|, D = a^2 - t^2,
// [R(h+t) - R(h-t)]/2 = (t/D) (1 - (3a^2 + t^2)/D^2) + O(t/a^6), times
// sqrt(2/pi); the FP64 form out of line (|h| > 1e6: rare)
template <typename T>
__device__ __forceinline__ T series_asymptote_inline(T h, T t) {
  const T D = h * h - t * t;
  return T(kSqrt2OverPi) * (t / D) * (T(1) - (T(3) * h * h + t * t) / (D * D));
}
static __device__ __noinline__ double series_asymptote(double h, double t) {
  return series_asymptote_inline<double>(h, t);
}
__device__ __forceinline__ float series_asymptote(float h, float t) {
  return series_asymptote_inline<float>(h, t);
}

template <typename T, bool kIntHalf = true>
__device__ __forceinline__ void nb_eval(T x, T s, bool comp, NB<T>& o, bool with_e,
                                        T bmax = T(-1), bool log_space = false, int pref = -1) {
  o.inv_s = recip(s);
  o.h = x * o.inv_s;
  o.t = halved<T, kIntHalf>(s);
  const T h = o.h, t = o.t;
  o.e = with_e ? f_exp(-halved<T, kIntHalf>(h * h + t * t)) : T(0);
  const bool small = small_t_pref(t, pref) && !comp && (!log_space || series_in_log_space(x, s));
  const bool via_comp = with_e && !comp && !small && has_bound(bmax) && positive(h + t);
  // erfcx of w/sqrt2 with w = -h, h + t or -(h + t)
  const T w1 = small ? -h : ((comp || via_comp) ? (h + t) : -(h + t));
  const T Y1 = f_erfcx_w(w1);
  if (small) {
    if (f_abs(h) < Prec<T>::h_asym) {
      o.B = T(kSqrt2OverPi) * small_t_series<T>(h, t, T(kSqrtPiOver2) * Y1);
    } else {
      o.B = series_asymptote(h, t);
    }
  } else {
    const T Y2 = f_erfcx_w(t - h);
    o.B = halved<T, kIntHalf>((comp || via_comp) ? Y1 + Y2 : Y1 - Y2);
  }
  o.b = via_comp ? bmax - o.e * o.B : o.e * o.B;
}

// ln of the value nb_eval describes
template <typename T, bool kIntHalf = true>
__device__ __forceinline__ T nb_log(const NB<T>& v) {
  return f_log(v.B) - halved<T, kIntHalf>(v.h * v.h + v.t * v.t);
}

// full normalised Black b(x, s, theta) for any x, s >= 0 (FP64)
__device__ __forceinline__ double normalised_black(double x, double s, int theta) {
  double E;
  const double Em = exp_expm1_64(-half64(fabs(x)), E);  // e^{-|x|/2}, its expm1
  double iota = 0.0;
  const long long bx = __double_as_longlong(x);  // theta x > 0 on the sign bits
  if (theta > 0 ? bx > 0 : (bx < 0 && bx != (long long)0x8000000000000000ULL))
    iota = div64(-E * (1.0 + Em), Em);
  if (!(s > 0.0)) return iota;
  NB<double> v;
  nb_eval<double>(-fabs(x), s, false, v, true, Em);
  return iota + v.b;
}

// ---------------------------------------------------------------------------
// "Let's Be Rational" (Section 2.2): boundaries, guess, objective, HH(3)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T hermite_guess(T beta, T b0, T b1, T s0, T s1, T d0, T d1) {
  const T db = b1 - b0;
  if (!(db > T(0))) return T(0.5) * (s0 + s1);
  const T tau = (beta - b0) / db, tau2 = tau * tau, tau3 = tau2 * tau;
  const T h00 = T(2) * tau3 - T(3) * tau2 + T(1), h10 = tau3 - T(2) * tau2 + tau;
  const T h01 = T(-2) * tau3 + T(3) * tau2, h11 = tau3 - tau2;
  return h00 * s0 + h10 * db * d0 + h01 * s1 + h11 * db * d1;
}

// inverse normal CDF of p = e^{ln_p} (p < 1/2), with the tail asymptote
// z^2 = L - ln(L) - ln(2 pi), L = -2 ln p, where p underflows the type.
template <typename T>
__device__ __forceinline__ T ncdfinv_log(T ln_p) {
  if (ln_p > Prec<T>::ln_p_floor) return f_ncdfinv(f_exp(ln_p));
  const T L = T(-2) * ln_p;
  return -f_sqrt(L - f_log(L) - T(kLn2Pi));
}

// Quantities the solver needs besides (beta, x): ln beta and b_max - beta
// (both from FP64 when T is float), and b_max = e^{x/2}.
template <typename T>
struct Reduced {
  T beta, c_beta, x, bmax;
  // ln beta: 0 until computed (beta < 1 after the reduction, so 0 is free);
  // preset from log(P) for prices near the bottom of the FP64 range
  T ln_beta;
  T inv_ln_beta, ln_c_beta;  // 1/ln beta (lowest region), ln(b_max - beta) (highest)
};

// The logarithms only the wing objectives need, for the region the guess chose.
template <typename T>
__device__ __forceinline__ void wing_logs(Reduced<T>& q, int reg) {
  if (reg == 0) {
    if (q.ln_beta == T(0)) q.ln_beta = f_log(q.beta);
    q.inv_ln_beta = T(1) / q.ln_beta;
  } else if (reg == 3) {
    q.ln_c_beta = f_log(q.c_beta);
  }
}

template <typename T>
struct Objective {
  T nu, h2, h3;  // -g/g', g''/g', g'''/g'
};

// Householder(3) ingredients for the three-branch objective of Section 2.2:
//   region 0 (lowest):        g = 1/ln b - 1/ln beta
//   regions 1, 2 (middle):    g = b - beta
//   region 3 (highest):       g = ln((b_max - beta)/(b_max - b))
template <typename T>
__device__ __forceinline__ Objective<T> objective(const Reduced<T>& q, T s, int reg) {
  NB<T> v;
  nb_eval<T>(q.x, s, reg == 3, v, reg == 1 || reg == 2, q.bmax);
  const T hh = v.h * v.h;
  const T u = hh * v.inv_s - T(0.25) * s;                    // b''/b'
  const T du = T(-3) * hh * v.inv_s * v.inv_s - T(0.25);     // d(b''/b')/ds
  Objective<T> o;
  if (reg == 1 || reg == 2) {
    const T bp = v.e * T(kInvSqrt2Pi);
    o.nu = (q.beta - v.b) / bp;
    o.h2 = u;
    o.h3 = u * u + du;
  } else {
    const T lnX = nb_log(v);
    const T qw = T(kInvSqrt2Pi) / v.B;  // b'/b (region 0) or b'/(b_max - b) (region 3)
    if (reg == 0) {
      const T iL = T(1) / lnX, k1 = T(1) + T(2) * iL;
      const T g = iL - q.inv_ln_beta;
      o.nu = g * lnX * lnX / qw;
      o.h2 = u - qw * k1;
      o.h3 = o.h2 * o.h2 + du - (qw * u - qw * qw) * k1 + T(2) * qw * qw * iL * iL;
    } else {
      const T g = q.ln_c_beta - lnX;
      o.nu = -g / qw;
      o.h2 = u + qw;
      o.h3 = o.h2 * o.h2 + du + qw * o.h2;
    }
  }
  return o;
}

// 1/e for the Newton step nu = (beta - b) sqrt(2 pi)/e: the FP32 reciprocal
// and one Newton step, relative error ~1e-14, which only scales the step
// (the next iteration, or nu -> 0 at the root, makes it invisible); e below
// 1e-30 takes the division
__device__ __forceinline__ double inv_e(double e) {
  if (__double2hiint(e) <= 0x39b4484b) return 1.0 / e;  // e >= 0
  const double r = f64_of(__frcp_rn(f32_trunc(e)));
  return fma(r, fma(-e, r, 1.0), r);
}

template <typename T>
__device__ __forceinline__ T hh3_step(const Objective<T>& o) {
  const T ds = o.nu * (T(1) + T(0.5) * o.h2 * o.nu) / (T(1) + o.nu * (o.h2 + o.h3 * o.nu / T(6)));
  return f_finite(ds) ? ds : o.nu;
}

// |ds| > tol s; for FP64 with tol a power of two and s >= 2^-960 (every
// solver's case) on the patterns: tol s is s with tol's exponent added
__device__ __forceinline__ bool moved_more(float ds, float s, float tol) {
  return fabsf(ds) > tol * s;
}
__device__ __forceinline__ bool moved_more(double ds, double s, double tol) {
  const long long bt = __double_as_longlong(tol), bs = __double_as_longlong(s);
  if ((bt & 0xfffffffffffffLL) != 0 || bs < (64LL << 52) || bt <= 0) return fabs(ds) > tol * s;
  const long long lim = bs + (bt - (1023LL << 52));  // pattern of tol * s
  return (__double_as_longlong(ds) & 0x7fffffffffffffffLL) > lim;
}

template <typename T>
__device__ __forceinline__ T guarded(T s, T ds) {
  return (s + ds <= T(0.25) * s) ? T(0.25) * s : s + ds;
}
// FP64: s > 0, so s/4 is the pattern of s less two in the exponent field
// (for s >= 2^-1018) and s + ds <= s/4 is the signed order of the patterns
// (a zero or negative s + ds compares as the FP64 test would; the FP64
// Householder step is finite)
template <>
__device__ __forceinline__ double guarded<double>(double s, double ds) {
  const long long bs = __double_as_longlong(s);
  if (bs < (5LL << 52)) return (s + ds <= 0.25 * s) ? 0.25 * s : s + ds;
  const double sn = s + ds;
  const long long bq = bs - (2LL << 52);
  return __double_as_longlong(sn) <= bq ? __longlong_as_double(bq) : sn;
}

// One Householder(3) step whose residual g and first derivative g' are FP64
// and whose second-order ratios h2 = g''/g', h3 = g'''/g' are FP32: they only
// shape the correction factor (1 + phi) of the Newton step nu, with
// phi = nu (-h2/2 - h3 nu/6) / (1 + nu (h2 + h3 nu/6)) = O(nu), so their
// relative error enters the step at order nu^2.  Returns the step ds (0 where
// it is not finite); the FP64 solver iterates it, the mixed solver applies it
// once after its FP32 iterations.
__device__ __forceinline__ double hh3_ds_mixed(const Reduced<double>& q, double s, int reg,
                                               double* nu_out = nullptr, int pref = -1) {
  NB<double> v;
  nb_eval<double>(q.x, s, reg == 3, v, reg == 1 || reg == 2, q.bmax, reg == 0, pref);
  const float hf = f32_trunc(v.h), sf = f32_trunc(s);
  const float hh = hf * hf, is = __frcp_rn(sf);
  const float u = hh * is - 0.25f * sf;
  const float du = -3.0f * hh * is * is - 0.25f;
  double nu;
  float h2, h3;
  if (reg == 1 || reg == 2) {
    nu = (q.beta - v.b) * (kSqrt2Pi * inv_e(v.e));
    h2 = u;
    h3 = u * u + du;
  } else {
    const double lnX = nb_log(v);
    // b/b' (region 0) or (b_max - b)/b' (region 3): B sqrt(2 pi), no division
    const double bq = v.B * kSqrt2Pi;
    const float qf = 1.0f / f32_trunc(bq);
    if (reg == 0) {
      // g = 1/ln b - 1/ln beta = (ln beta - ln b) / (ln b ln beta): the
      // residual as a difference of logarithms, no FP64 division
      nu = (q.ln_beta - lnX) * lnX * q.inv_ln_beta * bq;
      const float iLf = 1.0f / f32_trunc(lnX), k1 = 1.0f + 2.0f * iLf;
      h2 = u - qf * k1;
      h3 = h2 * h2 + du - (qf * u - qf * qf) * k1 + 2.0f * qf * qf * iLf * iLf;
    } else {
      nu = -(q.ln_c_beta - lnX) * bq;
      h2 = u + qf;
      h3 = h2 * h2 + du + qf * h2;
    }
  }
  if (nu_out) *nu_out = nu;
  const float nf = f32_trunc(nu);
  const float phi = nf * (-0.5f * h2 - h3 * nf * (1.0f / 6.0f)) / (1.0f + nf * (h2 + h3 * nf * (1.0f / 6.0f)));
  const double ds = isfinite(phi) ? fma(nu, f64_of(phi), nu) : nu;
  return bits_finite(ds) ? ds : 0.0;
}

__device__ __forceinline__ double hh3_correction(Reduced<double> q, double s, int reg) {
  wing_logs<double>(q, reg);
  return guarded<double>(s, hh3_ds_mixed(q, s, reg));
}

// The mixed solver's correction of its FP32 iterate s32 and sigma = s/sqrt(T):
// the Householder(3) step with the residual in double-float
// (fvdf::hh3_correction_df) where the quote's scales fit FP32's exponent
// range, else the FP64 step above.
// The FP64 step is out of line: it is rare here, and its code would otherwise
// sit in the hot loop's instruction stream.
static __device__ __noinline__ double mixed_sigma_fp64(Reduced<double> q, float s32, int reg, double T) {
  return hh3_correction(q, f64_of(s32), reg) * rsqrt(T);
}
__device__ __forceinline__ double mixed_sigma(const Reduced<double>& q, float s32, int reg, double T) {
  double sigma;
  if (fvdf::hh3_correction_df(q.beta, q.c_beta, q.x, q.ln_beta, T, s32, reg, sigma)) return sigma;
  return mixed_sigma_fp64(q, s32, reg, T);
}

// Boundaries (six normalised-Black values: b and b' at s_l, s_c, s_h, of which
// b' at s_c is closed form and only the side of s_c that beta falls on is
// evaluated), the four-region initial guess, and the region index.
template <typename T>
__device__ __forceinline__ T lbr_guess(Reduced<T>& q, int& reg) {
  const T x = q.x, beta = q.beta, bmax = q.bmax;
  const bool xneg = x < T(0);
  // inflection point s_c = sqrt(2|x|): there h + t = 0, h^2 + t^2 = |x|, so
  // e = e^{x/2} = b_max, erfcx(-(h+t)/sqrt2) = 1 and b'(s_c) = b_max/sqrt(2 pi);
  // the erfcx form reduces to b_c = b_max (1 - erfcx(sqrt|x|)) / 2
  const T sc = xneg ? f_sqrt(T(-2) * x) : T(0);
  T bc = T(0);
  if (xneg) {
    if (T(0.5) * sc < Prec<T>::t_small) {
      NB<T> vc_;
      nb_eval<T>(x, sc, false, vc_, true);
      bc = vc_.e * vc_.B;
    } else {
      bc = T(0.5) * bmax * (T(1) - f_erfcx(f_sqrt(-x)));
    }
  }
  const T vc = bmax * T(kInvSqrt2Pi);
  // tangent at s_c meets 0 at s_l and b_max at s_h; beta picks one side
  const bool lower = beta <= bc;
  T so = lower ? sc - bc / vc : sc + (bmax - bc) / vc;
  const bool degenerate = !(so > T(0));  // s_l lost to rounding next to x = 0
  if (degenerate) so = sc > T(0) ? sc : T(1);
  NB<T> vo_;
  nb_eval<T>(x, so, false, vo_, true, bmax);
  const T bo = degenerate ? T(0) : vo_.b;
  const T vo = vo_.e * T(kInvSqrt2Pi);
  // ln b_l, for the region test where b_l underflows the type and for the
  // lowest-region guess: an FP32 value is enough for both (a wrong side next
  // to b_l only changes which convergent objective is used)
  const float ln_bo = (lower && !degenerate)
                          ? (float)(T(-0.5) * (vo_.h * vo_.h + vo_.t * vo_.t)) + logf((float)vo_.B)
                          : 0.0f;
  if (lower) {
    if (degenerate) {
      reg = 1;
    } else if (bo > T(0)) {
      reg = beta < bo ? 0 : 1;
    } else {
      if (q.ln_beta == T(0)) q.ln_beta = f_log(beta);
      reg = (float)q.ln_beta < ln_bo ? 0 : 1;
    }
  } else {
    reg = (beta <= bo) ? 2 : 3;
  }
  T s;
  if (reg == 1 || reg == 2) {
    // cubic Hermite of s(beta) with slopes 1/b' on the inflection-bounded interior
    T b0, b1, s0, s1, d0, d1;
    if (reg == 1) {
      b0 = bo; b1 = bc; s0 = degenerate ? T(0) : so; s1 = sc;
      d1 = T(1) / vc;
      d0 = degenerate ? sc / bc : T(1) / vo;
      if (degenerate) d1 = d0;
    } else {
      b0 = bc; b1 = bo; s0 = sc; s1 = so;
      d0 = T(1) / vc;
      d1 = T(1) / vo;
    }
    s = hermite_guess(beta, b0, b1, s0, s1, d0, d1);
  } else {
    // wings: invert the limiting form, scaled to match b at the boundary
    //   lowest:  b ~ c Phi(-|x|/(sqrt3 s))^3   (s -> 0)
    //   highest: b_max - b ~ c' Phi(-s/2)       (s -> inf)
    // The limiting forms hold to ~1e-2 in s, so the inversion runs in FP32
    // whatever T is, with ln Phi(z) = ln(erfcx(-z/sqrt2)/2) - z^2/2 (z < 0),
    // which neither underflows nor cancels.
    if (reg == 0 && q.ln_beta == T(0)) q.ln_beta = f_log(beta);
    const float za = (reg == 0) ? -fabsf((float)x) * float(kInvSqrt3) / (float)so
                                : -0.5f * (float)so;
    const float ln_pa = logf(0.5f * erfcxf(-za * float(kInvSqrt2))) - 0.5f * za * za;
    const float ln_p = (reg == 0) ? ln_pa + ((float)q.ln_beta - ln_bo) * (1.0f / 3.0f)
                                  : ln_pa + logf((float)(q.c_beta / (bmax - bo)));
    const float z = ncdfinv_log<float>(ln_p);
    s = (reg == 0) ? f_abs(x) * T(kInvSqrt3) / T(fabsf(z)) : T(-2) * T(z);
  }
  if (!(s > T(0)) || !f_finite(s)) s = (so > T(0)) ? so : T(1);
  return s;
}

// LBR iterations from the guess s of region reg: n_min Householder(3) steps,
// then up to n_max while the last step still moved s by more than conv_tol
// relative.  pref: the small-t side near the threshold (small_t_pref).
template <typename T>
__device__ __forceinline__ T lbr_iterate(Reduced<T> q, T s, int reg, int n_min, int n_max,
                                         T conv_tol, int pref = -1) {
  wing_logs<T>(q, reg);
  for (int k = 0; k < n_max; k++) {
    // FP64: residual and Newton step in FP64, second-order ratios in FP32
    T ds;
    if constexpr (std::is_same<T, double>::value)
      ds = hh3_ds_mixed(q, s, reg, nullptr, pref);
    else
      ds = hh3_step<T>(objective<T>(q, s, reg));
    s = guarded<T>(s, ds);
    if (k + 1 >= n_min && !moved_more(ds, s, conv_tol)) break;
  }
  return s;
}

// LBR solve: guess, then the iterations
template <typename T>
__device__ __forceinline__ T lbr_solve(Reduced<T> q, int n_min, int n_max, T conv_tol, int& reg) {
  const T s = lbr_guess<T>(q, reg);
  return lbr_iterate<T>(q, s, reg, n_min, n_max, conv_tol);
}

__device__ __forceinline__ Reduced<double> reduced64(const Norm& n) {
  Reduced<double> q;
  q.beta = n.beta_otm;
  // out of the money, beta_otm = beta and the logarithm of P applies
  q.ln_beta = (n.ln_beta != 0.0 && n.beta_otm == n.beta) ? n.ln_beta : 0.0;
  q.c_beta = n.c_beta;
  q.x = n.x_otm;
  q.bmax = n.bmax;
  q.inv_ln_beta = 0.0;
  q.ln_c_beta = 0.0;
  return q;
}

__device__ __forceinline__ Reduced<float> reduced32(const Reduced<double>& q) {
  Reduced<float> f;
  f.beta = f32_trunc(q.beta);
  // below FP32's normal range ln beta comes from FP64 (the FP32 solve works
  // in log space there); above it logf of the FP32 beta is accurate enough
  f.ln_beta = q.ln_beta != 0.0 ? (float)q.ln_beta
                               : (__double2hiint(q.beta) < 0x3841039d ? (float)log(q.beta) : 0.0f);  // beta < 1e-37
  f.c_beta = f32_trunc(q.c_beta);
  f.x = f32_trunc(q.x);
  f.bmax = f32_trunc(q.bmax);
  f.inv_ln_beta = 0.0f;
  f.ln_c_beta = 0.0f;
  return f;
}

// The FP64 solver: two FP64 Householder(3) iterations (a third where the
// second still moved s by more than 2^-17) from the FP32 guess g of region
// reg.  The guess only seeds the iterations and is itself ~1e-2 off, so FP32
// rounding there changes nothing the iterations can see; where FP32 cannot
// hold the quote's scales (b_max below 1e-20, a guess outside 1e-30..1e30)
// the FP64 guess is taken instead.
__device__ __forceinline__ double lbr_solve64(const Reduced<double>& q, float g, int reg) {
  // near t_small the iterations keep the guess's side (the side the binned
  // tiles sort by)
  if (q.bmax > 1e-20 && g > 1e-30f && g < 1e30f)
    return lbr_iterate<double>(q, f64_of(g), reg, 2, 3, 0x1p-17,
                               0.5f * g < (float)Prec<double>::t_small ? 1 : 0);
  int reg64 = 1;
  return lbr_solve<double>(q, 2, 3, 0x1p-17, reg64);
}

// ---------------------------------------------------------------------------
// Halley x8 + fallback (Section 2.2, second item), FP64
// ---------------------------------------------------------------------------
constexpr int kHalleySteps = 8;
constexpr double kHalleyConvTol = 1e-10;
// The convergence test reads the relative Newton distance of the last sweep
// (at s_7).  Halley's iteration converges cubically, so from a distance d_k
// at sweep k it can reach the tolerance by then only if
// d_k <= kHalleyConvTol^(3^-(7-k)); a quote beyond that bound at a sweep
// k >= first_check goes to the fallback at once instead of spending the
// sweeps left (the fallback returns the same root; a quote the bound sends
// there too early only trades its remaining sweeps for the fallback's two or
// three evaluations).  The test starts at sweep first_check: 0 for large
// batches (on the 16.8 M BSM grid most quotes start far from the root, and
// leaving after the first evaluation instead of the second took the kernel
// from 25.3 to 19.9 ms), 1 for small latency-bound ones (75.9 against 80.0 us
// on 4,096 Black-76 quotes).
__constant__ const double kHalleyReach[kHalleySteps] = {
    0.9895267209580416, 0.9689080827862817, 0.9095943135230796, 0.7525636023261612,
    0.4262158829015324, 0.07742636826811272, 0.0004641588833612781, 1e-10};

struct HalleyOut {
  double s, lo, hi;
  bool converged;
};

// One quote's sweeps so far: the iterate, the bracket [lo, hi], the last
// Newton distance relative to s, and whether the sweeps have ended (the root,
// the handoff test, or the last sweep).
struct HalleyState {
  double s, lo, hi, nerr;
  bool done;
};

__device__ __forceinline__ HalleyState halley_start(double beta) {
  HalleyState h;
  h.s = kSqrt2Pi * beta;  // Brenner-Subrahmanyam: b ~ s/sqrt(2 pi) at the money
  h.lo = 0.0;
  h.hi = __longlong_as_double(0x7ff0000000000000LL);
  h.nerr = h.hi;
  h.done = false;
  return h;
}

// Sweeps k0 .. k1 - 1 of the eight, from the state h.  The residual
// g = b - beta is evaluated as (b_max - beta) - (b_max - b) when
// beta > b_max/2: b_max - b then comes from the cancellation-free complement,
// so g carries an error relative to b_max - b instead of to b_max (the same
// function, with the same Halley step).  Running 0..8 at once or in pieces
// gives the same result bit for bit.
__device__ __forceinline__ void halley_sweeps(double beta, double c_beta, double x, double bmax,
                                              HalleyState& h, int k0, int k1, int first_check) {
  const bool upper = beta > 0.5 * bmax;
  for (int k = k0; k < k1; k++) {
    NB<double> v;
    nb_eval<double, false>(x, h.s, upper, v, true, bmax);
    const double g = upper ? c_beta - v.e * v.B : v.b - beta;
    if (g < 0.0) {
      h.lo = h.s;
    } else if (g > 0.0) {
      h.hi = h.s;
    } else {
      // g == 0 is the root; a NaN residual leaves the quote unconverged
      h.nerr = (g == 0.0) ? 0.0 : h.hi;
      h.done = true;
      return;
    }
    // Newton step nu = g/b' = g sqrt(2 pi)/e (e^-1 as in the Householder step)
    // and its distance to the root relative to s (the convergence test)
    const double nu = g * (kSqrt2Pi * inv_e(v.e));
    h.nerr = fabs(nu) * v.inv_s;
    if (k >= first_check && k < kHalleySteps - 1 && !(h.nerr <= kHalleyReach[k])) {
      h.done = true;
      return;
    }
    // Halley: ds = -2 g g' / (2 g'^2 - g g'') = -nu / (1 - nu u / 2), u = b''/b';
    // the factor 1 / (1 - nu u / 2) only shapes the step (its rounding enters at
    // order nu^2), so it is formed in FP32
    const float hf = f32_trunc(v.h), sf = f32_trunc(h.s);
    const float u = hf * hf * __frcp_rn(sf) - 0.25f * sf;
    const double step = -nu * f64_of(1.0f / (1.0f - 0.5f * f32_trunc(nu) * u));
    double sn = h.s + step;
    // lo <= sn <= hi, sn finite: lo, hi >= 0, so on the signed patterns
    const long long bn = __double_as_longlong(sn);
    if (!(bn >= __double_as_longlong(h.lo) && bn <= __double_as_longlong(h.hi) && bits_finite(sn)))
      sn = bits_finite(h.hi) ? 0.5 * (h.lo + h.hi) : 2.0 * h.s;
    h.s = sn;
  }
  if (k1 >= kHalleySteps) h.done = true;
}

__device__ __forceinline__ bool halley_converged(const HalleyState& h) {
  return isfinite(h.s) && h.s > 0.0 && h.nerr <= kHalleyConvTol;
}

// All eight sweeps at once
__device__ __forceinline__ HalleyOut halley_solve(double beta, double c_beta, double x,
                                                 double bmax, int first_check = 0) {
  HalleyState h = halley_start(beta);
  halley_sweeps(beta, c_beta, x, bmax, h, 0, kHalleySteps, first_check);
  HalleyOut o;
  o.s = h.s;
  o.lo = h.lo;
  o.hi = h.hi;
  o.converged = halley_converged(h);
  return o;
}

// Bisection in [lo, hi] on a residual increasing in s, each bisection replaced
// by a Newton step when that step stays in the bracket.  The residual is the
// transformed objective of the LBR wings (Section 2.2), under which Newton does
// not crawl where b is exponentially small:
//   beta <= b_max/2:  f = 1/ln beta - 1/ln b,               f' = (b'/b) / ln^2 b
//   beta >  b_max/2:  f = ln(b_max - beta) - ln(b_max - b),  f' = b'/(b_max - b)
// Without an upper end the Newton step (at least doubling s, at most x16)
// grows the bracket; without a lower end it shrinks it (at least halving, at
// most /16).  ln_beta is passed in: for subnormal-range prices it comes from
// log(P).
__device__ __forceinline__ double bisect_fallback(double ln_beta, double beta, double x,
                                                  double bmax, double lo, double hi) {
  const double eps = 2.220446049250313e-16;
  const bool upper = beta > 0.5 * bmax;
  const double ln_c_beta = upper ? log64(bmax - beta) : 0.0;
  const double inv_ln_beta = upper ? 0.0 : 1.0 / ln_beta;
  const bool has_hi = isfinite(hi);
  double s = (lo > 0.0 && has_hi) ? 0.5 * (lo + hi) : (has_hi ? 0.5 * hi : fmax(2.0 * lo, 1e-3));
  for (int it = 0; it < 400; it++) {
    NB<double> v;
    nb_eval<double, false>(x, s, upper, v, false);
    const double L = nb_log<double, false>(v);
    // 1/f' = b/b' (lower: times ln^2 b) or (b_max - b)/b' = B sqrt(2 pi): no division
    const double bq = v.B * kSqrt2Pi;
    double f, inv_fp;
    if (upper) {
      f = ln_c_beta - L;
      inv_fp = bq;
    } else {
      f = inv_ln_beta - 1.0 / L;
      inv_fp = bq * L * L;
    }
    // a NaN residual comes from b underflowing at s far below the root
    if (f > 0.0)
      hi = s;
    else if (f < 0.0 || f != f)
      lo = s;
    else
      break;
    double sn = s - f * inv_fp;
    if (!isfinite(hi))
      sn = (isfinite(sn) && sn > s) ? fmin(sn, 16.0 * s) : 2.0 * s;
    else if (!(lo > 0.0))
      sn = (isfinite(sn) && sn > 0.0 && sn < s) ? fmax(sn, s * 0.0625) : 0.5 * s;
    else if (!(sn > lo && sn < hi))
      sn = 0.5 * (lo + hi);
    const double ds = sn - s;
    s = sn;
    if (lo > 0.0 && isfinite(hi) && (fabs(ds) <= 2.0 * eps * s || hi - lo <= 4.0 * eps * hi)) break;
  }
  return s;
}

// The fallback of the Halley solver for a quote whose sweeps failed the
// convergence test (Section 2.2 sends those quotes to a bracketing fallback).
// The sweeps leave the root inside [lo, hi] (hi = +inf when no sweep landed
// above it).  The fallback starts from the LBR's four-region rational guess,
// moved into the bracket when it falls outside, and takes Householder(3)
// steps on the LBR objective of the guess's region (the transformed residuals
// under which Newton-type steps do not crawl in the wings).  A step that
// would leave the bracket is replaced by a bisection (or, without an upper
// end, by doubling s); the sign of the Newton step nu = -g/g' tells which end
// s replaces.  It stops after a Householder step, not the first, that moved s
// by at most 2^-17 relative (the LBR's criterion: with quartic convergence the
// remaining error is far below an ulp) or when the bracket has shrunk to a
// few ulp: two or three evaluations from the guess, against ~50 halvings of
// a plain bisection.
// The fallback's start: region and guess as the FP64 LBR solver takes them,
// FP32 where FP32 holds the quote's scales, FP64 otherwise
__device__ __forceinline__ double halley_fallback_guess(Reduced<double> q, int& reg) {
  reg = 1;
  Reduced<float> q32 = reduced32(q);
  int reg32 = 1;
  const float g32 = lbr_guess<float>(q32, reg32);
  if (q.bmax > 1e-20 && g32 > 1e-30f && g32 < 1e30f) {
    reg = reg32;
    return f64_of(g32);
  }
  return lbr_guess<double>(q, reg);
}

// The fallback's bracketed Householder(3) steps from the guess s of region reg
__device__ __forceinline__ double halley_fallback_steps(Reduced<double> q, double s, int reg,
                                                        double lo, double hi) {
  const bool has_hi = bits_finite(hi);
  if (!(s > lo && s < hi)) s = has_hi ? 0.5 * (lo + hi) : 2.0 * fmax(lo, 0.5 * s);
  wing_logs<double>(q, reg);
  for (int it = 0; it < 64; it++) {
    double nu;
    const double ds = hh3_ds_mixed(q, s, reg, &nu);
    // nu > 0: the root lies above s (a NaN step comes from b underflowing at
    // an s far below the root)
    if (nu > 0.0 || nu != nu)
      lo = s;
    else if (nu < 0.0)
      hi = s;
    else
      break;  // the residual vanished: s is the root
    double sn = s + ds;
    const bool inside = sn > lo && sn < hi && ds != 0.0;
    if (!inside) sn = bits_finite(hi) ? 0.5 * (lo + hi) : 2.0 * s;
    const bool done = (inside && it >= 1 && !moved_more(ds, sn, 0x1p-17)) ||
                      (bits_finite(hi) && hi - lo <= 0x1p-50 * hi);
    s = sn;
    if (done) break;
  }
  return s;
}

__device__ __forceinline__ double halley_fallback64(const Reduced<double>& q, double lo, double hi) {
  int reg;
  const double s = halley_fallback_guess(q, reg);
  return halley_fallback_steps(q, s, reg, lo, hi);
}

// ---------------------------------------------------------------------------
// Halley x8 in FP32 on the direct residual with plain Phi (the paper's
// throughput path for float32 label pipelines, Section 2.2)
// ---------------------------------------------------------------------------
constexpr float kHalley32ConvTol = 1e-5f;

// b(x, s) = e^{x/2} Phi(h+t) - e^{-x/2} Phi(h-t), x <= 0, plain FP32 CDFs;
// with `upper` the complement b_max - b = e^{x/2} Phi(-h-t) + e^{-x/2} Phi(h-t)
__device__ __forceinline__ float nb_plain32(float x, float s, float ep, float em, bool upper,
                                            float& bp, float& u) {
  const float h = x / s, t = 0.5f * s;
  bp = ep * (float)kInvSqrt2Pi * expf(-0.5f * (h + t) * (h + t));
  u = h * h / s - 0.25f * s;
  return upper ? ep * normcdff(-(h + t)) + em * normcdff(h - t)
               : ep * normcdff(h + t) - em * normcdff(h - t);
}

struct Halley32Out {
  float s, lo, hi;
  bool converged;
};

// beta and b_max - beta come from FP64; above b_max/2 the residual is
// evaluated as (b_max - beta) - (b_max - b), as in the FP64 solver
__device__ __forceinline__ Halley32Out halley32_solve(float beta, float c_beta, float x) {
  const float ep = expf(0.5f * x), em = expf(-0.5f * x);
  const bool upper = c_beta < beta;
  float s = (float)kSqrt2Pi * beta;
  float lo = 0.0f, hi = __int_as_float(0x7f800000), nerr = hi;
  for (int k = 0; k < kHalleySteps; k++) {
    float bp, u;
    const float v = nb_plain32(x, s, ep, em, upper, bp, u);
    const float g = upper ? c_beta - v : v - beta;
    if (g < 0.0f) {
      lo = s;
    } else if (g > 0.0f) {
      hi = s;
    } else {
      nerr = (g == 0.0f) ? 0.0f : hi;
      break;
    }
    nerr = fabsf(g / bp) / s;
    float sn = s - 2.0f * g / (2.0f * bp - g * u);
    if (!(sn >= lo && sn <= hi) || !isfinite(sn)) sn = isfinite(hi) ? 0.5f * (lo + hi) : 2.0f * s;
    s = sn;
  }
  Halley32Out o;
  o.s = s;
  o.lo = lo;
  o.hi = hi;
  o.converged = isfinite(s) && s > 0.0f && nerr <= kHalley32ConvTol;
  return o;
}

// FP32 bisection on the same residual, Newton steps kept inside the bracket
__device__ __forceinline__ float bisect32_fallback(float beta, float c_beta, float x, float lo,
                                                   float hi) {
  const float ep = expf(0.5f * x), em = expf(-0.5f * x);
  const bool upper = c_beta < beta;
  float bp, u;
  auto resid = [&](float s_) {
    const float v = nb_plain32(x, s_, ep, em, upper, bp, u);
    return upper ? c_beta - v : v - beta;
  };
  if (!isfinite(hi)) {
    hi = fmaxf(2.0f * lo, 1e-3f);
    for (int it = 0; it < 64 && resid(hi) <= 0.0f; it++) {
      lo = hi;
      hi *= 2.0f;
    }
  }
  float s = 0.5f * (lo + hi);
  for (int it = 0; it < 100; it++) {
    const float g = resid(s);
    if (g < 0.0f)
      lo = s;
    else if (g > 0.0f)
      hi = s;
    else
      break;
    const float sn = s - g / bp;
    const float next = (sn > lo && sn < hi) ? sn : 0.5f * (lo + hi);
    const float ds = next - s;
    s = next;
    if (fabsf(ds) <= 2.4e-7f * s || hi - lo <= 4.8e-7f * hi) break;
  }
  return s;
}

}  // namespace fvd
