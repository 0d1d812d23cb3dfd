// op_count.cpp -- the counted build of the oracle's FP64 LBR (measurement
// infrastructure, part of the oracle: only oracle/count_ops.py and the tests
// use it).
//
// lbr_steps.h is compiled twice: once over double (the plain functions), once
// over Counted, a scalar that counts every FP64 operation applied to it.  The
// counted build runs the FP64 status rule and the LBR steps of Section 2.2
// (boundaries, four-region guess, Householder(3) iterations) with the
// oracle's FP64 normalised Black, quote by quote, and reports per quote:
//   additions and subtractions, multiplications, divisions, square roots,
//   fused multiply-adds, comparisons, and calls of each elementary function
//   (exp, expm1, log, log1p, erfc, erfcx, cbrt, sinh, the inverse normal CDF).
// erfcx and the inverse normal CDF are counted as single calls: the oracle
// reaches their values by iterations (a continued fraction, Newton steps)
// that are its own slow way, not the method's work.  Negation, absolute
// value and finiteness tests are sign and bit operations and are not counted.
#include <math.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "fv_oracle.h"

namespace plain {
#define R double
#include "lbr_steps.h"
#undef R
#undef LBR_STEPS_PHASE  // the header's empty default hook
}  // namespace plain

namespace counted {

enum { OP_ADD, OP_MUL, OP_DIV, OP_SQRT, OP_FMA, OP_CMP, C_EXP, C_EXPM1, C_LOG, C_LOG1P, C_ERFC,
       C_ERFCX, C_CBRT, C_SINH, C_PHI_INV, N_COUNTS };
long long g_n[N_COUNTS];

struct Counted {
  double v;
  Counted() = default;
  Counted(double x) : v(x) {}
};
inline Counted tick(int k, double v) {
  g_n[k]++;
  return Counted(v);
}
inline Counted operator+(Counted a, Counted b) { return tick(OP_ADD, a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { return tick(OP_ADD, a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { return tick(OP_MUL, a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { return tick(OP_DIV, a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted& operator+=(Counted& a, Counted b) { return a = a + b; }
inline Counted& operator-=(Counted& a, Counted b) { return a = a - b; }
inline Counted& operator*=(Counted& a, Counted b) { return a = a * b; }
inline Counted& operator/=(Counted& a, Counted b) { return a = a / b; }
inline bool cmp(bool r) {
  g_n[OP_CMP]++;
  return r;
}
inline bool operator<(Counted a, Counted b) { return cmp(a.v < b.v); }
inline bool operator>(Counted a, Counted b) { return cmp(a.v > b.v); }
inline bool operator<=(Counted a, Counted b) { return cmp(a.v <= b.v); }
inline bool operator>=(Counted a, Counted b) { return cmp(a.v >= b.v); }
inline bool operator==(Counted a, Counted b) { return cmp(a.v == b.v); }
inline bool operator!=(Counted a, Counted b) { return cmp(a.v != b.v); }
inline Counted sqrt(Counted a) { return tick(OP_SQRT, std::sqrt(a.v)); }
inline Counted fma(Counted a, Counted b, Counted c) { return tick(OP_FMA, std::fma(a.v, b.v, c.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
inline bool isfinite(Counted a) { return std::isfinite(a.v); }
inline bool isinf(Counted a) { return std::isinf(a.v); }
inline bool isnan(Counted a) { return std::isnan(a.v); }
inline Counted exp(Counted a) { return tick(C_EXP, std::exp(a.v)); }
inline Counted expm1(Counted a) { return tick(C_EXPM1, std::expm1(a.v)); }
inline Counted log(Counted a) { return tick(C_LOG, std::log(a.v)); }
inline Counted log1p(Counted a) { return tick(C_LOG1P, std::log1p(a.v)); }
inline Counted erfc(Counted a) { return tick(C_ERFC, std::erfc(a.v)); }
inline Counted cbrt(Counted a) { return tick(C_CBRT, std::cbrt(a.v)); }
inline Counted sinh(Counted a) { return tick(C_SINH, std::sinh(a.v)); }
// single counted calls in place of the oracle's iterations
inline Counted erfcx_f64(Counted z) { return tick(C_ERFCX, plain::erfcx_f64(z.v)); }
inline Counted Phi_inv_d(Counted p) { return tick(C_PHI_INV, plain::Phi_inv_d(p.v)); }

// cumulative counts at the end of each phase of the solver: the status rule,
// the boundaries and initial guess, each Householder(3) iteration
constexpr int kMaxPhases = 16;
long long g_mark[kMaxPhases][N_COUNTS];
int g_marked;
inline void mark(int slot) {
  if (slot < kMaxPhases) {
    std::memcpy(g_mark[slot], g_n, sizeof(g_n));
    if (slot + 1 > g_marked) g_marked = slot + 1;
  }
}

#define R Counted
#define LBR_STEPS_PRIMITIVES
#define LBR_STEPS_PHASE(k) mark(1 + (k))
#include "lbr_steps.h"
#undef LBR_STEPS_PHASE
#undef LBR_STEPS_PRIMITIVES
#undef R

const nb_eval_t kFp64 = {nb_f64, nb_log_f64, nbc_f64};

}  // namespace counted

extern "C" {

// number of counts per quote (the layout of `counts`)
int oc_num_counts(void) { return counted::N_COUNTS; }

// For each quote: the status rule, then (for quotes that need a root) the
// LBR with n_iter Householder(3) steps (1 <= n_iter <= 12).  counts:
// n x (n_iter + 3) x oc_num_counts() int64, the cumulative counts after the
// status rule, after the boundaries and guess, after each iteration, and at
// the end (sigma = s / sqrt(T)); phases a quote does not reach repeat the last
// counts.  region: the LBR region (0..3) or -1 where no root was needed;
// sigma: the result (NaN unless the status is OK).  Single-threaded.
void oc_count_lbr(int model, const double* P, const double* S_or_F, const double* K,
                  const double* T, const double* r, const double* q, const int8_t* flag, int64_t n,
                  int n_iter, int64_t* counts, int8_t* region, double* sigma) {
  using namespace counted;
  if (n_iter < 1) n_iter = 1;
  if (n_iter > kMaxPhases - 3) n_iter = kMaxPhases - 3;
  const int slots = n_iter + 3;
  for (int64_t i = 0; i < n; i++) {
    std::memset(g_n, 0, sizeof(g_n));
    g_marked = 0;
    quote_f64 d;
    decide_f64(model, P[i], S_or_F[i], K[i], T[i], r[i], q ? q[i] : 0.0, flag[i], &d);
    mark(0);
    int reg = -1;
    double sg = NAN;
    if (d.status == ORC_OK) {
      sg = 0.0;
      if (d.solve) {
        const Counted s = lbr_otm(d.beta_otm, d.x_otm, n_iter, &reg, &kFp64);
        sg = (s / sqrt(Counted(T[i]))).v;
      }
    }
    for (int slot = 0; slot < slots; slot++) {
      const long long* src = slot == slots - 1 ? g_n : g_mark[slot < g_marked ? slot : g_marked - 1];
      for (int k = 0; k < N_COUNTS; k++) counts[(i * slots + slot) * N_COUNTS + k] = src[k];
    }
    region[i] = (int8_t)reg;
    sigma[i] = sg;
  }
}

}  // extern "C"
