/*
 * fv_oracle.c -- plain, slow CPU oracle for batched implied volatility.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.  It shares no
 * code with the CUDA library.  Build: gcc -O2 -ffp-contract=off (see build.py
 * beside this file).
 *
 * Notation (paper Section 2.2 "normalised Black", Section 2.4 Black-76):
 *   theta = +1 call / -1 put, D = e^{-rT}, F = forward (Black-76) or
 *   S e^{(r-q)T} (BSM; Black-Scholes is BSM with q = 0), p = P / D,
 *   x = ln(F/K), s = sigma sqrt(T), beta = p / sqrt(F K),
 *   b(x,s,theta) = theta [e^{x/2} Phi(theta(x/s+s/2)) - e^{-x/2} Phi(theta(x/s-s/2))],
 *   so that P = D sqrt(F K) b(x, sigma sqrt(T), theta).
 *
 * Three kinds of function live here:
 *   1. the definitions, evaluated in IEEE binary128 (_Float128, glibc's
 *      expf128/erfcf128/...): price, normalised Black, implied volatility as a
 *      bisected root, Greeks and the implicit-function gradient;
 *   2. the per-quote status decision, in FP64, because an integer decided by
 *      floating point must be decided in the kernel's precision;
 *   3. the two solvers of Section 2.2 written step by step in FP64 (LBR:
 *      boundaries, four-region guess, three-branch objective, Householder(3);
 *      Halley x8 + bisection fallback), taking the normalised Black value from
 *      binary128 so that only the algorithm's steps are under test.
 */
#define _GNU_SOURCE
#include "fv_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef _Float128 q128;

/* ------------------------------------------------------------------------- */
/* binary128 primitives                                                       */
/* ------------------------------------------------------------------------- */
static q128 q_rsqrt2(void) { return sqrtf128(0.5f128); }
static q128 q_inv_sqrt_2pi(void) { return 1.0f128 / sqrtf128(2.0f128 * M_PIf128); }

/* standard normal CDF, Phi(z) = erfc(-z/sqrt 2)/2 (Section 2.3: the CDF is
 * evaluated through erfc for deep out-of-the-money precision) */
static q128 Phi_q(q128 z) { return 0.5f128 * erfcf128(-z * q_rsqrt2()); }
static q128 phi_q(q128 z) { return q_inv_sqrt_2pi() * expf128(-0.5f128 * z * z); }

/* normalised Black with the two exponentials passed in (ep = e^{x/2},
 * em = e^{-x/2}); s <= 0 gives the normalised intrinsic value. */
static q128 nb_q_e(q128 x, q128 s, int th, q128 ep, q128 em) {
  if (s <= 0) {
    q128 v = (q128)th * (ep - em);
    return v > 0 ? v : 0;
  }
  q128 h = x / s, t = 0.5f128 * s;
  return (q128)th * (ep * Phi_q((q128)th * (h + t)) - em * Phi_q((q128)th * (h - t)));
}
static q128 nb_q(q128 x, q128 s, int th) {
  return nb_q_e(x, s, th, expf128(0.5f128 * x), expf128(-0.5f128 * x));
}
/* b_max - b for a call: e^{x/2} Phi(-(h+t)) + e^{-x/2} Phi(h-t); both terms
 * are positive, so the complement carries no cancellation. */
static q128 nb_compl_q(q128 x, q128 s) {
  q128 h = x / s, t = 0.5f128 * s;
  return expf128(0.5f128 * x) * Phi_q(-(h + t)) + expf128(-0.5f128 * x) * Phi_q(h - t);
}

/* ------------------------------------------------------------------------- */
/* threading                                                                  */
/* ------------------------------------------------------------------------- */
typedef void (*range_fn)(void* ctx, int64_t i0, int64_t i1);
typedef struct {
  range_fn fn;
  void* ctx;
  int64_t i0, i1;
} job_t;
static void* job_run(void* a) {
  job_t* j = (job_t*)a;
  j->fn(j->ctx, j->i0, j->i1);
  return NULL;
}
int or_num_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}
static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
  if (n <= 0) return;
  if (nthreads <= 0) nthreads = or_num_threads();
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = (int)n;
  if (nthreads == 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t th[256];
  job_t jobs[256];
  for (int k = 0; k < nthreads; k++) {
    jobs[k].fn = fn;
    jobs[k].ctx = ctx;
    jobs[k].i0 = n * k / nthreads;
    jobs[k].i1 = n * (k + 1) / nthreads;
    pthread_create(&th[k], NULL, job_run, &jobs[k]);
  }
  for (int k = 0; k < nthreads; k++) pthread_join(th[k], NULL);
}

/* b(x,s) for the call, x <= 0, from binary128 rounded to FP64 */
static double nb_d(double x, double s) { return (double)nb_q((q128)x, (q128)s, 1); }
/* ln b(x,s) and b'/b for the call, from binary128 (no FP64 underflow in the
 * lowest wing, where the objective works with ln b) */
static void nb_log_d(double x, double s, double* L, double* qb) {
  const q128 b = nb_q((q128)x, (q128)s, 1);
  const q128 h = (q128)x / (q128)s, t = 0.5f128 * (q128)s;
  const q128 bp = q_inv_sqrt_2pi() * expf128(-0.5f128 * (h * h + t * t));
  *L = (double)logf128(b);
  *qb = (double)(bp / b);
}
static double nbc_d(double x, double s) { return (double)nb_compl_q((q128)x, (q128)s); }

/* The FP64 status rule, the oracle's FP64 normalised Black and the LBR steps
 * (shared with the counted build). */
#include "lbr_steps.h"

static const nb_eval_t NB_BINARY128 = {nb_d, nb_log_d, nbc_d};
static const nb_eval_t NB_FP64 = {nb_f64, nb_log_f64, nbc_f64};

/* ------------------------------------------------------------------------- */
/* binary128 normalisation (exact inputs -> x, beta) for the definitions      */
/* ------------------------------------------------------------------------- */
static void normalise_q(int model, double P, double SF, double K, double T, double r, double q,
                        q128* x, q128* beta) {
  q128 qq = (model == ORC_BSM) ? (q128)q : 0;
  if (model == ORC_BLACK76) {
    *x = logf128((q128)SF / (q128)K);
    *beta = (q128)P * expf128((q128)r * (q128)T) / sqrtf128((q128)SF * (q128)K);
  } else {
    *x = logf128((q128)SF / (q128)K) + ((q128)r - qq) * (q128)T;
    *beta = (q128)P * expf128(0.5f128 * ((q128)r + qq) * (q128)T) / sqrtf128((q128)SF * (q128)K);
  }
}

/* ------------------------------------------------------------------------- */
/* Definition: sigma with b(x_otm, s) = beta_otm, by bisection in binary128.  */
/* ------------------------------------------------------------------------- */
static q128 solve_definition_q(q128 beta, q128 x) {
  /* b(x, .) rises strictly from 0 to e^{x/2} (x <= 0); beta lies strictly in
   * between.  Bracket by doubling / halving, then bisect to 2^-80 relative. */
  const q128 ep = expf128(0.5f128 * x), em = expf128(-0.5f128 * x);
  if (!(beta > 0)) return 0;
  if (!(beta < ep)) return (q128)INFINITY;
  q128 hi = x < 0 ? sqrtf128(-2.0f128 * x) : 1.0f128;
  int guard = 0;
  while (nb_q_e(x, hi, 1, ep, em) <= beta) {
    hi *= 2;
    if (++guard > 4000) return (q128)INFINITY;
  }
  q128 lo = 0.5f128 * hi;
  guard = 0;
  while (nb_q_e(x, lo, 1, ep, em) >= beta) {
    hi = lo;
    lo *= 0.5f128;
    if (++guard > 4000) return 0;
  }
  const q128 tol = 0x1p-80f128;
  for (int it = 0; it < 400 && (hi - lo) > tol * hi; it++) {
    q128 mid = 0.5f128 * (lo + hi);
    if (nb_q_e(x, mid, 1, ep, em) < beta)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5f128 * (lo + hi);
}

/* ------------------------------------------------------------------------- */
/* exported: normalised Black, price, status                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  int model;
  const double *P, *SF, *K, *T, *r, *q, *sigma, *x, *s, *grad;
  const int8_t* flag;
  const uint8_t* status_in;
  double *out, *out2, *out3, *out4, *out5, *out6;
  uint8_t* status;
  int8_t* region;
  int n_iter;
  const nb_eval_t* ev;
} ctx_t;

static void nb_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++)
    c->out[i] = (double)nb_q((q128)c->x[i], (q128)c->s[i], c->flag[i] >= 0 ? 1 : -1);
}
void or_normalised_black(const double* x, const double* s, const int8_t* theta, int64_t n,
                         double* out, int nthreads) {
  ctx_t c = {0};
  c.x = x;
  c.s = s;
  c.flag = theta;
  c.out = out;
  parallel_for(n, nthreads, nb_range, &c);
}

/* erfcx in binary128: exp(z^2) erfc(z) directly while erfc(z) stays in the
 * binary128 range (z < 100, erfc ~ 1e-4345); beyond, the asymptotic series
 * 1/(z sqrt(pi)) sum_k (-1)^k (2k-1)!! / (2 z^2)^k, whose terms fall below
 * 1e-34 by k = 10 there.  Below zero: 2 exp(z^2) - erfcx(-z). */
static q128 erfcx_q(q128 z) {
  if (z != z) return z; /* NaN */
  if (z < 0) return 2 * expf128(z * z) - erfcx_q(-z);
  if (z < 100) return expf128(z * z) * erfcf128(z);
  const q128 v = 1 / (2 * z * z);
  q128 term = 1, sum = 1;
  for (int k = 1; k <= 12; k++) {
    term *= -(2 * k - 1) * v;
    sum += term;
  }
  return sum / (z * sqrtf128(M_PIf128));
}
static void erfcx_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) c->out[i] = (double)erfcx_q((q128)c->x[i]);
}
void or_erfcx(const double* z, int64_t n, double* out, int nthreads) {
  ctx_t c = {0};
  c.x = z;
  c.out = out;
  parallel_for(n, nthreads, erfcx_range, &c);
}

static int inputs_valid(int model, double SF, double K, double T, double r, double q,
                        int8_t flag) {
  if (!(flag == 1 || flag == -1)) return 0;
  if (!finite_pos(SF) || !finite_pos(K) || !finite_pos(T) || !isfinite(r)) return 0;
  if (model == ORC_BSM && !isfinite(q)) return 0;
  return 1;
}

/* Model price at sigma: P = D sqrt(FK) b(x, sigma sqrt(T), theta), which is the
 * textbook theta D [F Phi(theta d1) - K Phi(theta d2)]. */
static q128 price_q(int model, double SF, double K, double T, double r, double q, double sigma,
                    int th) {
  q128 qq = (model == ORC_BSM) ? (q128)q : 0;
  q128 D = expf128(-(q128)r * (q128)T);
  q128 F = (model == ORC_BLACK76) ? (q128)SF : (q128)SF * expf128(((q128)r - qq) * (q128)T);
  q128 s = (q128)sigma * sqrtf128((q128)T);
  q128 x = logf128(F / (q128)K);
  return D * sqrtf128(F * (q128)K) * nb_q(x, s, th);
}
static void price_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    double q = c->q ? c->q[i] : 0.0;
    if (!inputs_valid(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->flag[i]) ||
        !(c->sigma[i] >= 0) || !isfinite(c->sigma[i])) {
      c->out[i] = NAN;
      continue;
    }
    c->out[i] = (double)price_q(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->sigma[i],
                                c->flag[i]);
  }
}
void or_price(int model, const double* S_or_F, const double* K, const double* T, const double* r,
              const double* q, const double* sigma, const int8_t* flag, int64_t n, double* out,
              int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.sigma = sigma;
  c.flag = flag;
  c.out = out;
  parallel_for(n, nthreads, price_range, &c);
}

/* Textbook price in plain FP64 (glibc erfc): theta D [F Phi(theta d1) -
 * K Phi(theta d2)].  Fast; loses relative accuracy deep out of the money to
 * the subtraction.  Used to generate large input sets, whose implied
 * volatility the definition then inverts exactly as given. */
static void price_f64_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    const double q = c->q ? c->q[i] : 0.0;
    const double SF = c->SF[i], K = c->K[i], T = c->T[i], r = c->r[i], sg = c->sigma[i];
    const int th = c->flag[i];
    if (!inputs_valid(c->model, SF, K, T, r, q, c->flag[i]) || !(sg >= 0) || !isfinite(sg)) {
      c->out[i] = NAN;
      continue;
    }
    const double D = exp(-r * T);
    const double F = (c->model == ORC_BLACK76) ? SF : SF * exp((r - q) * T);
    double v;
    if (sg == 0) {
      v = th * (F - K);
      v = v > 0 ? v : 0;
    } else {
      const double s = sg * sqrt(T);
      const double d1 = log(F / K) / s + 0.5 * s, d2 = d1 - s;
      v = th * (F * Phi_d(th * d1) - K * Phi_d(th * d2));
      if (v < 0) v = 0;
    }
    c->out[i] = D * v;
  }
}
void or_price_f64(int model, const double* S_or_F, const double* K, const double* T,
                  const double* r, const double* q, const double* sigma, const int8_t* flag,
                  int64_t n, double* out, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.sigma = sigma;
  c.flag = flag;
  c.out = out;
  parallel_for(n, nthreads, price_f64_range, &c);
}

/* Relative distance, in units of 2^-52, of the three decision quantities of
 * the status rule to their thresholds (below-intrinsic, above-maximum, at
 * intrinsic).  A quote within a few units sits where one-ulp differences
 * between two libm implementations of exp/log1p/expm1 can flip the decision. */
static double status_margin(const quote_f64* d, int8_t flag) {
  if (d->status == ORC_INVALID) return INFINITY;
  const double eps = 2.220446049250313080847263336181640625e-16;
  const double x = d->x, beta = d->beta, th = (double)flag;
  const double E = expm1(-0.5 * fabs(x));
  const double Em = exp(-0.5 * fabs(x));
  const int itm = th * x > 0;
  const double iota = itm ? (-E * (1.0 + Em)) / Em : 0.0;
  const double bmax_otm = Em;
  const double beta_otm = itm ? beta - iota : beta;
  double m = INFINITY;
  if (iota > 0) {
    m = fmin(m, fabs(beta / (iota * (1.0 - EPS_S)) - 1.0));
    m = fmin(m, fabs(beta / (iota * (1.0 + EPS_S)) - 1.0));
  }
  m = fmin(m, fabs(beta_otm / (bmax_otm * (1.0 - EPS_S)) - 1.0) * (bmax_otm / (beta > bmax_otm ? beta : bmax_otm)));
  return m / eps;
}

static void status_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    quote_f64 d;
    decide_f64(c->model, c->P[i], c->SF[i], c->K[i], c->T[i], c->r[i], c->q ? c->q[i] : 0.0,
               c->flag[i], &d);
    c->status[i] = (uint8_t)d.status;
    if (c->out) c->out[i] = d.x;
    if (c->out2) c->out2[i] = d.beta;
    if (c->out3) c->out3[i] = status_margin(&d, c->flag[i]);
  }
}
void or_status(int model, const double* P, const double* S_or_F, const double* K, const double* T,
               const double* r, const double* q, const int8_t* flag, int64_t n, uint8_t* status,
               double* x_out, double* beta_out, double* margin_out, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.P = P;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.status = status;
  c.out = x_out;
  c.out2 = beta_out;
  c.out3 = margin_out;
  parallel_for(n, nthreads, status_range, &c);
}

/* ------------------------------------------------------------------------- */
/* Definition of implied volatility                                           */
/* ------------------------------------------------------------------------- */
static void iv_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    double q = c->q ? c->q[i] : 0.0;
    quote_f64 d;
    decide_f64(c->model, c->P[i], c->SF[i], c->K[i], c->T[i], c->r[i], q, c->flag[i], &d);
    c->status[i] = (uint8_t)d.status;
    if (d.status != ORC_OK) {
      c->out[i] = NAN;
      continue;
    }
    if (!d.solve) {
      c->out[i] = 0.0;
      continue;
    }
    q128 x, beta;
    normalise_q(c->model, c->P[i], c->SF[i], c->K[i], c->T[i], c->r[i], q, &x, &beta);
    const int th = c->flag[i];
    q128 iota = (q128)th * (expf128(0.5f128 * x) - expf128(-0.5f128 * x));
    if (iota < 0) iota = 0;
    q128 beta_otm = ((q128)th * x > 0) ? beta - iota : beta;
    q128 x_otm = x > 0 ? -x : x;
    q128 s = solve_definition_q(beta_otm, x_otm);
    c->out[i] = (double)(s / sqrtf128((q128)c->T[i]));
  }
}
void or_iv(int model, const double* P, const double* S_or_F, const double* K, const double* T,
           const double* r, const double* q, const int8_t* flag, int64_t n, double* sigma,
           uint8_t* status, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.P = P;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.out = sigma;
  c.status = status;
  parallel_for(n, nthreads, iv_range, &c);
}

static void cond_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    double q = c->q ? c->q[i] : 0.0;
    c->out[i] = NAN;
    c->out2[i] = NAN;
    if (!inputs_valid(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->flag[i])) continue;
    if (!(c->sigma[i] > 0) || !isfinite(c->sigma[i])) continue;
    q128 x, beta;
    normalise_q(c->model, c->P[i], c->SF[i], c->K[i], c->T[i], c->r[i], q, &x, &beta);
    q128 s = (q128)c->sigma[i] * sqrtf128((q128)c->T[i]);
    q128 h = x / s, t = 0.5f128 * s;
    q128 v = q_inv_sqrt_2pi() * expf128(-0.5f128 * (h * h + t * t));
    c->out[i] = (double)v;
    c->out2[i] = (double)(beta / (s * v));
  }
}
void or_conditioning(int model, const double* P, const double* S_or_F, const double* K,
                     const double* T, const double* r, const double* q, const int8_t* flag,
                     const double* sigma, int64_t n, double* vega_n, double* kappa,
                     int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.P = P;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.sigma = sigma;
  c.out = vega_n;
  c.out2 = kappa;
  parallel_for(n, nthreads, cond_range, &c);
}

static void lbr_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    quote_f64 d;
    decide_f64(c->model, c->P[i], c->SF[i], c->K[i], c->T[i], c->r[i], c->q ? c->q[i] : 0.0,
               c->flag[i], &d);
    c->status[i] = (uint8_t)d.status;
    if (c->region) c->region[i] = -1;
    if (d.status != ORC_OK) {
      c->out[i] = NAN;
      continue;
    }
    if (!d.solve) {
      c->out[i] = 0.0;
      continue;
    }
    int reg = -1;
    double s = lbr_otm(d.beta_otm, d.x_otm, c->n_iter, &reg, c->ev);
    if (c->region) c->region[i] = (int8_t)reg;
    c->out[i] = s / sqrt(c->T[i]);
  }
}
void or_iv_lbr(int model, const double* P, const double* S_or_F, const double* K, const double* T,
               const double* r, const double* q, const int8_t* flag, int64_t n, int n_iter,
               double* sigma, uint8_t* status, int8_t* region, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.P = P;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.out = sigma;
  c.status = status;
  c.region = region;
  c.n_iter = n_iter;
  c.ev = &NB_BINARY128;
  parallel_for(n, nthreads, lbr_range, &c);
}

void or_iv_lbr_f64(int model, const double* P, const double* S_or_F, const double* K,
                   const double* T, const double* r, const double* q, const int8_t* flag,
                   int64_t n, int n_iter, double* sigma, uint8_t* status, int8_t* region,
                   int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.P = P;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.out = sigma;
  c.status = status;
  c.region = region;
  c.n_iter = n_iter;
  c.ev = &NB_FP64;
  parallel_for(n, nthreads, lbr_range, &c);
}

static void nb_f64_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    const double x = c->x[i], s = c->s[i];
    const int th = c->flag[i] >= 0 ? 1 : -1;
    /* intrinsic part and the reduced call: b(x,s,th) = iota + b(-|x|, s) */
    const double iota = th * x > 0 ? 2.0 * sinh(0.5 * fabs(x)) : 0.0;
    c->out[i] = s > 0 ? iota + nb_f64(-fabs(x), s) : iota;
  }
}
void or_normalised_black_f64(const double* x, const double* s, const int8_t* theta, int64_t n,
                             double* out, int nthreads) {
  ctx_t c = {0};
  c.x = x;
  c.s = s;
  c.flag = theta;
  c.out = out;
  parallel_for(n, nthreads, nb_f64_range, &c);
}

/* ------------------------------------------------------------------------- */
/* Halley x8 + bisection fallback (Section 2.2, second item), FP64            */
/* ------------------------------------------------------------------------- */
#define HALLEY_STEPS 8
#define HALLEY_CONV_TOL 1e-10

/* Fallback: bisection inside [lo, hi] on a residual increasing in s, each
 * bisection replaced by a Newton step when that step stays in the bracket.
 * The residual is the transformed objective of the LBR wings (Section 2.2),
 * under which Newton does not crawl where b is exponentially small:
 *   beta <= b_max/2:  f = 1/ln beta - 1/ln b,               f' = (b'/b) / ln^2 b
 *   beta >  b_max/2:  f = ln(b_max - beta) - ln(b_max - b),  f' = b'/(b_max - b)
 * Without an upper end the Newton step (at least doubling s, at most x16)
 * grows the bracket; without a lower end it shrinks it (at least halving,
 * at most /16). */
static double fallback_resid(double x, double s, int upper, double ln_c_beta, double inv_ln_beta,
                             double* fp) {
  const double vega = vega_d(x, s);
  if (upper) {
    const double c = nbc_d(x, s);
    *fp = vega / c;
    return ln_c_beta - log(c);
  }
  double L, qb;
  nb_log_d(x, s, &L, &qb);
  *fp = qb / (L * L);
  return inv_ln_beta - 1.0 / L;
}

static double bisect_fallback(double beta, double x, double lo, double hi) {
  const double eps = 2.220446049250313e-16;
  const double bmax = exp(0.5 * x);
  const int upper = beta > 0.5 * bmax;
  const double ln_c_beta = upper ? log(bmax - beta) : 0.0;
  const double inv_ln_beta = upper ? 0.0 : 1.0 / log(beta);
  double s;
  if (lo > 0 && isfinite(hi))
    s = 0.5 * (lo + hi);
  else if (isfinite(hi))
    s = 0.5 * hi;
  else
    s = fmax(2.0 * lo, 1e-3);
  for (int it = 0; it < 400; it++) {
    double fp;
    const double f = fallback_resid(x, s, upper, ln_c_beta, inv_ln_beta, &fp);
    /* a NaN residual comes from b underflowing at s far below the root */
    if (f > 0)
      hi = s;
    else if (f < 0 || f != f)
      lo = s;
    else
      return s;
    double sn = s - f / fp;
    if (!isfinite(hi))
      sn = (isfinite(sn) && sn > s) ? fmin(sn, 16.0 * s) : 2.0 * s;
    else if (!(lo > 0))
      sn = (isfinite(sn) && sn > 0 && sn < s) ? fmax(sn, s / 16.0) : 0.5 * s;
    else if (!(sn > lo && sn < hi))
      sn = 0.5 * (lo + hi);
    const double ds = sn - s;
    s = sn;
    if (lo > 0 && isfinite(hi) && (fabs(ds) <= 2.0 * eps * s || hi - lo <= 4.0 * eps * hi)) break;
  }
  return s;
}

static double halley_otm(double beta, double x, int* fell_back) {
  /* Brenner-Subrahmanyam: at the money b ~ s / sqrt(2 pi) */
  double s = SQRT_2PI * beta;
  double lo = 0.0, hi = INFINITY, newton_err = INFINITY;
  /* g = b - beta, evaluated as (b_max - beta) - (b_max - b) above b_max / 2 */
  const double bmax = exp(0.5 * x);
  const int upper = beta > 0.5 * bmax;
  for (int k = 0; k < HALLEY_STEPS; k++) {
    const double g = upper ? (bmax - beta) - nbc_d(x, s) : nb_d(x, s) - beta;
    if (g < 0)
      lo = s;
    else if (g > 0)
      hi = s;
    else {
      newton_err = 0;
      break;
    }
    const double h = x / s, t = 0.5 * s;
    const double bp = exp(-0.5 * (h * h + t * t)) * INV_SQRT_2PI;
    const double u = h * h / s - 0.25 * s;
    /* Newton estimate of the distance to the root, relative to s: the
     * convergence test of the last sweep (a tiny Halley step alone can come
     * from a flat residual far from the root) */
    newton_err = fabs(g / bp) / s;
    /* Halley on g = b - beta: ds = -2 g g' / (2 g'^2 - g g'') */
    double step = -2.0 * g / (2.0 * bp - g * u);
    double sn = s + step;
    /* a step that leaves the bracket [lo, hi] becomes a bisection (or a
     * doubling while no upper end is known) */
    if (!(sn >= lo && sn <= hi) || !isfinite(sn)) sn = isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * s;
    s = sn;
  }
  int ok = isfinite(s) && s > 0 && newton_err <= HALLEY_CONV_TOL;
  if (!ok) {
    *fell_back = 1;
    s = bisect_fallback(beta, x, lo, hi);
  } else {
    *fell_back = 0;
  }
  return s;
}

static void halley_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    quote_f64 d;
    decide_f64(c->model, c->P[i], c->SF[i], c->K[i], c->T[i], c->r[i], c->q ? c->q[i] : 0.0,
               c->flag[i], &d);
    c->status[i] = (uint8_t)d.status;
    if (c->region) ((uint8_t*)c->region)[i] = 0;
    if (d.status != ORC_OK) {
      c->out[i] = NAN;
      continue;
    }
    if (!d.solve) {
      c->out[i] = 0.0;
      continue;
    }
    int fb = 0;
    double s = halley_otm(d.beta_otm, d.x_otm, &fb);
    if (c->region) ((uint8_t*)c->region)[i] = (uint8_t)fb;
    c->out[i] = s / sqrt(c->T[i]);
  }
}
void or_iv_halley(int model, const double* P, const double* S_or_F, const double* K,
                  const double* T, const double* r, const double* q, const int8_t* flag, int64_t n,
                  double* sigma, uint8_t* status, uint8_t* fallback, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.P = P;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.out = sigma;
  c.status = status;
  c.region = (int8_t*)fallback;
  parallel_for(n, nthreads, halley_range, &c);
}

/* ------------------------------------------------------------------------- */
/* Greeks and the implicit-function gradient (binary128 closed forms)         */
/* ------------------------------------------------------------------------- */
typedef struct {
  q128 V, dS, dK, dT, dr, dq, vega, gamma;
} partials_q;

/* raw partial derivatives of the model price at sigma */
static void partials(int model, double SF, double K, double T, double r, double q, double sigma,
                     int th, partials_q* o) {
  const q128 qT = (q128)T, sq = sqrtf128(qT), sv = (q128)sigma * sq, qK = (q128)K;
  const q128 qth = (q128)th, qr = (q128)r;
  const q128 Dr = expf128(-qr * qT);
  if (model == ORC_BLACK76) {
    const q128 F = (q128)SF;
    const q128 d1 = (logf128(F / qK) + 0.5f128 * sv * sv) / sv, d2 = d1 - sv;
    const q128 N1 = Phi_q(qth * d1), N2 = Phi_q(qth * d2), n1 = phi_q(d1);
    o->V = Dr * qth * (F * N1 - qK * N2);
    o->dS = qth * Dr * N1;
    o->dK = -qth * Dr * N2;
    o->vega = F * Dr * n1 * sq;
    o->dT = -qr * o->V + Dr * F * n1 * (q128)sigma / (2 * sq);
    o->dr = -qT * o->V;
    o->dq = 0;
    o->gamma = Dr * n1 / (F * sv);
  } else {
    const q128 S = (q128)SF, qq = (model == ORC_BSM) ? (q128)q : 0;
    const q128 Dq = expf128(-qq * qT);
    const q128 d1 = (logf128(S / qK) + (qr - qq + 0.5f128 * (q128)sigma * (q128)sigma) * qT) / sv;
    const q128 d2 = d1 - sv;
    const q128 N1 = Phi_q(qth * d1), N2 = Phi_q(qth * d2), n1 = phi_q(d1);
    o->V = qth * (S * Dq * N1 - qK * Dr * N2);
    o->dS = qth * Dq * N1;
    o->dK = -qth * Dr * N2;
    o->vega = S * Dq * n1 * sq;
    o->dT = S * Dq * n1 * (q128)sigma / (2 * sq) - qth * qq * S * Dq * N1 + qth * qr * qK * Dr * N2;
    o->dr = qth * qK * qT * Dr * N2;
    o->dq = -qth * S * qT * Dq * N1;
    o->gamma = Dq * n1 / (S * sv);
  }
}

static void greeks_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    double q = c->q ? c->q[i] : 0.0;
    double* outs[5] = {c->out, c->out2, c->out3, c->out4, c->out5};
    if (!inputs_valid(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->flag[i]) ||
        !(c->sigma[i] > 0) || !isfinite(c->sigma[i])) {
      for (int k = 0; k < 5; k++)
        if (outs[k]) outs[k][i] = NAN;
      continue;
    }
    partials_q p;
    partials(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->sigma[i], c->flag[i], &p);
    if (c->out) c->out[i] = (double)p.dS;
    if (c->out2) c->out2[i] = (double)p.gamma;
    if (c->out3) c->out3[i] = (double)(p.vega * 0.01f128);
    if (c->out4) c->out4[i] = (double)(-p.dT / 365.0f128);
    if (c->out5) c->out5[i] = (double)(p.dr * 0.01f128);
  }
}
void or_greeks(int model, const double* S_or_F, const double* K, const double* T, const double* r,
               const double* q, const double* sigma, const int8_t* flag, int64_t n, double* delta,
               double* gamma, double* vega, double* theta, double* rho, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.sigma = sigma;
  c.flag = flag;
  c.out = delta;
  c.out2 = gamma;
  c.out3 = vega;
  c.out4 = theta;
  c.out5 = rho;
  parallel_for(n, nthreads, greeks_range, &c);
}

static void grad_range(void* c_, int64_t i0, int64_t i1) {
  ctx_t* c = (ctx_t*)c_;
  for (int64_t i = i0; i < i1; i++) {
    double q = c->q ? c->q[i] : 0.0;
    double* outs[6] = {c->out, c->out2, c->out3, c->out4, c->out5, c->out6};
    for (int k = 0; k < 6; k++)
      if (outs[k]) outs[k][i] = 0.0;
    if (c->status_in[i] != ORC_OK || !(c->sigma[i] > 0) || !isfinite(c->sigma[i])) continue;
    if (!inputs_valid(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->flag[i])) continue;
    partials_q p;
    partials(c->model, c->SF[i], c->K[i], c->T[i], c->r[i], q, c->sigma[i], c->flag[i], &p);
    if (!(p.vega > 0) || (double)p.vega == 0.0) continue;
    const q128 g = (q128)c->grad[i];
    if (c->out) c->out[i] = (double)(g / p.vega);
    if (c->out2) c->out2[i] = (double)(-g * p.dS / p.vega);
    if (c->out3) c->out3[i] = (double)(-g * p.dK / p.vega);
    if (c->out4) c->out4[i] = (double)(-g * p.dT / p.vega);
    if (c->out5) c->out5[i] = (double)(-g * p.dr / p.vega);
    if (c->out6) c->out6[i] = (double)(-g * p.dq / p.vega);
  }
}
void or_iv_grad(int model, const double* S_or_F, const double* K, const double* T, const double* r,
                const double* q, const int8_t* flag, const double* sigma, const uint8_t* status,
                const double* grad_sigma, int64_t n, double* gP, double* gS, double* gK,
                double* gT, double* gr, double* gq, int nthreads) {
  ctx_t c = {0};
  c.model = model;
  c.SF = S_or_F;
  c.K = K;
  c.T = T;
  c.r = r;
  c.q = (model == ORC_BSM) ? q : NULL;
  c.flag = flag;
  c.sigma = sigma;
  c.status_in = status;
  c.grad = grad_sigma;
  c.out = gP;
  c.out2 = gS;
  c.out3 = gK;
  c.out4 = gT;
  c.out5 = gr;
  c.out6 = gq;
  parallel_for(n, nthreads, grad_range, &c);
}
