/*
 * fv_oracle.h -- plain, slow CPU oracle for batched implied volatility.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, constant or helper with
 * the CUDA library.
 *
 * What it computes (paper: "fast-vollib", Sections 2.2-2.4 and 3):
 *   - the Black-76 / Black-Scholes / Black-Scholes-Merton price of a European
 *     quote (Section 3 "Pricing models"; Black-76 prices are discounted,
 *     Section 2.4);
 *   - the implied volatility as its DEFINITION: the unique sigma >= 0 whose
 *     model price equals the quote, found by bisection in IEEE binary128;
 *   - the same root by Jaeckel's "Let's Be Rational" steps (Section 2.2, first
 *     item) and by the Halley x8 + bisection path (Section 2.2, second item),
 *     written step by step in FP64 with the normalised Black function taken
 *     from binary128 (so only the algorithm, not its wing arithmetic, is under
 *     test);
 *   - the five Greeks (Section 3 "Greeks") and the implicit-function gradient
 *     of sigma with respect to every market input (Section 3 "Differentiable
 *     IV").
 *
 * All arrays are host memory, length n, owned by the caller.  nthreads <= 0
 * means "all online cores".
 */
#ifndef FV_ORACLE_H
#define FV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* models (Section 3 "Pricing models") */
#define ORC_BLACK76 0       /* forward F, discounted price (Section 2.4) */
#define ORC_BLACK_SCHOLES 1 /* spot S, no dividend yield                  */
#define ORC_BSM 2           /* spot S, continuous dividend yield q        */

/* per-quote status */
#define ORC_OK 0
#define ORC_BELOW_INTRINSIC 1
#define ORC_ABOVE_MAX 2
#define ORC_INVALID 3

int or_num_threads(void);

/* Normalised Black b(x, s, theta) in binary128, rounded to double.
 * b = theta*[e^{x/2} Phi(theta(x/s + s/2)) - e^{-x/2} Phi(theta(x/s - s/2))],
 * s = 0 gives the normalised intrinsic value. */
void or_normalised_black(const double* x, const double* s, const int8_t* theta,
                         int64_t n, double* out, int nthreads);

/* erfcx(z) = exp(z^2) erfc(z) in binary128, rounded to double (the function
 * of the erfcx branch of Section 2.2's normalised Black evaluation). */
void or_erfcx(const double* z, int64_t n, double* out, int nthreads);

/* Model price at sigma (binary128, rounded).  q is ignored unless model is BSM
 * (may be NULL otherwise).  Invalid inputs give NaN. */
void or_price(int model, const double* S_or_F, const double* K, const double* T,
              const double* r, const double* q, const double* sigma,
              const int8_t* flag, int64_t n, double* out, int nthreads);

/* The same price by the textbook formula in plain FP64 (fast; deep out of
 * the money it loses relative accuracy to the subtraction).  A generator of
 * large input sets. */
void or_price_f64(int model, const double* S_or_F, const double* K, const double* T,
                  const double* r, const double* q, const double* sigma,
                  const int8_t* flag, int64_t n, double* out, int nthreads);

/* Status only, by the FP64 decision rule (also returns the FP64 normalised
 * log-moneyness x, the normalised price beta, and the relative distance of
 * the rule's quantities to its nearest threshold in units of 2^-52; NULL to
 * skip any of the three). */
void or_status(int model, const double* P, const double* S_or_F, const double* K,
               const double* T, const double* r, const double* q,
               const int8_t* flag, int64_t n, uint8_t* status, double* x_out,
               double* beta_out, double* margin_out, int nthreads);

/* Implied volatility by definition: binary128 bisection on the normalised
 * Black function.  sigma = NaN unless status is OK; sigma = 0 at intrinsic. */
void or_iv(int model, const double* P, const double* S_or_F, const double* K,
           const double* T, const double* r, const double* q, const int8_t* flag,
           int64_t n, double* sigma, uint8_t* status, int nthreads);

/* Conditioning of each quote at sigma: normalised vega b'(x, s) and
 * kappa = beta / (s * b'), with beta the full normalised price. */
void or_conditioning(int model, const double* P, const double* S_or_F,
                     const double* K, const double* T, const double* r,
                     const double* q, const int8_t* flag, const double* sigma,
                     int64_t n, double* vega_n, double* kappa, int nthreads);

/* "Let's Be Rational" in FP64, n_iter Householder(3) steps.  region (may be
 * NULL) receives 0 lowest, 1 lower-middle, 2 upper-middle, 3 highest, -1 when
 * no iteration ran. */
void or_iv_lbr(int model, const double* P, const double* S_or_F, const double* K,
               const double* T, const double* r, const double* q,
               const int8_t* flag, int64_t n, int n_iter, double* sigma,
               uint8_t* status, int8_t* region, int nthreads);

/* The same LBR steps with the normalised Black function evaluated in plain
 * FP64 by the oracle's own routine (erfcx difference with a continued-
 * fraction erfcx, the small-t odd series of the Mills ratio, the CDF-direct
 * form past the inflection point): an FP64 CPU implementation of the whole
 * solver, the CPU baseline of the benchmark. */
void or_iv_lbr_f64(int model, const double* P, const double* S_or_F, const double* K,
                   const double* T, const double* r, const double* q, const int8_t* flag,
                   int64_t n, int n_iter, double* sigma, uint8_t* status, int8_t* region,
                   int nthreads);

/* That FP64 normalised Black b(x, s, theta) (intrinsic part plus the reduced
 * call), exported so that it can be pinned against the binary128 one. */
void or_normalised_black_f64(const double* x, const double* s, const int8_t* theta, int64_t n,
                             double* out, int nthreads);

/* Halley x8 from the Brenner-Subrahmanyam guess, bisection fallback on the
 * quotes that fail the convergence test; fallback (may be NULL) flags them. */
void or_iv_halley(int model, const double* P, const double* S_or_F,
                  const double* K, const double* T, const double* r,
                  const double* q, const int8_t* flag, int64_t n, double* sigma,
                  uint8_t* status, uint8_t* fallback, int nthreads);

/* Greeks in the py_vollib scaling: delta, gamma, vega per 1% vol, theta per
 * calendar day (dV/dt = -dV/dT over 365), rho per 1% rate.  Black-76 Greeks
 * are with respect to F.  NaN unless sigma > 0 and inputs valid. */
void or_greeks(int model, const double* S_or_F, const double* K, const double* T,
               const double* r, const double* q, const double* sigma,
               const int8_t* flag, int64_t n, double* delta, double* gamma,
               double* vega, double* theta, double* rho, int nthreads);

/* Gradient of sigma(P, S|F, K, T, r, q) by the implicit-function theorem,
 * times grad_sigma: g_i = grad_sigma * (-dV/d theta_i) / (dV/d sigma),
 * g_P = grad_sigma / (dV/d sigma).  Zero where status != OK, sigma <= 0 or the
 * raw vega is 0.  g_q is 0 unless model is BSM. */
void or_iv_grad(int model, const double* S_or_F, const double* K,
                const double* T, const double* r, const double* q,
                const int8_t* flag, const double* sigma, const uint8_t* status,
                const double* grad_sigma, int64_t n, double* gP, double* gS,
                double* gK, double* gT, double* gr, double* gq, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
