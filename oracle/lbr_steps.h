/*
 * lbr_steps.h -- the oracle's FP64 status rule and its step-by-step FP64
 * "Let's Be Rational" solver with its own FP64 normalised Black function.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle; see fv_oracle.h).
 *
 * Written in the common subset of C and C++ over a scalar type R, so that the
 * same source serves two builds:
 *   - fv_oracle.c includes it with R = double: the oracle itself;
 *   - op_count.cpp includes it with R = an operation-counting type: the
 *     counted build that measures the method's FP64 work per quote (every
 *     +, -, *, /, square root and comparison, and every elementary-function
 *     call).  There LBR_STEPS_PRIMITIVES is defined and erfcx_f64 and
 *     Phi_inv_d, whose iterations here are a slow oracle's way of reaching a
 *     function value, are supplied as single counted calls.
 * No include guard: op_count.cpp includes it twice, once per scalar type.
 * Values that are constants of the method (1/sqrt(2 pi), factorials, the
 * status band) stay double.
 */
#ifndef R
#define R double
#endif
/* LBR_STEPS_PHASE(k): a hook at the end of each phase of the solver (0: the
 * boundaries and the initial guess; 1, 2, ...: each Householder(3) iteration),
 * by which the counted build attributes its counts; nothing here. */
#ifndef LBR_STEPS_PHASE
#define LBR_STEPS_PHASE(k)
#endif

/* ------------------------------------------------------------------------- */
/* FP64 status decision (the same rule, the same operation order, is what the
 * kernels implement).                                                        */
/* ------------------------------------------------------------------------- */
/* relative slack band of the bound tests: 64 * 2^-52.  Prices that sit at
 * the intrinsic value up to their own rounding land within a few ulp of it;
 * the band is wide enough that one-ulp differences between libm
 * implementations cannot move such a quote across its edge. */
#define EPS_S (64.0 * 2.220446049250313080847263336181640625e-16)

typedef struct {
  int status;      /* ORC_* */
  int solve;       /* 1: OK and a positive root must be found; 0: sigma = 0 */
  R x;        /* ln(F/K) */
  R beta;     /* full normalised price */
  R beta_otm; /* out-of-the-money normalised price (intrinsic removed) */
  R x_otm;    /* -|x| */
} quote_f64;

static int finite_pos(R v) { return isfinite(v) && v > 0; }

static void decide_f64(int model, R P, R SF, R K, R T, R r,
                       R q, int8_t flag, quote_f64* o) {
  memset(o, 0, sizeof(*o));
  o->status = ORC_INVALID;
  if (!(flag == 1 || flag == -1)) return;
  if (!isfinite(P) || !finite_pos(SF) || !finite_pos(K) || !finite_pos(T) || !isfinite(r))
    return;
  R qq = 0.0;
  if (model == ORC_BSM) {
    if (!isfinite(q)) return;
    qq = q;
  }
  /* ln(F/K) (or ln(S/K)): near the money F - K is exact (Sterbenz), so
   * log1p((F-K)/K) keeps x accurate relative to itself; log(F/K) would carry
   * an absolute error of one ulp of 1, which costs ~eps/s in sigma. */
  R lm;
  if (SF >= 0.5 * K && SF <= 2.0 * K)
    lm = log1p((SF - K) / K);
  else
    lm = log(SF / K);
  R x, beta;
  if (model == ORC_BLACK76) {
    x = lm;
    beta = (P * exp(r * T)) / sqrt(SF * K);
  } else {
    x = lm + (r - qq) * T;
    beta = (P * exp(0.5 * (r + qq) * T)) / sqrt(SF * K);
  }
  if (!isfinite(x) || !isfinite(beta)) return;
  const double th = (double)flag;
  /* Em = e^{-|x|/2} is the reduced call's bound; with E = Em - 1 from expm1
   * an in-the-money quote's intrinsic value e^{|x|/2} - e^{-|x|/2} is
   * -E (1 + Em) / Em, accurate near the money and far from it */
  const R E = expm1(-0.5 * fabs(x));
  const R Em = exp(-0.5 * fabs(x));
  const int itm = th * x > 0;
  const R iota = itm ? (-E * (1.0 + Em)) / Em : 0.0;
  o->x = x;
  o->beta = beta;
  if (beta < iota * (1.0 - EPS_S)) {
    o->status = ORC_BELOW_INTRINSIC;
    return;
  }
  const R beta_otm = itm ? beta - iota : beta;
  const R bmax_otm = Em;
  if (beta_otm >= bmax_otm * (1.0 - EPS_S)) {
    o->status = ORC_ABOVE_MAX;
    return;
  }
  o->status = ORC_OK;
  o->beta_otm = beta_otm;
  o->x_otm = -fabs(x);
  o->solve = beta_otm > iota * EPS_S;
}

/* ------------------------------------------------------------------------- */
/* FP64 helpers for the step-by-step solvers                                  */
/* ------------------------------------------------------------------------- */
static const double INV_SQRT_2PI = 0.398942280401432677939946059934381868;
static const double SQRT_2PI = 2.50662827463100050241576528481104525;
static const double SQRT3 = 1.73205080756887729352744634150587237;

/* normalised vega b'(s) = exp(-(h^2 + t^2)/2) / sqrt(2 pi) */
static R vega_d(R x, R s) {
  R h = x / s, t = 0.5 * s;
  return exp(-0.5 * (h * h + t * t)) * INV_SQRT_2PI;
}
static R Phi_d(R z) { return 0.5 * erfc(-z * 0.70710678118654752440); }
#ifndef LBR_STEPS_PRIMITIVES
/* inverse normal CDF: Newton on ln Phi(z) = ln p from the tail asymptote */
static R Phi_inv_d(R p) {
  if (!(p > 0)) return -INFINITY;
  if (!(p < 1)) return INFINITY;
  if (p > 0.5) return -Phi_inv_d(1.0 - p);
  R z = (p > 0.3) ? SQRT_2PI * (p - 0.5) : -sqrt(-2.0 * log(p));
  const R lp = log(p);
  for (int it = 0; it < 100; it++) {
    R Pz = Phi_d(z);
    R pdf = exp(-0.5 * z * z) * INV_SQRT_2PI;
    R dz = (log(Pz) - lp) * Pz / pdf;
    z -= dz;
    if (fabs(dz) <= 1e-15 * (1.0 + fabs(z))) break;
  }
  return z;
}
#endif

/* ------------------------------------------------------------------------- */
/* The normalised Black function in plain FP64 (the oracle's own evaluation, */
/* for the FP64 LBR that serves as the CPU baseline)                          */
/* ------------------------------------------------------------------------- */
static const double SQRT_PI = 1.77245385090551602729816748334114518;
static const double SQRT_PI_OVER_2 = 1.25331413731550025120788264240552263;
static const double LN_SQRT_2PI = 0.918938533204672741780329736405617640;

#ifndef LBR_STEPS_PRIMITIVES
/* erfcx(z) = exp(z^2) erfc(z) for z >= 0 (the solvers' arguments).  Below
 * z = 2: glibc's erfc times exp(z^2) (the rounding of z^2 < 4 costs a few
 * ulp at most).  From z = 2 on: the Laplace continued fraction (Abramowitz &
 * Stegun 7.1.14)
 *   sqrt(pi) erfcx(z) = 1/(z + (1/2)/(z + (2/2)/(z + (3/2)/(z + ...)))),
 * evaluated by the modified Lentz method, which never forms exp(-z^2). */
static R erfcx_f64(R z) {
  if (z != z) return z;
  if (z < 2.0) return exp(z * z) * erfc(z);
  if (isinf(z)) return 0.0;
  const R tiny = 1e-300;
  R f = z, C = z, D = 0.0;
  for (int k = 1; k < 1000; k++) {
    const double a = 0.5 * k;
    D = z + a * D;
    if (D == 0) D = tiny;
    D = 1.0 / D;
    C = z + a / C;
    if (C == 0) C = tiny;
    const R delta = C * D;
    f *= delta;
    if (fabs(delta - 1.0) < 2e-16) break;
  }
  return 1.0 / (SQRT_PI * f);
}
#endif

/* Mills ratio R(z) = Phi(z) / phi(z) = sqrt(pi/2) erfcx(-z/sqrt 2) */
static R mills_f64(R z) { return SQRT_PI_OVER_2 * erfcx_f64(-z * 0.70710678118654752440); }

/* D = R(h+t) - R(h-t) for h + t <= 0, so that b = b' D with the normalised
 * vega b' = e^{x/2} phi(h+t) = e^{-x/2} phi(h-t) = exp(-(h^2+t^2)/2)/sqrt(2pi)
 * (x = 2 h t).  For small t the difference cancels; there the odd part of
 * its Taylor series in t is summed instead,
 *   R(h+t) - R(h-t) = 2 sum_{k odd} R^(k)(h) t^k / k!,
 * with the derivatives from R' = 1 + h R (since phi' = -z phi), hence
 * R^(k+1) = k R^(k-1) + h R^(k) for k >= 1.  The series is taken where
 * t < 0.1 and |h| <= 10 (its recurrence loses about log10(h^2) digits);
 * elsewhere the erfcx difference (which loses log10(|h|/2t) digits). */
static R mills_diff_f64(R h, R t) {
  if (t < 0.1 && fabs(h) <= 10.0) {
    R Rm = mills_f64(h);   /* R^(k-1), starting at R^(0) */
    R Rk = 1.0 + h * Rm;   /* R^(k),   starting at R^(1) */
    R tk = t;          /* t^k */
    double fact = 1.0;  /* k! */
    R sum = Rk * t;
    for (int k = 1; k < 40; k += 2) {
      const R R2 = k * Rm + h * Rk;        /* R^(k+1) */
      const R R3 = (k + 1) * Rk + h * R2;  /* R^(k+2) */
      tk *= t * t;
      fact *= (double)(k + 1) * (k + 2);
      const R term = R3 * tk / fact;
      sum += term;
      Rm = R2;
      Rk = R3;
      if (fabs(term) <= 1e-18 * fabs(sum)) break;
    }
    return 2.0 * sum;
  }
  return mills_f64(h + t) - mills_f64(h - t);
}

/* b(x, s) of the call with x <= 0, s > 0: b' D, except past the inflection
 * point (h + t > 0) outside the small-t series' domain, where b is not small
 * and the CDF-direct form e^{x/2} Phi(h+t) - e^{-x/2} Phi(h-t) loses at most
 * a small factor (with t < 0.1 it would cancel: there the series applies). */
static int cdf_direct(R h, R t) { return h + t > 0 && !(t < 0.1 && fabs(h) <= 10.0); }
static R nb_f64(R x, R s) {
  const R h = x / s, t = 0.5 * s;
  if (cdf_direct(h, t)) return exp(0.5 * x) * Phi_d(h + t) - exp(-0.5 * x) * Phi_d(h - t);
  return vega_d(x, s) * mills_diff_f64(h, t);
}
/* ln b and b'/b without underflow: ln b = ln D - (h^2+t^2)/2 - ln sqrt(2pi) */
static void nb_log_f64(R x, R s, R* L, R* qb) {
  const R h = x / s, t = 0.5 * s;
  if (cdf_direct(h, t)) {
    const R b = nb_f64(x, s);
    *L = log(b);
    *qb = vega_d(x, s) / b;
    return;
  }
  const R D = mills_diff_f64(h, t);
  *L = log(D) - 0.5 * (h * h + t * t) - LN_SQRT_2PI;
  *qb = 1.0 / D;
}
/* b_max - b = e^{x/2} Phi(-(h+t)) + e^{-x/2} Phi(h-t): two positive terms */
static R nbc_f64(R x, R s) {
  const R h = x / s, t = 0.5 * s;
  return exp(0.5 * x) * Phi_d(-(h + t)) + exp(-0.5 * x) * Phi_d(h - t);
}

/* The normalised Black evaluation the step-by-step solvers use: b, ln b with
 * b'/b, and b_max - b of the reduced call (x <= 0). */
typedef struct nb_eval_s {
  R (*nb)(R x, R s);
  void (*nb_log)(R x, R s, R* L, R* qb);
  R (*nbc)(R x, R s);
} nb_eval_t;

/* cubic Hermite interpolation of s(beta) on [b0, b1] from end values and
 * slopes ds/dbeta = 1/b' (the interior initial guess of Section 2.2) */
static R hermite_guess(R beta, R b0, R b1, R s0, R s1, R d0,
                            R d1) {
  R dbeta = b1 - b0;
  if (!(dbeta > 0)) return 0.5 * (s0 + s1);
  R tau = (beta - b0) / dbeta, tau2 = tau * tau, tau3 = tau2 * tau;
  R h00 = 2 * tau3 - 3 * tau2 + 1, h10 = tau3 - 2 * tau2 + tau;
  R h01 = -2 * tau3 + 3 * tau2, h11 = tau3 - tau2;
  return h00 * s0 + h10 * dbeta * d0 + h01 * s1 + h11 * dbeta * d1;
}

/* ------------------------------------------------------------------------- */
/* "Let's Be Rational" (Section 2.2, first item), FP64 step by step           */
/* ------------------------------------------------------------------------- */
/* beta in (0, e^{x/2}), x <= 0 (the reduced out-of-the-money call). */
static R lbr_otm(R beta, R x, int n_iter, int* region, const nb_eval_t* ev) {
  const R bmax = exp(0.5 * x);
  R sc, bc, vc, sl = 0, bl = 0, vl = 0;
  /* boundary points: inflection s_c = sqrt(2|x|), where the tangent of b meets
   * 0 (s_l) and b_max (s_h); six normalised-Black evaluations (b and b' at
   * s_l, s_c, s_h) */
  if (x < 0) {
    sc = sqrt(-2.0 * x);
    bc = ev->nb(x, sc);
    vc = vega_d(x, sc);
    sl = sc - bc / vc;
    if (sl > 0) {
      bl = ev->nb(x, sl);
      vl = vega_d(x, sl);
    } else {
      sl = 0;
    }
  } else {
    sc = 0;
    bc = 0;
    vc = INV_SQRT_2PI;
  }
  const R sh = sc + (bmax - bc) / vc;
  const R bh = ev->nb(x, sh), vh = vega_d(x, sh);

  /* four-region initial guess */
  int reg;
  R s;
  if (beta < bl) {
    /* lowest wing: b ~ c Phi(-|x|/(sqrt3 s))^3 as s -> 0; c matched at s_l */
    reg = 0;
    const R zl = -fabs(x) / (SQRT3 * sl);
    const R Pl = Phi_d(zl);
    const R cl = bl / (Pl * Pl * Pl);
    const R z = Phi_inv_d(cbrt(beta / cl));
    s = fabs(x) / (SQRT3 * fabs(z));
  } else if (beta <= bc) {
    reg = 1;
    s = hermite_guess(beta, bl, bc, sl, sc, vl > 0 ? 1.0 / vl : 0.0, 1.0 / vc);
  } else if (beta <= bh) {
    reg = 2;
    s = hermite_guess(beta, bc, bh, sc, sh, 1.0 / vc, 1.0 / vh);
  } else {
    /* highest wing: b_max - b ~ c' Phi(-s/2) as s -> inf; c' matched at s_h */
    reg = 3;
    const R ch = ev->nbc(x, sh) / Phi_d(-0.5 * sh);
    s = -2.0 * Phi_inv_d((bmax - beta) / ch);
  }
  if (region) *region = reg;

  LBR_STEPS_PHASE(0);
  /* three-branch objective + Householder(3) */
  const R ln_beta = log(beta);
  const R c_beta = bmax - beta;
  for (int k = 0; k < n_iter; k++) {
    if (!(s > 0) || !isfinite(s)) break;
    const R h = x / s, t = 0.5 * s;
    const R bp = exp(-0.5 * (h * h + t * t)) * INV_SQRT_2PI;
    const R u = h * h / s - 0.25 * s;           /* b''/b' */
    const R du = -3.0 * h * h / (s * s) - 0.25; /* d(b''/b')/ds */
    R nu, h2, h3;
    if (reg == 0) {
      /* g = 1/ln b - 1/ln beta */
      R L, qb;
      ev->nb_log(x, s, &L, &qb);
      if (!isfinite(L)) { /* b = 0 even in binary128: s far too small */
        s *= 1.5;
        continue;
      }
      const R k1 = 1.0 + 2.0 / L;
      const R g = 1.0 / L - 1.0 / ln_beta;
      const R gp = -qb / (L * L);
      nu = -g / gp;
      h2 = u - qb * k1;
      h3 = h2 * h2 + du - (qb * u - qb * qb) * k1 + 2.0 * qb * qb / (L * L);
    } else if (reg == 3) {
      /* g = ln((b_max - beta)/(b_max - b)) */
      const R cb = ev->nbc(x, s);
      const R w = bp / cb;
      const R g = log(c_beta / cb);
      nu = -g / w;
      h2 = u + w;
      h3 = h2 * h2 + du + w * h2;
    } else {
      /* g = b - beta */
      const R b = ev->nb(x, s);
      nu = -(b - beta) / bp;
      h2 = u;
      h3 = u * u + du;
    }
    R ds = nu * (1.0 + 0.5 * h2 * nu) / (1.0 + nu * (h2 + h3 * nu / 6.0));
    if (!isfinite(ds)) ds = nu;
    /* keep s positive */
    if (s + ds <= 0.25 * s) ds = -0.75 * s;
    s += ds;
    LBR_STEPS_PHASE(k + 1);
  }
  return s;
}

