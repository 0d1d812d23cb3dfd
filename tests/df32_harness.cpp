// Host build of the kernels' double-float functions (paper_2604_27210_gb300/
// csrc/fv_df32.cuh) for the CPU tests: compiled with the host C++ compiler
// (-ffp-contract=off) and loaded with ctypes.  Double-float values cross as
// pairs of floats.
#include "fv_df32.cuh"

using fvdf::df;

extern "C" {

void h_dexp(float ah, float al, float* out) {
  const df r = fvdf::dexp(df{ah, al});
  out[0] = r.h;
  out[1] = r.l;
}

void h_dlog(float yh, float yl, float* out) {
  const df r = fvdf::dlog(df{yh, yl});
  out[0] = r.h;
  out[1] = r.l;
}

void h_dlog_of(double d, float* out) {
  const df r = fvdf::dlog_of(d);
  out[0] = r.h;
  out[1] = r.l;
}

void h_derfcx(float zh, float zl, float* out) {
  const df r = fvdf::derfcx(df{zh, zl});
  out[0] = r.h;
  out[1] = r.l;
}

int h_df_of(double d, float* out) {
  df r;
  const bool ok = fvdf::df_of(d, r);
  out[0] = r.h;
  out[1] = r.l;
  return ok ? 1 : 0;
}

void h_drsqrt(float yh, float yl, float* out) {
  const df r = fvdf::drsqrt(df{yh, yl});
  out[0] = r.h;
  out[1] = r.l;
}

// B (or the complement C), E and h of the normalised Black evaluation
int h_nb(double x, float s, int reg, float* out) {
  df xd;
  if (x == 0.0) xd = fvdf::mk(0.0f);
  else if (!fvdf::df_of(x, xd)) return 0;
  fvdf::NBdf v;
  if (!fvdf::nb_df(xd, s, reg, v)) return 0;
  out[0] = v.B.h;
  out[1] = v.B.l;
  out[2] = v.E.h;
  out[3] = v.E.l;
  out[4] = v.h.h;
  out[5] = v.h.l;
  out[6] = v.via_comp ? 1.0f : 0.0f;
  return 1;
}

int h_corr(double beta, double c_beta, double x, double ln_beta, double T, float s, int reg,
           double* sigma) {
  return fvdf::hh3_correction_df(beta, c_beta, x, ln_beta, T, s, reg, *sigma) ? 1 : 0;
}
}

extern "C" {
// the double-float status rule: out = {status, solve, fp64, tiny}, vals = the
// reduced quote (beta, x, bmax, c_beta, ln_beta as hi, lo pairs)
void h_decide(int model, const double* P, const double* SF, const double* K, const double* T,
              const double* r, const double* q, const signed char* flag, long n, int* out,
              float* vals) {
  for (long i = 0; i < n; i++) {
    const fvdf::NormDF d = fvdf::decide_df(model, P[i], SF[i], K[i], T[i], r[i], q[i], flag[i]);
    out[4 * i] = d.status;
    out[4 * i + 1] = d.solve;
    out[4 * i + 2] = d.fp64;
    out[4 * i + 3] = d.tiny;
    const df v[5] = {d.beta, d.x, d.bmax, d.c_beta, d.ln_beta};
    for (int k = 0; k < 5; k++) {
      vals[10 * i + 2 * k] = v[k].h;
      vals[10 * i + 2 * k + 1] = v[k].l;
    }
  }
}

void h_dlog1p(float uh, float ul, float* out) {
  const df r = fvdf::dlog1p(df{uh, ul});
  out[0] = r.h;
  out[1] = r.l;
}
}

extern "C" void h_dexp_em1(float ah, float al, float* out) {
  df em1;
  const df e = fvdf::dexp_em1(df{ah, al}, em1);
  out[0] = e.h;
  out[1] = e.l;
  out[2] = em1.h;
  out[3] = em1.l;
}
