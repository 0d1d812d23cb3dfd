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
