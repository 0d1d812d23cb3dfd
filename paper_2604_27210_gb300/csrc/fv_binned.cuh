// fv_binned.cuh -- the LBR tile routine with CTA-local region binning, shared
// by the flat batch kernels (fv_kernels.cu) and the chains kernels
// (fv_chains.cu).
#pragma once

#include "fv_device.cuh"
#include "fv_internal.h"

namespace fvk {

using namespace fvd;

// ---------------------------------------------------------------------------
// LBR with CTA-local region binning (FP64 and mixed)
//
// Phase 1 decides every quote of a tile (one quote per thread per round,
// coalesced loads) and, for the quotes that need a root, evaluates an FP32
// proxy of the LBR region and of the small-t class (t < t_small of the FP64
// normalised Black function) from the FP32 boundaries and guess; the mixed
// path runs its whole FP32 solve here.  A shared-memory counting sort orders
// the tile's solving quotes by that key.  Phase 2 runs the FP64 work on the
// sorted quotes, so a warp's lanes take the same guess branch, the same
// objective (and its logarithms only where that region needs them) and mostly
// the same normalised-Black branch, and non-solving quotes do not occupy lanes.
// The arithmetic of every quote is that of the unbinned solver.
// ---------------------------------------------------------------------------
constexpr int kBinKeys = 8;  // room for 4 regions x {small t, not}; bin_key uses 6

// The sort key of a solving quote: which code its FP64 work runs.  The two
// middle regions share the objective (b - beta) and the normalised-Black
// call, so they share keys; the small-t series and the erfcx form are
// different code, and so are the two wing objectives.  Keys run lowest
// (erfcx, series), middle (series, erfcx), highest (erfcx, series): the
// neighbouring bins of a tile share the normalised-Black branch where they
// can, so the warps that straddle two bins diverge less.  (Five bins ordered
// to leave one series/erfcx boundary per tile measured slower on the
// double-float tiles: mixed +2.5 % on Black-76 quotes, FP32 +1.6 %.)
__device__ __forceinline__ unsigned char bin_key(int reg, bool series) {
  const int cls = reg == 0 ? 0 : (reg == 3 ? 2 : 1);
  return (unsigned char)(cls * 2 + ((cls == 1) ? !series : series));
}

template <int THREADS, int Q, bool INLINE = false>
struct BinSmem {
  static constexpr int N = THREADS * Q;
  double beta[N], x[N], bmax[N], lnb[N], T[N];
  double cbeta[INLINE ? N : 1];  // the refined c_beta (tiles that refine in place)
  float s32[N];
  unsigned char reg[N];
  unsigned short perm[N];  // the sorted order of the solving quotes
  int cnt[kBinKeys], off[kBinKeys + 1];
};

// One tile of up to THREADS * Q quotes (THREADS = blockDim.x).  `load(li, P, SF, K, T, r, q,
// flag)` returns false past the tile's end; `out(li)` gives the index of the
// quote's sigma / status.  LATE32: the mixed path's FP32 iterations run in
// phase 2 (phase 1 only evaluates the FP32 guess that gives the sort key).
// An ill-conditioned quote (needs_refine) is not solved here: its status is
// written with kRefineMark and the refinement kernel solves it.  INLINE
// (medium batches, one launch): phase 1 refines its reduced price in place
// and the quote is binned and solved with the others, the arithmetic of the
// refinement kernel.
template <int PREC, int THREADS, int Q, bool LATE32, bool INLINE = false, typename Load>
__device__ __forceinline__ void lbr_binned_tile(BinSmem<THREADS, Q, INLINE>& sm, int model,
                                                const Load& load, double* sigma, uint8_t* status,
                                                int64_t out0) {
  const int tid = threadIdx.x;
  if (tid < kBinKeys) sm.cnt[tid] = 0;
  __syncthreads();
  unsigned char key[Q];
  unsigned short rank[Q];
#pragma unroll
  for (int k = 0; k < Q; k++) {
    const int li = k * THREADS + tid;
    key[k] = 0xff;
    rank[k] = 0;
    double P, SF, K, T, r, q;
    int flag;
    if (load(li, P, SF, K, T, r, q, flag)) {
      Norm nq = decide(model, P, SF, K, T, r, q, flag);
      const bool refine = needs_refine(nq) && !INLINE;  // left to the refinement kernel
      if (INLINE && needs_refine(nq))
        refine_reduced(model, P, SF, K, T, r, q, flag, positive64(nq.iota), nq.beta_otm, nq.c_beta);
      status[out0 + li] = (uint8_t)nq.status | (refine ? kRefineMark : 0);
      if (nq.status == Q_OK && nq.solve && !refine) {
        const Reduced<double> q64 = reduced64(nq);
        if constexpr (INLINE) sm.cbeta[li] = q64.c_beta;
        sm.beta[li] = q64.beta;
        sm.x[li] = q64.x;
        sm.bmax[li] = q64.bmax;
        sm.lnb[li] = q64.ln_beta;
        sm.T[li] = T;
        Reduced<float> q32 = reduced32(q64);
        int reg = 1;
        float sg;
        if (PREC == P_MIXED && !LATE32) {
          sg = lbr_solve<float>(q32, 2, 2, 0.0f, reg);
        } else {
          sg = lbr_guess<float>(q32, reg);
        }
        sm.s32[li] = sg;
        sm.reg[li] = (unsigned char)reg;
        // small-t class: the FP64 objective of this region takes the series
        const bool series = 0.5f * sg < (float)fvd::Prec<double>::t_small &&
                            (reg != 0 || series_in_log_space<float>(q32.x, sg));
        key[k] = bin_key(reg, series);
        rank[k] = (unsigned short)atomicAdd(&sm.cnt[key[k]], 1);
      } else if (!refine) {
        sigma[out0 + li] = nq.status == Q_OK ? 0.0 : qnan();
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int k = 0; k < kBinKeys; k++) {
      sm.off[k] = acc;
      acc += sm.cnt[k];
    }
    sm.off[kBinKeys] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < Q; k++)
    if (key[k] != 0xff) sm.perm[sm.off[key[k]] + rank[k]] = (unsigned short)(k * THREADS + tid);
  __syncthreads();
  const int ns = sm.off[kBinKeys];
  for (int j = tid; j < ns; j += THREADS) {
    const int li = sm.perm[j];
    Reduced<double> q;
    q.beta = sm.beta[li];
    q.x = sm.x[li];
    q.bmax = sm.bmax[li];
    if constexpr (INLINE)
      q.c_beta = sm.cbeta[li];
    else
      q.c_beta = q.bmax - q.beta;  // as decide computes it
    q.ln_beta = sm.lnb[li];
    q.inv_ln_beta = 0.0;
    q.ln_c_beta = 0.0;
    if (PREC == P_FP64) {
      sigma[out0 + li] = lbr_solve64(q, sm.s32[li], sm.reg[li]) * rsqrt(sm.T[li]);
    } else {
      int reg = sm.reg[li];
      float s32 = sm.s32[li];
      if (LATE32) {
        // the FP32 Householder steps from the stored guess (same region)
        Reduced<float> q32 = reduced32(q);
        wing_logs<float>(q32, reg);
        for (int it = 0; it < 2; it++)
          s32 = guarded<float>(s32, hh3_step<float>(objective<float>(q32, s32, reg)));
      }
      sigma[out0 + li] = mixed_sigma(q, s32, reg, sm.T[li]);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The mixed and FP32 solvers' tile: the status rule and reduction in
// double-float
//
// On this GPU the FP64 status rule (logarithm, exponentials, reciprocal
// square root) takes more time than the mixed solver's FP32 iterations and
// double-float correction together, and several times the FP32 solver's
// whole solve.  Pass A decides each quote with the
// double-float rule (fvdf::decide_df), which leaves to the FP64 rule the
// quotes it cannot decide with certainty: in the money (the intrinsic value
// cancels), within its guard band of a threshold, BSM log-moneyness that
// cancels, scales outside FP32's range.  Those go to a shared-memory list,
// and pass B applies the FP64 rule to the list with every thread of the block
// (packed lanes whatever the tile's mix).  Statuses are the FP64 rule's.
// Pass C evaluates the FP32 guess and the sort key of every solving quote;
// phase 2 is the binned tile's, with the reduced quote as double-float: the
// FP32 iterations, then (mixed) the double-float correction.  The FP32 path
// marks nothing for the refinement pass (its 1e-5 does not need it).
// ---------------------------------------------------------------------------
template <int THREADS, int Q, bool INLINE = false>
struct BinSmemMixed {
  static constexpr int N = THREADS * Q;
  fvdf::df beta[N], x[N], bmax[N], cbeta[N], lnb[N];
  double T[N];
  float s32[N];
  unsigned char reg[N];
  unsigned char state[N];  // 0: no root to solve here, 1: solve, 2: solve from ln beta
  unsigned short perm[N], list[N];
  unsigned short rlist[INLINE ? N : 1];  // ill-conditioned quotes refined in place
  int cnt[kBinKeys], off[kBinKeys + 1];
  int nlist, nref;
};

__device__ __forceinline__ Reduced<float> reduced32_df(const fvdf::df& beta, const fvdf::df& cbeta,
                                                       const fvdf::df& x, const fvdf::df& bmax,
                                                       const fvdf::df& lnb, bool tiny) {
  Reduced<float> f;
  f.beta = tiny ? 0.0f : beta.h;
  f.ln_beta = tiny ? lnb.h : 0.0f;
  f.c_beta = cbeta.h;
  f.x = x.h;
  f.bmax = bmax.h;
  f.inv_ln_beta = 0.0f;
  f.ln_c_beta = 0.0f;
  return f;
}

// the mixed FP64 solve of one quote (the refinement pass's arithmetic), out of
// line: only quotes whose scales leave FP32's range take it
template <int PREC>
__device__ __forceinline__ double lbr_solve_quote(const Reduced<double>& q64);
static __device__ __noinline__ double mixed_solve_fp64(Reduced<double> q64, double T) {
  return lbr_solve_quote<P_MIXED>(q64) * rsqrt(T);
}

// INLINE (medium batches, one launch): the mixed path's ill-conditioned
// quotes are not marked for the refinement kernel but listed, and phase 2
// solves them first, with the refinement kernel's arithmetic.
template <int PREC, int THREADS, int Q, bool INLINE = false, typename Load>
__device__ __forceinline__ void lbr_binned_tile_df(BinSmemMixed<THREADS, Q, INLINE>& sm, int model,
                                                      const Load& load, double* sigma,
                                                      uint8_t* status, int64_t out0) {
  using fvdf::df;
  const int tid = threadIdx.x;
  if (tid < kBinKeys) sm.cnt[tid] = 0;
  if (tid == 0) {
    sm.nlist = 0;
    sm.nref = 0;
  }
  __syncthreads();
  // pass A: the double-float status rule
#pragma unroll 1
  for (int k = 0; k < Q; k++) {
    const int li = k * THREADS + tid;
    sm.state[li] = 0;
    double P, SF, K, T, r, q;
    int flag;
    if (!load(li, P, SF, K, T, r, q, flag)) continue;
    const fvdf::NormDF d = fvdf::decide_df(model, P, SF, K, T, r, q, flag);
    if (d.fp64) {
      sm.list[atomicAdd(&sm.nlist, 1)] = (unsigned short)li;
      continue;
    }
    // ill-conditioned (mixed path) where b_max - beta < b_max/64
    const bool refine = PREC == P_MIXED && d.solve && d.c_beta.h < 0.015625f * d.bmax.h;
    if (INLINE && refine) {
      sm.rlist[atomicAdd(&sm.nref, 1)] = (unsigned short)li;
      continue;
    }
    status[out0 + li] = (uint8_t)d.status | (refine ? kRefineMark : 0);
    if (d.solve && !refine) {
      sm.beta[li] = d.beta;
      sm.x[li] = d.x;
      sm.bmax[li] = d.bmax;
      sm.cbeta[li] = d.c_beta;
      sm.lnb[li] = d.ln_beta;
      sm.T[li] = T;
      sm.state[li] = d.tiny ? 2 : 1;
    } else if (!refine) {
      sigma[out0 + li] = d.status == Q_OK ? 0.0 : qnan();
    }
  }
  __syncthreads();
  // pass B: the FP64 rule on the list, packed
  const int nl = sm.nlist;
  for (int j = tid; j < nl; j += THREADS) {
    const int li = sm.list[j];
    double P, SF, K, T, r, q;
    int flag;
    load(li, P, SF, K, T, r, q, flag);
    const Norm nq = decide(model, P, SF, K, T, r, q, flag);
    const bool refine = PREC == P_MIXED && needs_refine(nq);
    if (INLINE && refine) {
      sm.rlist[atomicAdd(&sm.nref, 1)] = (unsigned short)li;
      continue;
    }
    status[out0 + li] = (uint8_t)nq.status | (refine ? kRefineMark : 0);
    if (nq.status == Q_OK && nq.solve && !refine) {
      const Reduced<double> q64 = reduced64(nq);
      df b, x, bm, cb, T2, lb = fvdf::mk(0.0f);
      bool tiny = false, ok = fvdf::df_of0(q64.x, x) && fvdf::df_of(q64.bmax, bm) &&
                              fvdf::df_of(q64.c_beta, cb) && fvdf::df_of(T, T2);
      if (ok && !fvdf::df_of(q64.beta, b)) {
        // beta below the double-float range: carried as ln beta
        tiny = true;
        b = fvdf::mk(0.0f);
        if (q64.ln_beta != 0.0) ok = fvdf::df_of(q64.ln_beta, lb);
        else lb = fvdf::dlog_of(q64.beta);
      }
      if (ok) {
        sm.beta[li] = b;
        sm.x[li] = x;
        sm.bmax[li] = bm;
        sm.cbeta[li] = cb;
        sm.lnb[li] = lb;
        sm.T[li] = T;
        sm.state[li] = tiny ? 2 : 1;
      } else if (PREC == P_MIXED) {
        // scales outside FP32's range: the whole mixed solve in FP64 here
        sigma[out0 + li] = mixed_solve_fp64(q64, T);
      } else {
        int reg = 1;
        sigma[out0 + li] = (double)lbr_solve<float>(reduced32(q64), 2, 2, 0.0f, reg) * rsqrt(T);
      }
    } else if (!refine) {
      sigma[out0 + li] = nq.status == Q_OK ? 0.0 : qnan();
    }
  }
  __syncthreads();
  // pass C: the FP32 guess (the sort key) of every solving quote
  unsigned char key[Q];
  unsigned short rank[Q];
#pragma unroll
  for (int k = 0; k < Q; k++) {
    const int li = k * THREADS + tid;
    key[k] = 0xff;
    rank[k] = 0;
    const int stt = sm.state[li];
    if (stt != 0) {
      Reduced<float> q32 = reduced32_df(sm.beta[li], sm.cbeta[li], sm.x[li], sm.bmax[li], sm.lnb[li],
                                        stt == 2);
      int reg = 1;
      const float sg = lbr_guess<float>(q32, reg);
      sm.s32[li] = sg;
      sm.reg[li] = (unsigned char)reg;
      const bool series = 0.5f * sg < (float)fvd::Prec<double>::t_small &&
                          (reg != 0 || series_in_log_space<float>(q32.x, sg));
      key[k] = bin_key(reg, series);
      rank[k] = (unsigned short)atomicAdd(&sm.cnt[key[k]], 1);
    }
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int k = 0; k < kBinKeys; k++) {
      sm.off[k] = acc;
      acc += sm.cnt[k];
    }
    sm.off[kBinKeys] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < Q; k++)
    if (key[k] != 0xff) sm.perm[sm.off[key[k]] + rank[k]] = (unsigned short)(k * THREADS + tid);
  __syncthreads();
  // phase 2: the FP32 iterations and (mixed) the double-float correction;
  // INLINE: the listed ill-conditioned quotes first, in FP64
  const int nr = INLINE ? sm.nref : 0;
  const int ns = sm.off[kBinKeys] + nr;
  for (int j = tid; j < ns; j += THREADS) {
    if (INLINE && j < nr) {
      const int li = sm.rlist[j];
      double P, SF, K, T, r, q;
      int flag;
      load(li, P, SF, K, T, r, q, flag);
      Norm nq = decide(model, P, SF, K, T, r, q, flag);
      refine_reduced(model, P, SF, K, T, r, q, flag, positive64(nq.iota), nq.beta_otm, nq.c_beta);
      sigma[out0 + li] = mixed_solve_fp64(reduced64(nq), T);
      status[out0 + li] = (uint8_t)nq.status;
      continue;
    }
    const int li = sm.perm[j - nr];
    const bool tiny = sm.state[li] == 2;
    const df beta = sm.beta[li], x = sm.x[li], bmax = sm.bmax[li], cbeta = sm.cbeta[li],
             lnb = sm.lnb[li];
    const double T = sm.T[li];
    int reg = sm.reg[li];
    float s32 = sm.s32[li];
    Reduced<float> q32 = reduced32_df(beta, cbeta, x, bmax, lnb, tiny);
    wing_logs<float>(q32, reg);
#pragma unroll 1
    for (int it = 0; it < 2; it++)
      s32 = guarded<float>(s32, hh3_step<float>(objective<float>(q32, s32, reg)));
    df Td;
    double sig;
    if (PREC == P_FP32) {
      // sigma = s/sqrt(T) with the double-float reciprocal square root
      sigma[out0 + li] = fvdf::df_of(T, Td) ? fvdf::to_double(fvdf::dmulf(fvdf::drsqrt(Td), s32))
                                            : (double)s32 * rsqrt(T);
      continue;
    }
    if (!(fvdf::df_of(T, Td) &&
          fvdf::hh3_correction_dfv(beta, cbeta, x, lnb, tiny, Td, s32, reg, sig))) {
      // the FP64 correction from the double-float values (rare)
      const double lb = tiny ? fvdf::to_double(lnb) : 0.0;
      Reduced<double> q64;
      q64.beta = tiny ? exp(lb) : fvdf::to_double(beta);
      q64.x = fvdf::to_double(x);
      q64.bmax = fvdf::to_double(bmax);
      q64.c_beta = fvdf::to_double(cbeta);
      q64.ln_beta = lb;
      q64.inv_ln_beta = 0.0;
      q64.ln_c_beta = 0.0;
      sig = mixed_sigma_fp64(q64, s32, reg, T);
    }
    sigma[out0 + li] = sig;
  }
  __syncthreads();
}

// The FP64 LBR or mixed solve of one quote from its (refined) reduced
// values, the arithmetic phase 1 and phase 2 above apply to a tile's quote.
template <int PREC>
__device__ __forceinline__ double lbr_solve_quote(const Reduced<double>& q64) {
  Reduced<float> q32 = reduced32(q64);
  int reg = 1;
  if (PREC == P_FP64) {
    const float g = lbr_guess<float>(q32, reg);
    return lbr_solve64(q64, g, reg);
  }
  const float g = lbr_guess<float>(q32, reg);
  Reduced<float> f = reduced32(q64);
  wing_logs<float>(f, reg);
  float s32 = g;
  for (int it = 0; it < 2; it++) s32 = guarded<float>(s32, hh3_step<float>(objective<float>(f, s32, reg)));
  return hh3_correction(q64, f64_of(s32), reg);
}

}  // namespace fvk
