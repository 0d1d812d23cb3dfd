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
constexpr int kBinKeys = 8;  // 4 regions x {small t, not}

template <int THREADS, int Q>
struct BinSmem {
  static constexpr int N = THREADS * Q;
  double beta[N], x[N], bmax[N], lnb[N], T[N];
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
// written with kRefineMark and the refinement kernel solves it.
template <int PREC, int THREADS, int Q, bool LATE32, typename Load>
__device__ __forceinline__ void lbr_binned_tile(BinSmem<THREADS, Q>& sm, int model, const Load& load,
                                                double* sigma, uint8_t* status, int64_t out0) {
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
      const Norm nq = decide(model, P, SF, K, T, r, q, flag);
      const bool refine = needs_refine(nq);
      status[out0 + li] = (uint8_t)nq.status | (refine ? kRefineMark : 0);
      if (nq.status == Q_OK && nq.solve && !refine) {
        const Reduced<double> q64 = reduced64(nq);
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
        key[k] = (unsigned char)(reg * 2 + (series ? 1 : 0));
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
    q.c_beta = q.bmax - q.beta;
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
