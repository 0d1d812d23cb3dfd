// fv_kernels.cu -- CUDA kernels (sm_103a) of the implied-volatility library.
//
// One thread per quote, grid-stride loops over structure-of-arrays inputs (a
// warp reads 32 consecutive elements of each array: fully coalesced).  The
// work per quote is transcendental FP64 arithmetic, so the kernels are bound
// by the FP64 pipe, not by HBM; no tensor cores are involved.
#include <cuda_runtime.h>

#include <algorithm>

#include "fv_binned.cuh"
#include "fv_device.cuh"
#include "fv_internal.h"
#include "fv_tiles.cuh"

namespace fvk {

using namespace fvd;

namespace {
int g_sm_count[64] = {0};
}

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (g_sm_count[dev] <= 0) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
      c = 1;
    g_sm_count[dev] = c;
  }
  return g_sm_count[dev];
}

int grid_for(int64_t n, int block, int per_sm) {
  const int64_t need = (n + block - 1) / block;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (int)std::max<int64_t>(1, std::min(need, cap));
}

// Grid of a grid-stride kernel: one wave of resident blocks (SMs x blocks
// that fit on an SM at once, cached per device), so every block slot walks
// the same share of the units and no partial second wave leaves SMs idle;
// fewer blocks when there is less work.
template <auto Kernel>
int persistent_grid(int64_t units, int units_per_block, int block) {
  static int resident[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (resident[dev] <= 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, block, 0) != cudaSuccess || b <= 0)
      b = 1;
    resident[dev] = b;
  }
  return grid_for(units, units_per_block, resident[dev]);
}

// Launch of a one-quote-per-thread grid-stride kernel over n quotes: a small
// batch takes 64-thread blocks, one per 64 quotes, so that it reaches as many
// SMs as it can fill; a large one a single resident wave of 256-thread blocks.
template <auto Kernel, typename... Args>
void launch_shaped(int64_t n, cudaStream_t st, Args... args) {
  if (n < kSmallBatch)
    Kernel<<<grid_for(n, 64, 32), 64, 0, st>>>(args...);
  else
    Kernel<<<persistent_grid<Kernel>(n, 256, 256), 256, 0, st>>>(args...);
}

// ---------------------------------------------------------------------------
// implied volatility, LBR: FP64, mixed (FP32 bulk + one FP64 HH3 step), FP32
// ---------------------------------------------------------------------------
template <typename InT, int PREC>
__global__ void __launch_bounds__(256) k_iv_lbr(IvArgs a) {
  // unbinned: one quote per thread per round (small batches and the FP32 path)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double P, SF, K, T, r, q;
    int flag;
    load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
    Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
    // FP64 and mixed: the ill-conditioned quotes' reduced price in
    // double-double (the FP32 path's 1e-5 does not need it); the mixed path
    // takes their correction in FP64
    const bool ill = PREC == P_MIXED && needs_refine(nq);
    if (PREC != P_FP32) refine_if_needed<true>(a.model, P, SF, K, T, r, q, flag, nq);
    double sigma = qnan();
    if (nq.status == Q_OK) {
      if (!nq.solve) {
        sigma = 0.0;
      } else {
        const Reduced<double> q64 = reduced64(nq);
        int reg = 1;
        double s;
        float s32 = 0.0f;
        if (PREC == P_FP64) {
          // two Householder(3) steps, a third where the second still moved s
          // by more than 2^-17 (quartic convergence: a smaller second step
          // leaves an error far below one ulp)
          Reduced<float> q32 = reduced32(q64);
          const float g = lbr_guess<float>(q32, reg);
          s = lbr_solve64(q64, g, reg);
        } else {
          s32 = lbr_solve<float>(reduced32(q64), 2, 2, 0.0f, reg);
          s = (double)s32;
          if (PREC == P_MIXED && ill) s = hh3_correction(q64, s, reg);
        }
        // sigma = s / sqrt(T) within 1.5 ulp, one FP64 step fewer; the mixed
        // path's well-conditioned quotes take the double-float correction
        sigma = (PREC == P_MIXED && !ill) ? mixed_sigma(q64, s32, reg, T) : s * rsqrt(T);
      }
    }
    a.sigma[i] = sigma;
    a.status[i] = (uint8_t)nq.status;
  }
}


// ---------------------------------------------------------------------------
// The refinement kernel: the ill-conditioned quotes a large-batch LBR kernel
// marked (status | kRefineMark) are solved here from their double-double
// refined reduced price.  The blocks scan the status bytes in 256-quote
// chunks (chunk c to block c mod grid), append the marked quotes to a
// shared-memory list, and solve the list with every thread of the block when
// it could not take another chunk, and at the end: so a block solves up to
// 1,024 quotes at once however sparse they are (about 1 % of the benchmark
// grid's quotes, 8 % where half the quotes are in the money).  It runs on the
// same stream right after the kernel that marked them, in that kernel's
// precision PREC (FP64 or mixed).
// ---------------------------------------------------------------------------
constexpr int kRefThreads = 256, kRefList = 1024;

template <typename InT, int PREC>
__device__ __forceinline__ void refine_solve(const IvArgs& a, int64_t i) {
  double P, SF, K, T, r, q;
  int flag;
  load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
  Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
  refine_reduced(a.model, P, SF, K, T, r, q, flag, positive64(nq.iota), nq.beta_otm, nq.c_beta);
  const double s = lbr_solve_quote<PREC>(reduced64(nq));
  a.sigma[i] = s * rsqrt(T);
  a.status[i] = (uint8_t)nq.status;
}

template <typename InT, int PREC>
__global__ void __launch_bounds__(kRefThreads, 4) k_refine(IvArgs a) {
  __shared__ int64_t list[kRefList];
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int64_t chunks = (a.n + kRefThreads - 1) / kRefThreads;
  for (int64_t c = blockIdx.x;; c += gridDim.x) {
    const bool more = c < chunks;
    if (more) {
      const int64_t i = c * kRefThreads + threadIdx.x;
      if (i < a.n && (a.status[i] & kRefineMark)) list[atomicAdd(&cnt, 1)] = i;
    }
    __syncthreads();
    const int m = cnt;
    __syncthreads();  // every thread has read m: the decision below is the block's
    // solve when the list could not take another chunk, and at the end
    if (m > kRefList - kRefThreads || (!more && m > 0)) {
      for (int j = threadIdx.x; j < m; j += kRefThreads) refine_solve<InT, PREC>(a, list[j]);
      __syncthreads();
      if (threadIdx.x == 0) cnt = 0;
      __syncthreads();
    }
    if (!more) break;
  }
}

template <typename InT, int PREC>
static cudaError_t launch_refine(const IvArgs& a, cudaStream_t st) {
  constexpr auto kernel = k_refine<InT, PREC>;
  kernel<<<persistent_grid<kernel>(a.n, kRefThreads, kRefThreads), kRefThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// large batches (>= kSmallBatch quotes): dynamic tiles over one resident wave,
// then the refinement kernel; medium ones (INLINE): one tile per block, every
// tile resident at once, the ill-conditioned quotes refined in the tile
template <typename InT, int PREC, int THREADS, int Q, int MINB, bool LATE32, bool INLINE = false>
static cudaError_t launch_binned(const IvArgs& a, cudaStream_t st) {
  constexpr auto kernel = k_iv_lbr_binned<InT, PREC, THREADS, Q, MINB, LATE32, INLINE>;
  const bool dynamic = a.n >= kSmallBatch;
  const TileSched ts = make_sched(a, THREADS * Q, dynamic);
  const cudaError_t e = reset_sched(ts, st);
  if (e != cudaSuccess) return e;
  const int grid = dynamic ? persistent_grid<kernel>(a.n, THREADS * Q, THREADS) : (int)ts.n_tiles;
  kernel<<<grid, THREADS, 0, st>>>(a, ts);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return le;
  if constexpr (PREC == P_FP32 || INLINE)
    return cudaSuccess;  // nothing marked for refinement
  else
    return launch_refine<InT, PREC>(a, st);
}

// Tile shapes measured on GB300 (16.8 M quotes of the BSM grid, one resident
// wave of blocks): the FP64 solve runs 2 quotes per thread at 4 blocks per SM
// (9.39 ms; 1 x 4 9.30 ms, 3 x 4 9.32 ms, 2 x 3 9.45 ms: within 1 %, while
// 5 blocks per SM would cap the registers at 48 and spill).  The mixed and
// FP32 paths run the tile whose status rule is in double-float (2 quotes per
// thread, 4 blocks per SM; their FP32 iterations in phase 2).  Batches below
// kSmallBatch take the medium-batch tiles (fv_kernels_mid.cu) from
// kMidBatch[precision] quotes, and the unbinned kernel with 64-thread blocks
// below that.

template <typename InT, int PREC>
static void launch_flat_prec(const IvArgs& a, int block, cudaStream_t st) {
  constexpr auto kernel = k_iv_lbr<InT, PREC>;
  // small batches: one 64-thread block per 64 quotes; large: one resident wave
  const int grid = block == 256 ? persistent_grid<kernel>(a.n, block, block)
                                : grid_for(a.n, block, 2048 / block);
  kernel<<<grid, block, 0, st>>>(a);
}

template <typename InT>
static void launch_flat(const IvArgs& a, int prec, int block, cudaStream_t st) {
  if (prec == P_FP64) launch_flat_prec<InT, P_FP64>(a, block, st);
  else if (prec == P_MIXED) launch_flat_prec<InT, P_MIXED>(a, block, st);
  else launch_flat_prec<InT, P_FP32>(a, block, st);
}

cudaError_t launch_iv_lbr(const IvArgs& a, int prec, cudaStream_t st) {
  if (a.n >= kMidBatch[prec] && a.n < kSmallBatch) return launch_iv_lbr_mid(a, prec, st);
  if (a.n < kSmallBatch) {
    const int block = a.n < kSmallBatch ? 64 : 256;
    if (a.f32_inputs)
      launch_flat<float>(a, prec, block, st);
    else
      launch_flat<double>(a, prec, block, st);
    return cudaGetLastError();
  }
  if (a.f32_inputs)
    return prec == P_FP64    ? launch_binned<float, P_FP64, kBinThreads, 2, 4, false>(a, st)
           : prec == P_MIXED ? launch_binned<float, P_MIXED, kBinThreads, 2, 4, true>(a, st)
                             : launch_binned<float, P_FP32, kBinThreads, 2, 4, true>(a, st);
  return prec == P_FP64    ? launch_binned<double, P_FP64, kBinThreads, 2, 4, false>(a, st)
         : prec == P_MIXED ? launch_binned<double, P_MIXED, kBinThreads, 2, 4, true>(a, st)
                           : launch_binned<double, P_FP32, kBinThreads, 2, 4, true>(a, st);
}

// ---------------------------------------------------------------------------
// implied volatility, Halley x8 + fallback on the quotes that fail the
// convergence test (Section 2.2)
//
// Two arrangements of the same per-quote arithmetic:
//  - tiled (fv_implied_vol, the stream plan): a block sweeps a tile of quotes,
//    compacts the tile's failures into shared memory and runs the fallback
//    on them with every thread of the block, so the fallback needs no device
//    workspace and no second launch;
//  - workspace (fv_implied_vol_ws, the no-allocation entry point): the sweep
//    kernel appends the failures to a compacted list in a device workspace
//    and a second kernel runs the fallback over the whole list.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Reduced<double> reduced_of(double beta, double c_beta, double x,
                                                      double bmax, double ln_beta) {
  Reduced<double> q;
  q.beta = beta;
  q.x = x;
  q.bmax = bmax;
  q.c_beta = c_beta;
  q.ln_beta = ln_beta;
  q.inv_ln_beta = 0.0;
  q.ln_c_beta = 0.0;
  return q;
}

template <int THREADS, int Q>
struct HalleySmem {
  // per quote of the tile, at its place li: the reduced quote, the maturity
  // and the sweeps' state (iterate and bracket); then the two compacted lists
  // of places: the quotes still sweeping after their first sweep, and the
  // quotes for the fallback
  static constexpr int N = THREADS * Q;
  double beta[N], cbeta[N], x[N], bmax[N], lnb[N], T[N], s[N], lo[N], hi[N];
  unsigned short sweep[N], fall[N];
  unsigned char reg[N];  // the fallback's start region
  int n_sweep, n_fall;
  int cnt[kBinKeys], off[kBinKeys + 1];  // the fallback's counting sort
};

// A block solves a tile in three phases, each over packed lanes:
//   1. every quote: status, refinement where needed, the first sweep;
//   2. the quotes the first sweep left sweeping, compacted: the other seven;
//   3. the quotes that did not converge, compacted and sorted by the region
//      and small-t class of their start (the key of the binned LBR tile):
//      the fallback.
// On the benchmark grid 80 % of the quotes leave after the first sweep and
// about 10 % sweep on, so phase 2 keeps the long sweeps of the few converging
// quotes from holding warps whose other lanes are done.  The arithmetic of
// every quote is that of halley_solve and halley_fallback64.
template <typename InT, int THREADS, int Q>
__global__ void __launch_bounds__(THREADS, 2048 / THREADS / 2) k_iv_halley_tiled(IvArgs a, TileSched ts) {
  __shared__ HalleySmem<THREADS, Q> sm;
  // the handoff test from the first sweep on (large batches) or the second
  // (the 64-thread small-batch tiles)
  constexpr int kFirstCheck = THREADS == 64 ? 1 : 0;
  for_each_tile(ts, THREADS * Q, a.n, [&](int64_t base, int count) {
    if (threadIdx.x == 0) {
      sm.n_sweep = 0;
      sm.n_fall = 0;
    }
    if (threadIdx.x < kBinKeys) sm.cnt[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < Q; k++) {
      const int li = k * THREADS + threadIdx.x;
      if (li >= count) break;
      const int64_t i = base + li;
      double P, SF, K, T, r, q;
      int flag;
      load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
      Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
      refine_if_needed(a.model, P, SF, K, T, r, q, flag, nq);
      a.status[i] = (uint8_t)nq.status;
      double sigma = qnan();
      if (nq.status == Q_OK) {
        if (!nq.solve) {
          sigma = 0.0;
        } else {
          const Reduced<double> q64 = reduced64(nq);
          HalleyState h = halley_start(q64.beta);
          halley_sweeps(q64.beta, q64.c_beta, q64.x, q64.bmax, h, 0, 1, kFirstCheck);
          if (h.done && halley_converged(h)) {
            sigma = h.s * rsqrt(T);
          } else {
            sm.beta[li] = q64.beta;
            sm.cbeta[li] = q64.c_beta;
            sm.x[li] = q64.x;
            sm.bmax[li] = q64.bmax;
            sm.lnb[li] = q64.ln_beta;
            sm.T[li] = T;
            sm.s[li] = h.s;
            sm.lo[li] = h.lo;
            sm.hi[li] = h.hi;
            if (h.done)
              sm.fall[atomicAdd(&sm.n_fall, 1)] = (unsigned short)li;
            else
              sm.sweep[atomicAdd(&sm.n_sweep, 1)] = (unsigned short)li;
            continue;  // sigma comes from phase 2 or 3
          }
        }
      }
      a.sigma[i] = sigma;
    }
    __syncthreads();
    const int nsw = sm.n_sweep;
    for (int j = threadIdx.x; j < nsw; j += THREADS) {
      const int li = sm.sweep[j];
      HalleyState h;
      h.s = sm.s[li];
      h.lo = sm.lo[li];
      h.hi = sm.hi[li];
      h.nerr = __longlong_as_double(0x7ff0000000000000LL);
      h.done = false;
      halley_sweeps(sm.beta[li], sm.cbeta[li], sm.x[li], sm.bmax[li], h, 1, kHalleySteps,
                    kFirstCheck);
      if (halley_converged(h)) {
        a.sigma[base + li] = h.s * rsqrt(sm.T[li]);
      } else {
        sm.lo[li] = h.lo;
        sm.hi[li] = h.hi;
        sm.fall[atomicAdd(&sm.n_fall, 1)] = (unsigned short)li;
      }
    }
    __syncthreads();
    const int nf = sm.n_fall;
    unsigned char key[Q];
    unsigned short rank[Q];
#pragma unroll
    for (int k = 0; k < Q; k++) {
      const int j = k * THREADS + threadIdx.x;
      key[k] = 0xff;
      rank[k] = 0;
      if (j < nf) {
        const int li = sm.fall[j];
        int reg;
        const double g = halley_fallback_guess(
            reduced_of(sm.beta[li], sm.cbeta[li], sm.x[li], sm.bmax[li], sm.lnb[li]), reg);
        sm.s[li] = g;
        sm.reg[li] = (unsigned char)reg;
        const float gf = f32_trunc(g);
        const bool series = 0.5f * gf < (float)fvd::Prec<double>::t_small &&
                            (reg != 0 || series_in_log_space<float>(f32_trunc(sm.x[li]), gf));
        key[k] = bin_key(reg, series);
        rank[k] = (unsigned short)atomicAdd(&sm.cnt[key[k]], 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int k = 0; k < kBinKeys; k++) {
        sm.off[k] = acc;
        acc += sm.cnt[k];
      }
      sm.off[kBinKeys] = acc;
    }
    __syncthreads();
    // the sorted order of the fallback's quotes, in place of the sweep list
#pragma unroll
    for (int k = 0; k < Q; k++)
      if (key[k] != 0xff) sm.sweep[sm.off[key[k]] + rank[k]] = sm.fall[k * THREADS + threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.x; j < nf; j += THREADS) {
      const int li = sm.sweep[j];
      const double s = halley_fallback_steps(
          reduced_of(sm.beta[li], sm.cbeta[li], sm.x[li], sm.bmax[li], sm.lnb[li]), sm.s[li],
          sm.reg[li], sm.lo[li], sm.hi[li]);
      a.sigma[base + li] = s * rsqrt(sm.T[li]);
    }
    __syncthreads();
  });
}

template <int THREADS, int Q>
struct Halley32Smem {
  float beta[THREADS * Q], c_beta[THREADS * Q], x[THREADS * Q], lo[THREADS * Q], hi[THREADS * Q];
  double T[THREADS * Q];
  unsigned short li[THREADS * Q];
  int n;
};

template <typename InT, int THREADS, int Q>
__global__ void __launch_bounds__(THREADS) k_iv_halley32_tiled(IvArgs a, TileSched ts) {
  __shared__ Halley32Smem<THREADS, Q> sm;
  for_each_tile(ts, THREADS * Q, a.n, [&](int64_t base, int count) {
    if (threadIdx.x == 0) sm.n = 0;
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < Q; k++) {
      const int li = k * THREADS + threadIdx.x;
      if (li >= count) break;
      const int64_t i = base + li;
      double P, SF, K, T, r, q;
      int flag;
      load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
      const Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
      a.status[i] = (uint8_t)nq.status;
      double sigma = qnan();
      if (nq.status == Q_OK) {
        if (!nq.solve) {
          sigma = 0.0;
        } else {
          const float b32 = (float)nq.beta_otm, c32 = (float)nq.c_beta,
                      x32 = (float)nq.x_otm;
          const Halley32Out h = halley32_solve(b32, c32, x32);
          if (h.converged) {
            sigma = (double)h.s * rsqrt(T);
          } else {
            const int j = atomicAdd(&sm.n, 1);
            sm.beta[j] = b32;
            sm.c_beta[j] = c32;
            sm.x[j] = x32;
            sm.lo[j] = h.lo;
            sm.hi[j] = h.hi;
            sm.T[j] = T;
            sm.li[j] = (unsigned short)li;
            continue;
          }
        }
      }
      a.sigma[i] = sigma;
    }
    __syncthreads();
    const int nf = sm.n;
    for (int j = threadIdx.x; j < nf; j += THREADS) {
      const float s = bisect32_fallback(sm.beta[j], sm.c_beta[j], sm.x[j], sm.lo[j], sm.hi[j]);
      a.sigma[base + sm.li[j]] = (double)s * rsqrt(sm.T[j]);
    }
    __syncthreads();
  });
}

// Small batches: 64-thread blocks, one tile each (as many SMs as the batch can
// fill); large ones: 256-thread blocks of two quotes per thread, dynamic tiles
// over one resident wave.
template <typename InT>
static cudaError_t launch_halley64_tiled(const IvArgs& a, cudaStream_t st) {
  if (a.n < kSmallBatch) {
    const TileSched ts = make_sched(a, 64, false);
    k_iv_halley_tiled<InT, 64, 1><<<(unsigned)ts.n_tiles, 64, 0, st>>>(a, ts);
    return cudaGetLastError();
  }
  constexpr auto kernel = k_iv_halley_tiled<InT, 256, 2>;
  const TileSched ts = make_sched(a, 512, true);
  const cudaError_t e = reset_sched(ts, st);
  if (e != cudaSuccess) return e;
  kernel<<<persistent_grid<kernel>(a.n, 512, 256), 256, 0, st>>>(a, ts);
  return cudaGetLastError();
}

template <typename InT>
static cudaError_t launch_halley32_tiled(const IvArgs& a, cudaStream_t st) {
  if (a.n < kSmallBatch) {
    const TileSched ts = make_sched(a, 64, false);
    k_iv_halley32_tiled<InT, 64, 1><<<(unsigned)ts.n_tiles, 64, 0, st>>>(a, ts);
    return cudaGetLastError();
  }
  constexpr auto kernel = k_iv_halley32_tiled<InT, 256, 2>;
  const TileSched ts = make_sched(a, 512, true);
  const cudaError_t e = reset_sched(ts, st);
  if (e != cudaSuccess) return e;
  kernel<<<persistent_grid<kernel>(a.n, 512, 256), 256, 0, st>>>(a, ts);
  return cudaGetLastError();
}

cudaError_t launch_iv_halley(const IvArgs& a, cudaStream_t st) {
  return a.f32_inputs ? launch_halley64_tiled<float>(a, st) : launch_halley64_tiled<double>(a, st);
}

cudaError_t launch_iv_halley32(const IvArgs& a, cudaStream_t st) {
  return a.f32_inputs ? launch_halley32_tiled<float>(a, st) : launch_halley32_tiled<double>(a, st);
}

// ---- workspace arrangement ------------------------------------------------
size_t halley_workspace_bytes(int64_t n) {
  const size_t idx_bytes = ((size_t)n * 4 + 15) / 16 * 16;
  return 16 + idx_bytes + (size_t)n * 16;
}

struct HalleyWs {
  unsigned int* count;
  unsigned int* idx;
  double* lo;
  double* hi;
};

static HalleyWs halley_ws(void* ws, int64_t n) {
  char* p = static_cast<char*>(ws);
  HalleyWs w;
  w.count = reinterpret_cast<unsigned int*>(p);
  w.idx = reinterpret_cast<unsigned int*>(p + 16);
  const size_t idx_bytes = ((size_t)n * 4 + 15) / 16 * 16;
  w.lo = reinterpret_cast<double*>(p + 16 + idx_bytes);
  w.hi = w.lo + n;
  return w;
}

// warp-aggregated append of the quotes that failed the convergence test
template <typename F>
__device__ __forceinline__ void ws_append(const HalleyWs& w, bool fallback, int64_t i, F lo, F hi) {
  const unsigned active = __activemask();
  const unsigned m = __ballot_sync(active, fallback);
  if (m) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(w.count, (unsigned)__popc(m));
    base = __shfl_sync(active, base, leader);
    if (fallback) {
      const unsigned pos = base + __popc(m & ((1u << lane) - 1u));
      w.idx[pos] = (unsigned)i;
      w.lo[pos] = lo;
      w.hi[pos] = hi;
    }
  }
}

template <typename InT>
__global__ void __launch_bounds__(256) k_iv_halley(IvArgs a, HalleyWs w) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double P, SF, K, T, r, q;
    int flag;
    load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
    Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
    refine_if_needed(a.model, P, SF, K, T, r, q, flag, nq);
    double sigma = qnan();
    bool fallback = false;
    double lo = 0.0, hi = 0.0;
    if (nq.status == Q_OK) {
      if (!nq.solve) {
        sigma = 0.0;
      } else {
        const HalleyOut h = halley_solve(nq.beta_otm, nq.c_beta, nq.x_otm, nq.bmax);
        if (h.converged) {
          sigma = h.s * rsqrt(T);
        } else {
          fallback = true;
          lo = h.lo;
          hi = h.hi;
        }
      }
    }
    a.sigma[i] = sigma;
    a.status[i] = (uint8_t)nq.status;
    ws_append(w, fallback, i, lo, hi);
  }
}

template <typename InT>
__global__ void __launch_bounds__(256) k_halley_fallback(IvArgs a, HalleyWs w) {
  const int64_t cnt = (int64_t)*w.count;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += stride) {
    const int64_t i = w.idx[k];
    double P, SF, K, T, r, q;
    int flag;
    load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
    Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
    refine_if_needed(a.model, P, SF, K, T, r, q, flag, nq);
    const double s = halley_fallback64(reduced64(nq), w.lo[k], w.hi[k]);
    a.sigma[i] = s * rsqrt(T);
  }
}

template <typename InT>
__global__ void __launch_bounds__(256) k_iv_halley32(IvArgs a, HalleyWs w) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double P, SF, K, T, r, q;
    int flag;
    load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
    const Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
    double sigma = qnan();
    bool fallback = false;
    float lo = 0.0f, hi = 0.0f;
    if (nq.status == Q_OK) {
      if (!nq.solve) {
        sigma = 0.0;
      } else {
        const Halley32Out h = halley32_solve((float)nq.beta_otm, (float)nq.c_beta,
                                             (float)nq.x_otm);
        if (h.converged) {
          sigma = (double)h.s * rsqrt(T);
        } else {
          fallback = true;
          lo = h.lo;
          hi = h.hi;
        }
      }
    }
    a.sigma[i] = sigma;
    a.status[i] = (uint8_t)nq.status;
    ws_append(w, fallback, i, (double)lo, (double)hi);
  }
}

template <typename InT>
__global__ void __launch_bounds__(256) k_halley32_fallback(IvArgs a, HalleyWs w) {
  const int64_t cnt = (int64_t)*w.count;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += stride) {
    const int64_t i = w.idx[k];
    double P, SF, K, T, r, q;
    int flag;
    load_quote<InT>(a, i, P, SF, K, T, r, q, flag);
    const Norm nq = decide(a.model, P, SF, K, T, r, q, flag);
    const float s = bisect32_fallback((float)nq.beta_otm, (float)nq.c_beta,
                                      (float)nq.x_otm, (float)w.lo[k], (float)w.hi[k]);
    a.sigma[i] = (double)s * rsqrt(T);
  }
}

cudaError_t launch_iv_halley32_ws(const IvArgs& a, void* ws, cudaStream_t st) {
  const HalleyWs w = halley_ws(ws, a.n);
  cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if (a.f32_inputs) {
    launch_shaped<k_iv_halley32<float>>(a.n, st, a, w);
    launch_shaped<k_halley32_fallback<float>>(a.n, st, a, w);
  } else {
    launch_shaped<k_iv_halley32<double>>(a.n, st, a, w);
    launch_shaped<k_halley32_fallback<double>>(a.n, st, a, w);
  }
  return cudaGetLastError();
}

cudaError_t launch_iv_halley_ws(const IvArgs& a, void* ws, cudaStream_t st) {
  const HalleyWs w = halley_ws(ws, a.n);
  cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if (a.f32_inputs) {
    launch_shaped<k_iv_halley<float>>(a.n, st, a, w);
    launch_shaped<k_halley_fallback<float>>(a.n, st, a, w);
  } else {
    launch_shaped<k_iv_halley<double>>(a.n, st, a, w);
    launch_shaped<k_halley_fallback<double>>(a.n, st, a, w);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// price, Greeks, adjoint, normalised Black
// ---------------------------------------------------------------------------
// e^{-rT} sqrt(F K) for the model
__device__ __forceinline__ double price_scale(int model, double SF, double K, double T, double r,
                                              double q) {
  if (model == M_BLACK76) return exp64(-r * T) * sqrt(SF * K);
  const double qq = model == M_BSM ? q : 0.0;
  return exp64(-half64(r + qq) * T) * sqrt(SF * K);
}

__global__ void __launch_bounds__(256)
    k_price(int model, const int8_t* flag, const double* SF, const double* K, const double* T,
            const double* r, const double* q, const double* sigma, int64_t n, double* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double sf = SF[i], k = K[i], t = T[i], rr = r[i], qq = (model == M_BSM) ? q[i] : 0.0;
    const double sg = sigma[i];
    const int th = flag[i];
    double p = qnan();
    if (inputs_valid(model, sf, k, t, rr, qq, th) && isfinite(sg) && sg >= 0.0) {
      const double x = model_x(model, sf, k, t, rr, qq);
      p = price_scale(model, sf, k, t, rr, qq) * normalised_black(x, sg * sqrt(t), th);
    }
    out[i] = p;
  }
}

cudaError_t launch_price(int model, const int8_t* flag, const double* SF, const double* K,
                         const double* T, const double* r, const double* q, const double* sigma,
                         int64_t n, double* out, cudaStream_t st) {
  launch_shaped<k_price>(n, st, model, flag, SF, K, T, r, q, sigma, n, out);
  return cudaGetLastError();
}

// d1, the two normal CDFs and the density at d1, shared by Greeks and adjoint
struct D12 {
  double d1, s, N1, N2, n1;
};
// e^{-z^2/2} with z^2 split exactly into zz + zl (so the exponent's rounding
// does not grow with z^2)
__device__ __forceinline__ double gauss64(double z) {
  const double zz = z * z, zl = fma(z, z, -zz);
  const double e = exp64(-0.5 * zz);
  return fma(e, -0.5 * zl, e);
}
// Phi(z) from the table erfcx and ez = e^{-z^2/2}: the lower tail
// erfcx(|z|/sqrt2) ez / 2 (no cancellation), or one minus it above zero
__device__ __forceinline__ double ncdf64(double z, double ez) {
  const double tail = half64(erfcx64_w(fabs(z)) * ez);
  return z <= 0.0 ? tail : 1.0 - tail;
}
__device__ __forceinline__ D12 d12(double x, double s, int th) {
  D12 o;
  o.s = s;
  o.d1 = fma(x, recip64(s), half64(s));
  const double d2 = o.d1 - s;
  const double e1 = gauss64(o.d1), e2 = gauss64(d2);
  o.N1 = ncdf64(th * o.d1, e1);
  o.N2 = ncdf64(th * d2, e2);
  o.n1 = kInvSqrt2Pi * e1;
  return o;
}

__global__ void __launch_bounds__(256)
    k_greeks(int model, const int8_t* flag, const double* SF, const double* K, const double* T,
             const double* r, const double* q, const double* sigma, int64_t n, double* delta,
             double* gamma, double* vega, double* theta, double* rho) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double sf = SF[i], k = K[i], t = T[i], rr = r[i], qq = (model == M_BSM) ? q[i] : 0.0;
    const double sg = sigma[i];
    const int th = flag[i];
    double gd = qnan(), gg = qnan(), gv = qnan(), gt = qnan(), gr = qnan();
    if (inputs_valid(model, sf, k, t, rr, qq, th) && isfinite(sg) && sg > 0.0) {
      const double sq = sqrt(t), s = sg * sq;
      const double x = model_x(model, sf, k, t, rr, qq);
      const D12 d = d12(x, s, th);
      const double Dr = exp64(-rr * t);
      if (model == M_BLACK76) {
        const double V = Dr * sqrt(sf * k) * normalised_black(x, s, th);
        gd = th * Dr * d.N1;
        gg = div64(Dr * d.n1, sf * s);
        gv = sf * Dr * d.n1 * sq * 0.01;
        gt = (-sf * Dr * d.n1 * sg * half64(recip64(sq)) + rr * V) * (1.0 / 365.0);
        gr = -t * V * 0.01;
      } else {
        const double Dq = exp64(-qq * t);
        gd = th * Dq * d.N1;
        gg = div64(Dq * d.n1, sf * s);
        gv = sf * Dq * d.n1 * sq * 0.01;
        gt = (-sf * Dq * d.n1 * sg * half64(recip64(sq)) - th * rr * k * Dr * d.N2 +
              th * qq * sf * Dq * d.N1) * (1.0 / 365.0);
        gr = th * k * t * Dr * d.N2 * 0.01;
      }
    }
    if (delta) delta[i] = gd;
    if (gamma) gamma[i] = gg;
    if (vega) vega[i] = gv;
    if (theta) theta[i] = gt;
    if (rho) rho[i] = gr;
  }
}

cudaError_t launch_greeks(int model, const int8_t* flag, const double* SF, const double* K,
                          const double* T, const double* r, const double* q, const double* sigma,
                          int64_t n, double* delta, double* gamma, double* vega, double* theta,
                          double* rho, cudaStream_t st) {
  launch_shaped<k_greeks>(n, st, model, flag, SF, K, T, r, q, sigma, n, delta,
                                                     gamma, vega, theta, rho);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
    k_adjoint(int model, const double* P, const double* SF, const double* K, const double* T,
              const double* r, const double* q, const int8_t* flag, const double* sigma,
              const uint8_t* status, const double* gsig, int64_t n, double* gP, double* gS,
              double* gK, double* gT, double* gr, double* gq) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double oP = 0.0, oS = 0.0, oK = 0.0, oT = 0.0, orr = 0.0, oq = 0.0;
    const double sg = sigma[i];
    if (status[i] == Q_OK && isfinite(sg) && sg > 0.0) {
      const double sf = SF[i], k = K[i], t = T[i], rr = r[i], qq = (model == M_BSM) ? q[i] : 0.0;
      const int th = flag[i];
      if (inputs_valid(model, sf, k, t, rr, qq, th)) {
        const double sq = sqrt(t), s = sg * sq;
        const double x = model_x(model, sf, k, t, rr, qq);
        const D12 d = d12(x, s, th);
        const double Dr = exp64(-rr * t);
        double vega, VS, VK, VT, Vr, Vq = 0.0;
        if (model == M_BLACK76) {
          const double V = P[i];
          vega = sf * Dr * d.n1 * sq;
          VS = th * Dr * d.N1;
          VK = -th * Dr * d.N2;
          VT = -rr * V + Dr * sf * d.n1 * sg * half64(recip64(sq));
          Vr = -t * V;
        } else {
          const double Dq = exp64(-qq * t);
          vega = sf * Dq * d.n1 * sq;
          VS = th * Dq * d.N1;
          VK = -th * Dr * d.N2;
          VT = sf * Dq * d.n1 * sg * half64(recip64(sq)) - th * qq * sf * Dq * d.N1 +
               th * rr * k * Dr * d.N2;
          Vr = th * k * t * Dr * d.N2;
          Vq = (model == M_BSM) ? -th * sf * t * Dq * d.N1 : 0.0;
        }
        if (vega > 0.0) {
          const double g = div64(gsig[i], vega);
          oP = g;
          oS = -g * VS;
          oK = -g * VK;
          oT = -g * VT;
          orr = -g * Vr;
          oq = -g * Vq;
        }
      }
    }
    if (gP) gP[i] = oP;
    if (gS) gS[i] = oS;
    if (gK) gK[i] = oK;
    if (gT) gT[i] = oT;
    if (gr) gr[i] = orr;
    if (gq) gq[i] = oq;
  }
}

cudaError_t launch_adjoint(int model, const double* P, const double* SF, const double* K,
                           const double* T, const double* r, const double* q, const int8_t* flag,
                           const double* sigma, const uint8_t* status, const double* gsig,
                           int64_t n, double* gP, double* gS, double* gK, double* gT, double* gr,
                           double* gq, cudaStream_t st) {
  launch_shaped<k_adjoint>(n, st, model, P, SF, K, T, r, q, flag, sigma, status,
                                                      gsig, n, gP, gS, gK, gT, gr, gq);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_nb(const double* x, const double* s, const int8_t* theta,
                                            int64_t n, double* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int th = theta[i];
    const double xv = x[i], sv = s[i];
    out[i] = (th == 1 || th == -1) && isfinite(xv) && !isnan(sv) ? normalised_black(xv, sv, th)
                                                                  : qnan();
  }
}

cudaError_t launch_normalised_black(const double* x, const double* s, const int8_t* theta,
                                    int64_t n, double* out, cudaStream_t st) {
  launch_shaped<k_nb>(n, st, x, s, theta, n, out);
  return cudaGetLastError();
}

template <int FN>
__global__ void __launch_bounds__(256) k_math(const double* z, int64_t n, double* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double em1;
    const double v = z[i];
    out[i] = FN == 0   ? erfcx64(v)
             : FN == 1 ? log64(v)
             : FN == 2 ? exp64(v)
             : FN == 3 ? (exp_expm1_64(v, em1), em1)
             : FN == 4 ? log1p64(v)
                       : erfcx64_w(v);
  }
}

cudaError_t launch_math(int fn, const double* z, int64_t n, double* out, cudaStream_t st) {
  switch (fn) {
    case 0: launch_shaped<k_math<0>>(n, st, z, n, out); break;
    case 1: launch_shaped<k_math<1>>(n, st, z, n, out); break;
    case 2: launch_shaped<k_math<2>>(n, st, z, n, out); break;
    case 3: launch_shaped<k_math<3>>(n, st, z, n, out); break;
    case 4: launch_shaped<k_math<4>>(n, st, z, n, out); break;
    default: launch_shaped<k_math<5>>(n, st, z, n, out); break;
  }
  return cudaGetLastError();
}

}  // namespace fvk
