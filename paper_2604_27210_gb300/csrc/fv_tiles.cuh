// fv_tiles.cuh -- what the flat LBR kernels of every batch size share: the
// quote loads, the tile schedule of the persistent tiled kernels and the
// region-binned LBR kernel (fv_kernels.cu instantiates it for large batches,
// fv_kernels_mid.cu for medium ones).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fv_binned.cuh"
#include "fv_device.cuh"
#include "fv_internal.h"

namespace fvk {

using namespace fvd;

// Below kSmallBatch quotes a launch is latency-bound (each warp runs one long
// chain of dependent FP64 instructions): 64-thread blocks spread the quotes
// over as many SMs and sub-partitions as possible.  The LBR solvers skip the
// binning below kMidBatch[precision] quotes; from there to kSmallBatch they
// bin 128-quote tiles, one per block, refining ill-conditioned quotes in the
// tile (fv_kernels_mid.cu).
constexpr int64_t kSmallBatch = 1 << 17;

template <typename InT>
__device__ __forceinline__ double ld(const void* p, int64_t i) {
  return (double)__ldg(static_cast<const InT*>(p) + i);
}

// quote i of an IV call (strided / broadcast inputs)
template <typename InT>
__device__ __forceinline__ void load_quote(const IvArgs& a, int64_t i, double& P, double& SF,
                                           double& K, double& T, double& r, double& q, int& flag) {
  P = ld<InT>(a.P, i * a.st[0]);
  SF = ld<InT>(a.SF, i * a.st[1]);
  K = ld<InT>(a.K, i * a.st[2]);
  T = ld<InT>(a.T, i * a.st[3]);
  r = ld<InT>(a.r, i * a.st[4]);
  q = (a.model == M_BSM) ? ld<InT>(a.q, i * a.st[5]) : 0.0;
  flag = a.flag[i * a.st[6]];
}

// ---------------------------------------------------------------------------
// Tile scheduling of the persistent tiled kernels
//
// Static (ctr == nullptr): block b solves tile b, one tile per block (small
// batches, where the grid covers the batch).  Dynamic: one resident wave of
// blocks claims tiles from an atomic counter, so that the blocks that drew
// cheap tiles take more of them and every SM finishes at about the same time
// (a static round-robin leaves the SMs' totals a few per cent apart).  The
// two 64-bit counters -- the next tile, and the blocks that have finished --
// live in the first two outputs sigma[0], sigma[1] (8-byte aligned doubles),
// which the launcher zeroes on the stream before the launch.  Tiles cover
// quotes [kHead, n); the head quotes [0, kHead), among them sigma[0..1], are
// solved by the last block to finish, after every other block has stopped
// using the counters, so the counters cost no memory of their own.  A caller
// whose outputs are host memory read over the CPU-GPU link passes device
// counters of its own instead (IvArgs::ctr); the tiles then cover [0, n).
// No block ever waits for another.
// ---------------------------------------------------------------------------
constexpr int64_t kHead = 32;

struct TileSched {
  unsigned long long* ctr;  // nullptr: static
  int64_t n_tiles;          // tiles after the head
  int64_t head;             // kHead (counters in sigma) or 0 (static, or own counters)
};

static inline TileSched make_sched(const IvArgs& a, int tile, bool dynamic) {
  TileSched t;
  t.ctr = !dynamic ? nullptr : a.ctr ? a.ctr : reinterpret_cast<unsigned long long*>(a.sigma);
  t.head = dynamic && a.ctr == nullptr ? kHead : 0;
  t.n_tiles = (a.n - t.head + tile - 1) / tile;
  return t;
}

// Runs body(first quote, quotes in the tile) for every tile this block takes.
// Every thread of the block calls it; body may use __syncthreads().
template <typename Body>
__device__ __forceinline__ void for_each_tile(const TileSched& ts, int tile, int64_t n,
                                              const Body& body) {
  __shared__ unsigned long long s_tile;
  __shared__ int s_last;
  if (ts.ctr == nullptr) {
    const int64_t base = (int64_t)blockIdx.x * tile;
    if (base < n) body(base, (int)min((int64_t)tile, n - base));
    return;
  }
  for (;;) {
    __syncthreads();  // the previous tile's readers of s_tile are done
    if (threadIdx.x == 0) s_tile = atomicAdd(ts.ctr, 1ULL);
    __syncthreads();
    const int64_t t = (int64_t)s_tile;
    if (t >= ts.n_tiles) break;
    const int64_t base = ts.head + t * tile;
    body(base, (int)min((int64_t)tile, n - base));
  }
  if (ts.head == 0) return;  // own counters: no head to solve (uniform over the block)
  if (threadIdx.x == 0) s_last = atomicAdd(ts.ctr + 1, 1ULL) == (unsigned long long)gridDim.x - 1;
  __syncthreads();
  if (s_last) body(0, (int)min(ts.head, n));
}

// zero the counters of a dynamic schedule on the launch stream
static inline cudaError_t reset_sched(const TileSched& ts, cudaStream_t st) {
  if (ts.ctr == nullptr) return cudaSuccess;
  return cudaMemsetAsync(ts.ctr, 0, 2 * sizeof(unsigned long long), st);
}

// threads of a large batch's region-binned block
constexpr int kBinThreads = 256;

// The region-binned LBR kernel: every block walks its tiles (dynamic or one
// static tile, TileSched) through the FP64 tile (PREC = P_FP64) or the
// double-float tile (mixed and FP32) of fv_binned.cuh.  INLINE: the tile
// refines its ill-conditioned quotes itself instead of marking them for the
// refinement kernel.
template <typename InT, int PREC, int THREADS, int Q, int MINB, bool LATE32, bool INLINE>
__global__ void __launch_bounds__(THREADS, MINB) k_iv_lbr_binned(IvArgs a, TileSched ts) {
  using Smem = typename std::conditional<PREC != P_FP64, BinSmemMixed<THREADS, Q, INLINE>,
                                         BinSmem<THREADS, Q, INLINE>>::type;
  __shared__ Smem sm;
  for_each_tile(ts, THREADS * Q, a.n, [&](int64_t base, int count) {
    auto load = [&](int li, double& P, double& SF, double& K, double& T, double& r, double& q,
                    int& flag) {
      if (li >= count) return false;
      load_quote<InT>(a, base + li, P, SF, K, T, r, q, flag);
      return true;
    };
    if constexpr (PREC != P_FP64)
      lbr_binned_tile_df<PREC, THREADS, Q, INLINE>(sm, a.model, load, a.sigma, a.status, base);
    else
      lbr_binned_tile<PREC, THREADS, Q, LATE32, INLINE>(sm, a.model, load, a.sigma, a.status, base);
  });
}

}  // namespace fvk
