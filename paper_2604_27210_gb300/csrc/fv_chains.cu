// fv_chains.cu -- the persistent kernel over many option chains (Section 3
// "batching": many chains of uneven length in one launch).
//
// A chain's quotes share one forward / spot, maturity and rate; each chain
// may live in its own allocation and is reached through a device descriptor.
// The plan cuts every chain into tiles of block x quotes-per-thread quotes
// (a host-built table: tile -> chain, offset); one resident wave of blocks
// claims tiles from an atomic counter (zeroed by a memset node before each
// launch), so blocks that draw short or cheap tiles take more of them.  Each
// tile runs the region-binned FP64 LBR of the flat kernels.  The block size
// and quotes per thread are template parameters: the plan's autotuner times
// the variants below and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>

#include "fv_binned.cuh"
#include "fv_internal.h"

namespace fvk {

namespace {

// at most 64 registers a thread (1024 / THREADS blocks of THREADS threads on
// an SM's 65,536); the tile's binning storage (up to ~56 KB for 1,024-quote
// tiles) is dynamic shared memory, opted in per variant
template <int THREADS, int Q>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_chains(int model, const ChainDesc* __restrict__ chains, const Tile* __restrict__ tiles,
             int64_t n_tiles, unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BinSmem<THREADS, Q>& sm = *reinterpret_cast<BinSmem<THREADS, Q>*>(smem_raw);
  __shared__ unsigned long long s_tile;
  for (;;) {
    __syncthreads();  // the previous tile's readers of s_tile are done
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1ULL);
    __syncthreads();
    const int64_t tile = (int64_t)s_tile;
    if (tile >= n_tiles) break;
    const Tile tl = tiles[tile];
    const ChainDesc c = chains[tl.chain];
    auto load = [&](int li, double& P, double& SF, double& K, double& T, double& r, double& q,
                    int& flag) {
      const int64_t j = tl.offset + li;
      if (j >= c.n) return false;
      P = c.P[j];
      SF = c.SF;
      K = c.K[j];
      T = c.T;
      r = c.r;
      q = c.q;
      flag = c.flag[j];
      return true;
    };
    // sigma / status of the chain, indexed from the tile's offset
    lbr_binned_tile<P_FP64, THREADS, Q, false>(sm, model, load, c.sigma + tl.offset,
                                               c.status + tl.offset, 0);
  }
}

// The chains' ill-conditioned quotes, which the kernel above marked
// (status | kRefineMark): the blocks scan the tiles (tile t to block t mod
// grid), append the marked quotes to a shared-memory list, and solve the list
// with every thread of the block from the quotes' double-double refined
// reduced price when it could not take another tile, and at the end.
constexpr int kRefThreads = 256, kRefList = 2048;

__device__ __forceinline__ void chains_refine_solve(int model, const ChainDesc& c, int64_t k) {
  const double P = c.P[k], K = c.K[k];
  const int flag = c.flag[k];
  Norm nq = decide(model, P, c.SF, K, c.T, c.r, c.q, flag);
  refine_reduced(model, P, c.SF, K, c.T, c.r, c.q, flag, positive64(nq.iota), nq.beta_otm, nq.c_beta);
  const double s = lbr_solve_quote<P_FP64>(reduced64(nq));
  c.sigma[k] = s * rsqrt(c.T);
  c.status[k] = (uint8_t)nq.status;
}

__global__ void __launch_bounds__(kRefThreads, 4)
    k_chains_refine(int model, const ChainDesc* __restrict__ chains, const Tile* __restrict__ tiles,
                    int64_t n_tiles, int tile_quotes) {
  // a marked quote: its tile (bits 10..63) and its place in the tile (< 1,024)
  __shared__ uint64_t list[kRefList];
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int64_t t = blockIdx.x;; t += gridDim.x) {
    const bool more = t < n_tiles;
    if (more) {
      const Tile tl = tiles[t];
      const ChainDesc& c = chains[tl.chain];
      const int count = (int)min((int64_t)tile_quotes, c.n - tl.offset);
      for (int li = threadIdx.x; li < count; li += kRefThreads)
        if (c.status[tl.offset + li] & kRefineMark)
          list[atomicAdd(&cnt, 1)] = ((uint64_t)t << 10) | (uint64_t)li;
    }
    __syncthreads();
    const int m = cnt;
    __syncthreads();  // every thread has read m: the decision below is the block's
    if (m > kRefList - tile_quotes || (!more && m > 0)) {
      for (int j = threadIdx.x; j < m; j += kRefThreads) {
        const uint64_t e = list[j];
        const Tile tl = tiles[e >> 10];
        chains_refine_solve(model, chains[tl.chain], tl.offset + (int64_t)(e & 1023));
      }
      __syncthreads();
      if (threadIdx.x == 0) cnt = 0;
      __syncthreads();
    }
    if (!more) break;
  }
}

using ChainsKernel = void (*)(int, const ChainDesc*, const Tile*, int64_t, unsigned long long*);

struct Variant {
  int block, qpt;
  ChainsKernel fn;
  int smem;  // dynamic shared memory of a block
};

#define FV_CHAINS_VARIANT(B, Q) {B, Q, k_chains<B, Q>, (int)sizeof(BinSmem<B, Q>)}
const Variant kVariants[] = {
    FV_CHAINS_VARIANT(64, 1),  FV_CHAINS_VARIANT(64, 2),  FV_CHAINS_VARIANT(64, 4),
    FV_CHAINS_VARIANT(128, 1), FV_CHAINS_VARIANT(128, 2), FV_CHAINS_VARIANT(128, 4),
    FV_CHAINS_VARIANT(256, 1), FV_CHAINS_VARIANT(256, 2), FV_CHAINS_VARIANT(256, 4),
    FV_CHAINS_VARIANT(512, 1), FV_CHAINS_VARIANT(512, 2),
};
#undef FV_CHAINS_VARIANT
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

const Variant* find(int block, int qpt) {
  for (const Variant& v : kVariants)
    if (v.block == block && v.qpt == qpt) return &v;
  return nullptr;
}

// allow the variant's dynamic shared memory on the current device (once per
// device and variant; a host call, not a stream operation)
cudaError_t opt_in(const Variant* v) {
  static bool done[64][kNumVariants] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int k = (int)(v - kVariants);
  if (dev >= 0 && dev < 64 && done[dev][k]) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v->smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev][k] = true;
  return e;
}

}  // namespace

int chains_variant_count() { return kNumVariants; }

void chains_variant(int k, int* block, int* qpt) {
  *block = kVariants[k].block;
  *qpt = kVariants[k].qpt;
}

int chains_max_blocks_per_sm(int block, int qpt) {
  const Variant* v = find(block, qpt);
  int b = 0;
  if (v == nullptr || opt_in(v) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, v->fn, block, v->smem) != cudaSuccess ||
      b <= 0) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}

cudaError_t launch_chains(int model, const ChainDesc* chains, const Tile* tiles, int64_t n_tiles,
                          unsigned long long* counter, int block, int qpt, int grid,
                          cudaStream_t st) {
  const Variant* v = find(block, qpt);
  if (v == nullptr || grid <= 0) return cudaErrorInvalidValue;
  cudaError_t e = opt_in(v);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  v->fn<<<grid, block, v->smem, st>>>(model, chains, tiles, n_tiles, counter);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int rgrid = (int)std::min<int64_t>((int64_t)sm_count() * 4, n_tiles);
  k_chains_refine<<<rgrid, kRefThreads, 0, st>>>(model, chains, tiles, n_tiles, block * qpt);
  return cudaGetLastError();
}

}  // namespace fvk
