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

#include "fv_binned.cuh"
#include "fv_internal.h"

namespace fvk {

namespace {

// at most 64 registers a thread (1024 / THREADS blocks of THREADS threads on
// an SM's 65,536), and tiles of at most 1,024 quotes (48 KB of static shared
// memory)
template <int THREADS, int Q>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_chains(int model, const ChainDesc* __restrict__ chains, const Tile* __restrict__ tiles,
             int64_t n_tiles, unsigned long long* counter) {
  __shared__ BinSmem<THREADS, Q> sm;
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

using ChainsKernel = void (*)(int, const ChainDesc*, const Tile*, int64_t, unsigned long long*);

struct Variant {
  int block, qpt;
  ChainsKernel fn;
};

const Variant kVariants[] = {
    {64, 1, k_chains<64, 1>},   {64, 2, k_chains<64, 2>},   {64, 4, k_chains<64, 4>},
    {128, 1, k_chains<128, 1>}, {128, 2, k_chains<128, 2>}, {128, 4, k_chains<128, 4>},
    {256, 1, k_chains<256, 1>}, {256, 2, k_chains<256, 2>}, {256, 4, k_chains<256, 4>},
    {512, 1, k_chains<512, 1>}, {512, 2, k_chains<512, 2>},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

const Variant* find(int block, int qpt) {
  for (const Variant& v : kVariants)
    if (v.block == block && v.qpt == qpt) return &v;
  return nullptr;
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
  if (v == nullptr ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, v->fn, block, 0) != cudaSuccess || b <= 0) {
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
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  v->fn<<<grid, block, 0, st>>>(model, chains, tiles, n_tiles, counter);
  return cudaGetLastError();
}

}  // namespace fvk
