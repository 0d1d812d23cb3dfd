// fv_internal.h -- host-side interface between the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace fvk {

enum Prec { P_FP64 = 0, P_MIXED = 1, P_FP32 = 2 };

struct IvArgs {
  int model;
  bool f32_inputs;  // price, S_or_F, K, T, r, q point to float when true
  const void *P, *SF, *K, *T, *r, *q;
  const int8_t* flag;
  int64_t n;
  double* sigma;
  uint8_t* status;
  // element strides of P, S_or_F, K, T, r, q, flag (1 = contiguous, 0 = one
  // value broadcast to every quote)
  int64_t st[7];
  // two 64-bit device counters for the dynamic tile schedule, or nullptr to
  // keep them in sigma[0..1] (outputs that live in host memory need these)
  unsigned long long* ctr = nullptr;
};

// grid sizing: blocks for n quotes, capped at `per_sm` resident blocks per SM
int sm_count();
int grid_for(int64_t n, int block, int per_sm);

// LBR: batches of kSmallBatch quotes or more run the region-binned kernel with
// dynamic tiles, whose counters are a.ctr or else the first two sigma outputs
// (zeroed on `st` before the launch), then the refinement kernel over the
// quotes it marked; medium ones (from kMidBatch[prec]) the medium-batch tiles
// below; smaller ones one unbinned kernel
cudaError_t launch_iv_lbr(const IvArgs& a, int prec, cudaStream_t st);
// Medium batches, kMidBatch[prec] <= n < 2^17 quotes: one launch of 128-quote
// region-binned tiles, one per block, that refine their ill-conditioned
// quotes themselves (launch_iv_lbr dispatches here)
constexpr int64_t kMidBatch[3] = {98304, 65536, 65536};  // FP64, mixed, FP32
cudaError_t launch_iv_lbr_mid(const IvArgs& a, int prec, cudaStream_t st);

// Halley x8 with the fallback and the double-double refinement of
// ill-conditioned quotes inside the same kernel (tile-local compaction in
// shared memory): no workspace.  Large batches zero the dynamic tile
// counters (a.ctr, else the first two sigma outputs) on `st` before the launch.
cudaError_t launch_iv_halley(const IvArgs& a, cudaStream_t st);
// Halley x8 in FP32 on the plain-Phi residual, the same arrangement
cudaError_t launch_iv_halley32(const IvArgs& a, cudaStream_t st);
// The same solvers with the failures compacted into a caller's workspace and
// a second kernel for the fallback.  Workspace layout:
// [count u32 | pad to 16][idx u32 x n | pad to 16][lo f64 x n][hi f64 x n]
size_t halley_workspace_bytes(int64_t n);
cudaError_t launch_iv_halley_ws(const IvArgs& a, void* ws, cudaStream_t st);
cudaError_t launch_iv_halley32_ws(const IvArgs& a, void* ws, cudaStream_t st);

cudaError_t launch_price(int model, const int8_t* flag, const double* SF, const double* K,
                         const double* T, const double* r, const double* q, const double* sigma,
                         int64_t n, double* out, cudaStream_t st);
cudaError_t launch_greeks(int model, const int8_t* flag, const double* SF, const double* K,
                          const double* T, const double* r, const double* q, const double* sigma,
                          int64_t n, double* delta, double* gamma, double* vega, double* theta,
                          double* rho, cudaStream_t st);
cudaError_t launch_adjoint(int model, const double* P, const double* SF, const double* K,
                           const double* T, const double* r, const double* q, const int8_t* flag,
                           const double* sigma, const uint8_t* status, const double* gsig,
                           int64_t n, double* gP, double* gS, double* gK, double* gT, double* gr,
                           double* gq, cudaStream_t st);
cudaError_t launch_normalised_black(const double* x, const double* s, const int8_t* theta,
                                    int64_t n, double* out, cudaStream_t st);
cudaError_t launch_math(int fn, const double* z, int64_t n, double* out, cudaStream_t st);

// chains: device descriptor and tile table entry
struct ChainDesc {
  const double* P;
  const double* K;
  const int8_t* flag;
  double* sigma;
  uint8_t* status;
  int64_t n;
  double SF, T, r, q;
};
struct Tile {
  int32_t chain;
  int32_t pad;
  int64_t offset;
};
// record the message fv_last_error() returns on the calling thread
void set_last_error(const char* msg);

// the chains kernel's variants (block size x quotes per thread) the plan's
// autotuner chooses from
int chains_variant_count();
void chains_variant(int k, int* block, int* quotes_per_thread);
// resident blocks of a variant on one SM (1 if the variant does not exist)
int chains_max_blocks_per_sm(int block, int quotes_per_thread);
// zero `counter` on `st`, launch the variant over the tile table, then the
// refinement kernel over the quotes it marked
cudaError_t launch_chains(int model, const ChainDesc* chains, const Tile* tiles, int64_t n_tiles,
                          unsigned long long* counter, int block, int qpt, int grid,
                          cudaStream_t st);

}  // namespace fvk
