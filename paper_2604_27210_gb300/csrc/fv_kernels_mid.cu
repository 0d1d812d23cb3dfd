// fv_kernels_mid.cu -- the LBR solvers for medium batches: from
// kMidBatch[precision] up to 2^17 quotes (kSmallBatch).
//
// Such a batch fills the GPU only once: a resident wave of large tiles would
// leave most SMs idle, while the unbinned one-quote-per-thread kernel lets
// every warp run all four LBR regions' code (alternating-flag workloads also
// send many in-the-money quotes through the FP64 status rule).  Here every
// block takes one 128-quote tile of the region-binned routine, all tiles are
// resident at once, and each tile refines its ill-conditioned quotes itself
// (the refinement kernel's arithmetic), so the call is one launch.  Measured
// on GB300 (CUDA events, 100,000 Black-76 quotes): FP64 125 -> 117 us, mixed
// 94 -> 58 us, FP32 29 -> 25 us against the unbinned kernel; below the
// kMidBatch thresholds the unbinned kernel's shorter dependent chain is faster.
// A translation unit of its own, so that nvcc compiles these instantiations
// beside the large-batch ones.
#include "fv_tiles.cuh"

namespace fvk {

namespace {

constexpr int kMidThreads = 128, kMidQ = 1, kMidMinBlocks = 8;

template <typename InT, int PREC>
cudaError_t launch_mid(const IvArgs& a, cudaStream_t st) {
  constexpr auto kernel =
      k_iv_lbr_binned<InT, PREC, kMidThreads, kMidQ, kMidMinBlocks, PREC != P_FP64, true>;
  const TileSched ts = make_sched(a, kMidThreads * kMidQ, false);  // block b: tile b
  kernel<<<(unsigned)ts.n_tiles, kMidThreads, 0, st>>>(a, ts);
  return cudaGetLastError();
}

template <typename InT>
cudaError_t launch_mid_prec(const IvArgs& a, int prec, cudaStream_t st) {
  return prec == P_FP64    ? launch_mid<InT, P_FP64>(a, st)
         : prec == P_MIXED ? launch_mid<InT, P_MIXED>(a, st)
                           : launch_mid<InT, P_FP32>(a, st);
}

}  // namespace

cudaError_t launch_iv_lbr_mid(const IvArgs& a, int prec, cudaStream_t st) {
  return a.f32_inputs ? launch_mid_prec<float>(a, prec, st) : launch_mid_prec<double>(a, prec, st);
}

}  // namespace fvk
