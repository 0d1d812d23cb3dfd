// fv_noalloc.cu -- the Halley implied-volatility entry point that allocates
// nothing.
//
// Who needs it: callers that must not call cudaMalloc at all -- code running
// under an allocator that forbids raw device allocations, processes that
// reserve all device memory up front, or real-time paths where a first-call
// allocation (and the device synchronisation that freeing an old buffer
// implies) is not acceptable.  fv_implied_vol allocates its Halley workspace
// on first use and fv_implied_vol_ws needs the caller to provide one; this
// entry point instead uses a fixed scratch array compiled into the library.
//
// The array lives in device global memory, one copy per GPU that loads the
// library, for the life of the process.  Its size bounds the batch:
// FV_NOALLOC_MAX_QUOTES quotes per call.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "fv.h"
#include "fv_internal.h"

namespace {

constexpr int64_t kMaxQuotes = FV_NOALLOC_MAX_QUOTES;
// fallback counter (16 B) + index list (4 B/quote) + bracket ends (16 B/quote)
constexpr size_t kScratchBytes = 16 + ((size_t)kMaxQuotes * 4 + 15) / 16 * 16 + (size_t)kMaxQuotes * 16;

static __device__ __align__(256) unsigned char g_halley_scratch[kScratchBytes];

// device address of g_halley_scratch, looked up once per device
std::mutex g_mu;
void* g_scratch_addr[64] = {nullptr};

fv_err fail(fv_err e, const char* msg) {
  fvk::set_last_error(msg);
  return e;
}

}  // namespace

extern "C" fv_err fv_implied_vol_halley_noalloc(fv_model model, const double* price,
                                                const double* S_or_F, const double* K,
                                                const double* T, const double* r, const double* q,
                                                const int8_t* flag, int64_t n, double* out_sigma,
                                                uint8_t* status, void* stream) {
  // a batch larger than the scratch is rejected before anything touches the
  // GPU; every other argument check is the workspace entry point's own
  if (n > kMaxQuotes) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "fv_implied_vol_halley_noalloc: n = %lld exceeds FV_NOALLOC_MAX_QUOTES = %lld",
             (long long)n, (long long)kMaxQuotes);
    return fail(FV_ERR_ARG, msg);
  }
  if (n <= 0) {
    // n = 0 and n < 0 follow fv_implied_vol_ws exactly (no GPU work)
    return fv_implied_vol_ws(model, FV_HALLEY, price, S_or_F, K, T, r, q, flag, n, out_sigma,
                             status, nullptr, 0, stream);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return fail(FV_ERR_CUDA, "fv_implied_vol_halley_noalloc: no usable current device");
  }
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
      // first call on this device: translate the array's host-side symbol
      // into its device address (the device must be current)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_halley_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return fail(FV_ERR_CUDA,
                    "fv_implied_vol_halley_noalloc: cudaGetSymbolAddress of the scratch failed");
      }
      g_scratch_addr[dev] = p;
    }
    ws = g_scratch_addr[dev];
  }
  // the Halley launcher clears the fallback counter at the start of the
  // scratch (an asynchronous memset on `stream`), then runs the two kernels
  return fv_implied_vol_ws(model, FV_HALLEY, price, S_or_F, K, T, r, q, flag, n, out_sigma,
                           status, ws, kScratchBytes, stream);
}
