// fv_abi.cu -- the extern "C" entry points declared in include/fv.h.
//
// Argument checks happen here, before any launch; the kernels live in
// fv_kernels.cu.  Nothing here synchronises except plan creation.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <unistd.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fv.h"
#include "fv_internal.h"

namespace {

thread_local char g_last_error[512] = "no error";

// FV_LOG=1 in the environment: every entry point prints its name and batch
// size, and every error its message, to stderr (read once per process)
bool log_on() {
  static const bool on = [] {
    const char* v = getenv("FV_LOG");
    return v != nullptr && v[0] != 0 && !(v[0] == '0' && v[1] == 0);
  }();
  return on;
}

// An NVTX range named after the entry point for the call's duration (seen by
// Nsight tools; without one attached NVTX does nothing), and the FV_LOG line.
struct Trace {
  Trace(const char* fn, int64_t n) {
    nvtxRangePushA(fn);
    if (log_on()) fprintf(stderr, "fv: %s n=%lld\n", fn, (long long)n);
  }
  ~Trace() { nvtxRangePop(); }
};

fv_err fail(fv_err e, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  if (log_on()) fprintf(stderr, "fv: error %d: %s\n", (int)e, g_last_error);
  return e;
}

fv_err cuda_result(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return FV_SUCCESS;
  return fail(FV_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

// A CUDA error left pending by earlier asynchronous work is reported, not lost.
fv_err pending_error(const char* where) {
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) return FV_SUCCESS;
  cudaGetLastError();
  return cuda_result(e, where);
}

bool model_ok(int m) { return m == FV_BLACK76 || m == FV_BLACK_SCHOLES || m == FV_BSM; }
bool solver_ok(int s) { return s == FV_LBR || s == FV_HALLEY; }

#define FV_REQUIRE(ptr, name, fn)                                         \
  do {                                                                    \
    if ((ptr) == nullptr) return fail(FV_ERR_ARG, "%s: %s is NULL", fn, name); \
  } while (0)

fv_err check_iv_args(const char* fn, int model, int solver, const void* P, const void* SF,
                     const void* K, const void* T, const void* r, const void* q,
                     const int8_t* flag, int64_t n, const double* sigma, const uint8_t* status) {
  if (!model_ok(model)) return fail(FV_ERR_ARG, "%s: unknown model %d", fn, model);
  if (!solver_ok(solver)) return fail(FV_ERR_ARG, "%s: unknown solver %d", fn, solver);
  if (n < 0) return fail(FV_ERR_ARG, "%s: n = %lld < 0", fn, (long long)n);
  if (n == 0) return FV_SUCCESS;
  FV_REQUIRE(P, "price", fn);
  FV_REQUIRE(SF, "S_or_F", fn);
  FV_REQUIRE(K, "K", fn);
  FV_REQUIRE(T, "T", fn);
  FV_REQUIRE(r, "r", fn);
  if (model == FV_BSM) FV_REQUIRE(q, "q", fn);
  FV_REQUIRE(flag, "flag", fn);
  FV_REQUIRE(sigma, "out_sigma", fn);
  FV_REQUIRE(status, "status", fn);
  return FV_SUCCESS;
}

// ws_path: the caller passed a workspace (fv_implied_vol_ws); the Halley
// solver then compacts its failures there and runs the fallback as a second
// kernel.  Otherwise every solver runs in one kernel without a workspace.
fv_err run_iv(const char* fn, int model, int solver, int prec, bool f32, const void* P,
              const void* SF, const void* K, const void* T, const void* r, const void* q,
              const int8_t* flag, int64_t n, double* sigma, uint8_t* status, void* ws,
              size_t ws_bytes, bool ws_path, void* stream, const int64_t* strides = nullptr) {
  Trace tr(fn, n);
  fv_err e = check_iv_args(fn, model, solver, P, SF, K, T, r, q, flag, n, sigma, status);
  if (e != FV_SUCCESS || n == 0) return e;
  if (strides)
    for (int k = 0; k < 7; k++)
      if (strides[k] < 0) return fail(FV_ERR_ARG, "%s: stride %d is negative", fn, k);
  if (solver == FV_HALLEY && prec == fvk::P_MIXED)
    return fail(FV_ERR_UNSUPPORTED, "%s: the Halley solver runs in FP64 or FP32", fn);
  const size_t need = solver == FV_HALLEY ? fvk::halley_workspace_bytes(n) : 0;
  if (solver == FV_HALLEY && ws_path) {
    if (ws == nullptr) return fail(FV_ERR_ARG, "%s: workspace is NULL", fn);
    if (ws_bytes < need)
      return fail(FV_ERR_ARG, "%s: workspace of %zu bytes, %zu needed", fn, ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(ws) % 16 != 0)
      return fail(FV_ERR_ARG, "%s: workspace not 16-byte aligned", fn);
  }
  // every argument check precedes the first CUDA call
  if ((e = pending_error(fn)) != FV_SUCCESS) return e;
  fvk::IvArgs a;
  a.model = model;
  a.f32_inputs = f32;
  a.P = P;
  a.SF = SF;
  a.K = K;
  a.T = T;
  a.r = r;
  a.q = (model == FV_BSM) ? q : nullptr;
  a.flag = flag;
  a.n = n;
  a.sigma = sigma;
  a.status = status;
  for (int k = 0; k < 7; k++) a.st[k] = strides ? strides[k] : 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (solver == FV_LBR) return cuda_result(fvk::launch_iv_lbr(a, prec, st), fn);
  if (ws_path)
    return cuda_result(prec == fvk::P_FP32 ? fvk::launch_iv_halley32_ws(a, ws, st)
                                           : fvk::launch_iv_halley_ws(a, ws, st),
                       fn);
  return cuda_result(prec == fvk::P_FP32 ? fvk::launch_iv_halley32(a, st)
                                         : fvk::launch_iv_halley(a, st),
                     fn);
}

}  // namespace

namespace fvk {
void set_last_error(const char* msg) { fail(FV_ERR_ARG, "%s", msg); }
}  // namespace fvk

// ---------------------------------------------------------------------------
// chains plan
// ---------------------------------------------------------------------------
struct fv_chains_plan {
  int model;
  int block, qpt, grid, blocks_per_sm;
  int64_t n_tiles, n_quotes;
  fvk::ChainDesc* d_chains;
  fvk::Tile* d_tiles;
  unsigned long long* d_counter;  // dynamic tile counter (zeroed before each launch)
  std::vector<fvk::ChainDesc> h_chains;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int device;
  // how the launch shape was chosen
  int source;      // FV_TUNE_DEFAULT, FV_TUNE_TIMED or FV_TUNE_CACHED
  int candidates;  // candidates timed
  double best_ms;  // median launch time of the chosen shape (timed or cached; 0 for the default)
  std::string key;
};

namespace {

fv_err build_tiles(fv_chains_plan* p, int block, int qpt, std::vector<fvk::Tile>& tiles) {
  tiles.clear();
  const int64_t tile = (int64_t)block * qpt;
  for (size_t c = 0; c < p->h_chains.size(); c++) {
    for (int64_t off = 0; off < p->h_chains[c].n; off += tile) {
      fvk::Tile t;
      t.chain = (int32_t)c;
      t.pad = 0;
      t.offset = off;
      tiles.push_back(t);
    }
  }
  return FV_SUCCESS;
}

fv_err upload_tiles(fv_chains_plan* p, const std::vector<fvk::Tile>& tiles, cudaStream_t st) {
  if (p->d_tiles) {
    cudaStreamSynchronize(st);
    cudaFree(p->d_tiles);
    p->d_tiles = nullptr;
  }
  p->n_tiles = (int64_t)tiles.size();
  if (tiles.empty()) return FV_SUCCESS;
  cudaError_t e = cudaMalloc(&p->d_tiles, tiles.size() * sizeof(fvk::Tile));
  if (e != cudaSuccess) return cuda_result(e, "fv_chains_plan_create: tile table");
  e = cudaMemcpyAsync(p->d_tiles, tiles.data(), tiles.size() * sizeof(fvk::Tile),
                      cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_result(e, "fv_chains_plan_create: tile upload");
}

int plan_grid(int blocks_per_sm, int64_t n_tiles) {
  return (int)std::min<int64_t>((int64_t)fvk::sm_count() * blocks_per_sm,
                                std::max<int64_t>(1, n_tiles));
}

// ---- the tuning cache ------------------------------------------------------
// A plan's launch shape (block size, quotes per thread, resident blocks per
// SM) is keyed by the device (name, SM count), the model and the workload's
// shape: floor(log2) of the chain count, of the quote count and of the mean
// chain length.  Winners are kept for the process and, when the environment
// variable FV_AUTOTUNE_CACHE names a file, in that file as one JSON object
// {"<key>": {"block": B, "qpt": Q, "blocks_per_sm": S, "ms": T}, ...}.
struct TuneEntry {
  int block, qpt, bps;
  double ms;
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_mem;

bool key_ok(const char* key) {
  if (key == nullptr || *key == 0) return false;
  for (const char* c = key; *c; c++)
    if (*c == '"' || *c == '\\' || *c == '\n' || *c == '\r') return false;
  return true;
}

// every entry of a cache file (an unreadable or absent file has none)
std::map<std::string, TuneEntry> cache_load(const char* path) {
  std::map<std::string, TuneEntry> out;
  FILE* f = fopen(path, "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    const char* q0 = strchr(line, '"');
    if (!q0) continue;
    const char* q1 = strstr(q0 + 1, "\": {");
    if (!q1) continue;
    TuneEntry t{0, 0, 0, 0.0};
    const char* b = strstr(q1, "\"block\":");
    const char* q = strstr(q1, "\"qpt\":");
    const char* s = strstr(q1, "\"blocks_per_sm\":");
    const char* m = strstr(q1, "\"ms\":");
    if (!b || !q || !s || sscanf(b + 8, "%d", &t.block) != 1 || sscanf(q + 6, "%d", &t.qpt) != 1 ||
        sscanf(s + 16, "%d", &t.bps) != 1)
      continue;
    if (m) sscanf(m + 5, "%lf", &t.ms);
    if (t.block <= 0 || t.qpt <= 0 || t.bps <= 0) continue;
    out[std::string(q0 + 1, q1)] = t;
  }
  fclose(f);
  return out;
}

// add or replace one entry; the file is rewritten through a temporary file
// and a rename, so a reader never sees half a file
fv_err cache_store(const char* path, const std::string& key, const TuneEntry& t) {
  std::map<std::string, TuneEntry> all = cache_load(path);
  all[key] = t;
  char tmp[4096];
  snprintf(tmp, sizeof(tmp), "%s.tmp%ld", path, (long)getpid());
  FILE* f = fopen(tmp, "w");
  if (!f) return fail(FV_ERR_ARG, "tuning cache: cannot write %s", tmp);
  fprintf(f, "{\n");
  size_t k = 0;
  for (const auto& kv : all) {
    fprintf(f, "  \"%s\": {\"block\": %d, \"qpt\": %d, \"blocks_per_sm\": %d, \"ms\": %.6f}%s\n",
            kv.first.c_str(), kv.second.block, kv.second.qpt, kv.second.bps, kv.second.ms,
            ++k < all.size() ? "," : "");
  }
  fprintf(f, "}\n");
  const bool ok = fclose(f) == 0 && rename(tmp, path) == 0;
  if (!ok) {
    remove(tmp);
    return fail(FV_ERR_ARG, "tuning cache: cannot replace %s", path);
  }
  return FV_SUCCESS;
}

int floor_log2(int64_t v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    b++;
  }
  return b;
}

std::string tune_key(int model, int64_t n_chains, int64_t n_quotes) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  char name[256] = "unknown";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    snprintf(name, sizeof(name), "%s", prop.name);
    for (char* c = name; *c; c++)
      if (*c == '"' || *c == '\\' || *c == '|') *c = '_';
  } else {
    cudaGetLastError();
  }
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d|model%d|chains2^%d|quotes2^%d|len2^%d", name, fvk::sm_count(),
           model, floor_log2(n_chains), floor_log2(n_quotes),
           floor_log2(n_chains > 0 ? n_quotes / n_chains : 0));
  return buf;
}

// FV_AUTOTUNE=0 or 1 overrides the plan's autotune argument
int autotune_setting(int requested) {
  const char* v = getenv("FV_AUTOTUNE");
  if (v && (v[0] == '0' || v[0] == '1') && v[1] == 0) return v[0] - '0';
  return requested ? 1 : 0;
}

bool variant_exists(int block, int qpt) {
  for (int k = 0; k < fvk::chains_variant_count(); k++) {
    int b, q;
    fvk::chains_variant(k, &b, &q);
    if (b == block && q == qpt) return true;
  }
  return false;
}

// median of `reps` timed launches of one shape (after one untimed launch)
fv_err time_shape(fv_chains_plan* p, int block, int qpt, int grid, cudaStream_t st, int reps,
                  double* ms_out) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_result(cudaGetLastError(), "autotune");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_result(cudaGetLastError(), "autotune");
  }
  std::vector<float> t;
  cudaError_t ce = fvk::launch_chains(p->model, p->d_chains, p->d_tiles, p->n_tiles, p->d_counter,
                                      block, qpt, grid, st);
  for (int k = 0; k < reps && ce == cudaSuccess; k++) {
    ce = cudaEventRecord(e0, st);
    if (ce == cudaSuccess)
      ce = fvk::launch_chains(p->model, p->d_chains, p->d_tiles, p->n_tiles, p->d_counter, block,
                              qpt, grid, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_result(ce, "fv_chains_plan_create: autotune");
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return FV_SUCCESS;
}

}  // namespace

extern "C" {

const char* fv_status_string(fv_err err) {
  switch (err) {
    case FV_SUCCESS: return "FV_SUCCESS";
    case FV_ERR_ARG: return "FV_ERR_ARG: invalid argument";
    case FV_ERR_CUDA: return "FV_ERR_CUDA: CUDA error";
    case FV_ERR_UNSUPPORTED: return "FV_ERR_UNSUPPORTED: unsupported combination";
    case FV_ERR_NOMEM: return "FV_ERR_NOMEM: device allocation failed";
  }
  return "unknown fv_err";
}

const char* fv_last_error(void) { return g_last_error; }

fv_err fv_price(fv_model model, const int8_t* flag, const double* S_or_F, const double* K,
                const double* T, const double* r, const double* q, const double* sigma, int64_t n,
                double* out_price, void* stream) {
  const char* fn = "fv_price";
  Trace tr(fn, n);
  if (!model_ok(model)) return fail(FV_ERR_ARG, "%s: unknown model %d", fn, (int)model);
  if (n < 0) return fail(FV_ERR_ARG, "%s: n = %lld < 0", fn, (long long)n);
  if (n == 0) return FV_SUCCESS;
  FV_REQUIRE(flag, "flag", fn);
  FV_REQUIRE(S_or_F, "S_or_F", fn);
  FV_REQUIRE(K, "K", fn);
  FV_REQUIRE(T, "T", fn);
  FV_REQUIRE(r, "r", fn);
  if (model == FV_BSM) FV_REQUIRE(q, "q", fn);
  FV_REQUIRE(sigma, "sigma", fn);
  FV_REQUIRE(out_price, "out_price", fn);
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(fvk::launch_price(model, flag, S_or_F, K, T, r, model == FV_BSM ? q : nullptr,
                                       sigma, n, out_price, static_cast<cudaStream_t>(stream)),
                     fn);
}

fv_err fv_implied_vol(fv_model model, fv_solver solver, const double* price, const double* S_or_F,
                      const double* K, const double* T, const double* r, const double* q,
                      const int8_t* flag, int64_t n, double* out_sigma, uint8_t* status,
                      void* stream) {
  return run_iv("fv_implied_vol", model, solver, fvk::P_FP64, false, price, S_or_F, K, T, r, q,
                flag, n, out_sigma, status, nullptr, 0, false, stream);
}

size_t fv_workspace_size(fv_solver solver, int64_t n) {
  if (solver != FV_HALLEY || n <= 0) return 0;
  return fvk::halley_workspace_bytes(n);
}

fv_err fv_implied_vol_ws(fv_model model, fv_solver solver, const double* price,
                         const double* S_or_F, const double* K, const double* T, const double* r,
                         const double* q, const int8_t* flag, int64_t n, double* out_sigma,
                         uint8_t* status, void* workspace, size_t workspace_bytes, void* stream) {
  return run_iv("fv_implied_vol_ws", model, solver, fvk::P_FP64, false, price, S_or_F, K, T, r, q,
                flag, n, out_sigma, status, workspace, workspace_bytes, true, stream);
}

fv_err fv_implied_vol_ex(fv_model model, fv_solver solver, fv_precision precision,
                         fv_dtype in_dtype, const void* price, const void* S_or_F, const void* K,
                         const void* T, const void* r, const void* q, const int8_t* flag,
                         int64_t n, double* out_sigma, uint8_t* status, void* stream) {
  const char* fn = "fv_implied_vol_ex";
  if (precision != FV_FP64 && precision != FV_MIXED && precision != FV_FP32)
    return fail(FV_ERR_ARG, "%s: unknown precision %d", fn, (int)precision);
  if (in_dtype != FV_DTYPE_F64 && in_dtype != FV_DTYPE_F32)
    return fail(FV_ERR_ARG, "%s: unknown input dtype %d", fn, (int)in_dtype);
  if (solver == FV_HALLEY && precision == FV_MIXED)
    return fail(FV_ERR_UNSUPPORTED, "%s: the Halley solver runs in FP64 or FP32", fn);
  return run_iv(fn, model, solver, (int)precision, in_dtype == FV_DTYPE_F32, price, S_or_F, K, T, r,
                q, flag, n, out_sigma, status, nullptr, 0, false, stream);
}

fv_err fv_implied_vol_strided(fv_model model, fv_solver solver, fv_precision precision,
                              fv_dtype in_dtype, const void* price, const void* S_or_F,
                              const void* K, const void* T, const void* r, const void* q,
                              const int8_t* flag, const int64_t* strides, int64_t n,
                              double* out_sigma, uint8_t* status, void* stream) {
  const char* fn = "fv_implied_vol_strided";
  if (precision != FV_FP64 && precision != FV_MIXED && precision != FV_FP32)
    return fail(FV_ERR_ARG, "%s: unknown precision %d", fn, (int)precision);
  if (in_dtype != FV_DTYPE_F64 && in_dtype != FV_DTYPE_F32)
    return fail(FV_ERR_ARG, "%s: unknown input dtype %d", fn, (int)in_dtype);
  if (n > 0) FV_REQUIRE(strides, "strides", fn);
  return run_iv(fn, model, solver, (int)precision, in_dtype == FV_DTYPE_F32, price, S_or_F, K, T, r,
                q, flag, n, out_sigma, status, nullptr, 0, false, stream, strides);
}

fv_err fv_greeks(fv_model model, const int8_t* flag, const double* S_or_F, const double* K,
                 const double* T, const double* r, const double* q, const double* sigma,
                 int64_t n, double* delta, double* gamma, double* vega, double* theta,
                 double* rho, void* stream) {
  const char* fn = "fv_greeks";
  Trace tr(fn, n);
  if (!model_ok(model)) return fail(FV_ERR_ARG, "%s: unknown model %d", fn, (int)model);
  if (n < 0) return fail(FV_ERR_ARG, "%s: n = %lld < 0", fn, (long long)n);
  if (n == 0) return FV_SUCCESS;
  FV_REQUIRE(flag, "flag", fn);
  FV_REQUIRE(S_or_F, "S_or_F", fn);
  FV_REQUIRE(K, "K", fn);
  FV_REQUIRE(T, "T", fn);
  FV_REQUIRE(r, "r", fn);
  if (model == FV_BSM) FV_REQUIRE(q, "q", fn);
  FV_REQUIRE(sigma, "sigma", fn);
  if (!delta && !gamma && !vega && !theta && !rho) return FV_SUCCESS;
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(fvk::launch_greeks(model, flag, S_or_F, K, T, r,
                                        model == FV_BSM ? q : nullptr, sigma, n, delta, gamma,
                                        vega, theta, rho, static_cast<cudaStream_t>(stream)),
                     fn);
}

fv_err fv_iv_adjoint(fv_model model, const double* price, const double* S_or_F, const double* K,
                     const double* T, const double* r, const double* q, const int8_t* flag,
                     const double* sigma, const uint8_t* status, const double* grad_sigma,
                     int64_t n, double* gP, double* gS, double* gK, double* gT, double* gr,
                     double* gq, void* stream) {
  const char* fn = "fv_iv_adjoint";
  Trace tr(fn, n);
  if (!model_ok(model)) return fail(FV_ERR_ARG, "%s: unknown model %d", fn, (int)model);
  if (n < 0) return fail(FV_ERR_ARG, "%s: n = %lld < 0", fn, (long long)n);
  if (n == 0) return FV_SUCCESS;
  if (model == FV_BLACK76) FV_REQUIRE(price, "price", fn);
  FV_REQUIRE(S_or_F, "S_or_F", fn);
  FV_REQUIRE(K, "K", fn);
  FV_REQUIRE(T, "T", fn);
  FV_REQUIRE(r, "r", fn);
  if (model == FV_BSM) FV_REQUIRE(q, "q", fn);
  FV_REQUIRE(flag, "flag", fn);
  FV_REQUIRE(sigma, "sigma", fn);
  FV_REQUIRE(status, "status", fn);
  FV_REQUIRE(grad_sigma, "grad_sigma", fn);
  if (!gP && !gS && !gK && !gT && !gr && !gq) return FV_SUCCESS;
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(
      fvk::launch_adjoint(model, price, S_or_F, K, T, r, model == FV_BSM ? q : nullptr, flag, sigma,
                          status, grad_sigma, n, gP, gS, gK, gT, gr, gq,
                          static_cast<cudaStream_t>(stream)),
      fn);
}

fv_err fv_normalised_black(const double* x, const double* s, const int8_t* theta, int64_t n,
                           double* out, void* stream) {
  const char* fn = "fv_normalised_black";
  Trace tr(fn, n);
  if (n < 0) return fail(FV_ERR_ARG, "%s: n = %lld < 0", fn, (long long)n);
  if (n == 0) return FV_SUCCESS;
  FV_REQUIRE(x, "x", fn);
  FV_REQUIRE(s, "s", fn);
  FV_REQUIRE(theta, "theta", fn);
  FV_REQUIRE(out, "out", fn);
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(
      fvk::launch_normalised_black(x, s, theta, n, out, static_cast<cudaStream_t>(stream)), fn);
}

fv_err fv_math(fv_math_fn which, const double* z, int64_t n, double* out, void* stream) {
  const char* fn = "fv_math";
  Trace tr(fn, n);
  if (which != FV_MATH_ERFCX && which != FV_MATH_LOG && which != FV_MATH_EXP &&
      which != FV_MATH_EXPM1 && which != FV_MATH_LOG1P && which != FV_MATH_ERFCX_SQRT2)
    return fail(FV_ERR_ARG, "%s: unknown function %d", fn, (int)which);
  if (n < 0) return fail(FV_ERR_ARG, "%s: n = %lld < 0", fn, (long long)n);
  if (n == 0) return FV_SUCCESS;
  FV_REQUIRE(z, "z", fn);
  FV_REQUIRE(out, "out", fn);
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(fvk::launch_math((int)which, z, n, out, static_cast<cudaStream_t>(stream)),
                     fn);
}

fv_err fv_chains_plan_create(fv_model model, fv_solver solver, const fv_chain* chains,
                             int64_t n_chains, int autotune, void* stream, fv_chains_plan** plan) {
  const char* fn = "fv_chains_plan_create";
  Trace tr(fn, n_chains);
  FV_REQUIRE(plan, "plan", fn);
  *plan = nullptr;
  if (!model_ok(model)) return fail(FV_ERR_ARG, "%s: unknown model %d", fn, (int)model);
  if (!solver_ok(solver)) return fail(FV_ERR_ARG, "%s: unknown solver %d", fn, (int)solver);
  if (solver != FV_LBR) return fail(FV_ERR_UNSUPPORTED, "%s: chains run the LBR solver", fn);
  if (n_chains < 0) return fail(FV_ERR_ARG, "%s: n_chains < 0", fn);
  if (n_chains > 0) FV_REQUIRE(chains, "chains", fn);
  if (n_chains >= (int64_t)1 << 31) return fail(FV_ERR_ARG, "%s: too many chains", fn);
  for (int64_t c = 0; c < n_chains; c++) {
    const fv_chain& ch = chains[c];
    if (ch.n < 0) return fail(FV_ERR_ARG, "%s: chain %lld has n < 0", fn, (long long)c);
    if (ch.n > 0 && (!ch.price || !ch.K || !ch.flag || !ch.sigma || !ch.status))
      return fail(FV_ERR_ARG, "%s: chain %lld has a NULL array", fn, (long long)c);
  }
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fv_chains_plan* p = new fv_chains_plan();
  p->model = model;
  p->d_chains = nullptr;
  p->d_tiles = nullptr;
  p->d_counter = nullptr;
  p->graph = nullptr;
  p->exec = nullptr;
  p->n_quotes = 0;
  p->n_tiles = 0;
  p->source = FV_TUNE_DEFAULT;
  p->candidates = 0;
  p->best_ms = 0.0;
  cudaGetDevice(&p->device);
  p->h_chains.resize((size_t)n_chains);
  for (int64_t c = 0; c < n_chains; c++) {
    fvk::ChainDesc& d = p->h_chains[(size_t)c];
    d.P = chains[c].price;
    d.K = chains[c].K;
    d.flag = chains[c].flag;
    d.sigma = chains[c].sigma;
    d.status = chains[c].status;
    d.n = chains[c].n;
    d.SF = chains[c].S_or_F;
    d.T = chains[c].T;
    d.r = chains[c].r;
    d.q = (model == FV_BSM) ? chains[c].q : 0.0;
    p->n_quotes += d.n;
  }
  auto cleanup = [&](fv_err err) {
    fv_chains_plan_destroy(p);
    return err;
  };
  if (n_chains > 0) {
    cudaError_t ce = cudaMalloc(&p->d_chains, (size_t)n_chains * sizeof(fvk::ChainDesc));
    if (ce != cudaSuccess) return cleanup(cuda_result(ce, "fv_chains_plan_create: descriptors"));
    ce = cudaMemcpyAsync(p->d_chains, p->h_chains.data(), (size_t)n_chains * sizeof(fvk::ChainDesc),
                         cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cleanup(cuda_result(ce, "fv_chains_plan_create: upload"));
  }
  cudaError_t ce = cudaMalloc(&p->d_counter, 16);
  if (ce != cudaSuccess) return cleanup(cuda_result(ce, "fv_chains_plan_create: tile counter"));
  p->key = tune_key(model, n_chains, p->n_quotes);
  // the default shape: 256 threads, 4 quotes per thread, every resident block
  p->block = 256;
  p->qpt = 4;
  p->blocks_per_sm = fvk::chains_max_blocks_per_sm(p->block, p->qpt);
  std::vector<fvk::Tile> tiles;
  if (p->n_quotes > 0 && autotune_setting(autotune)) {
    TuneEntry hit{0, 0, 0, 0.0};
    bool found = false;
    const char* path = getenv("FV_AUTOTUNE_CACHE");
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_mem.find(p->key);
      if (it != g_tune_mem.end()) {
        hit = it->second;
        found = true;
      } else if (path && *path) {
        const auto all = cache_load(path);
        auto jt = all.find(p->key);
        if (jt != all.end()) {
          hit = jt->second;
          found = true;
        }
      }
    }
    if (found && variant_exists(hit.block, hit.qpt)) {
      p->block = hit.block;
      p->qpt = hit.qpt;
      p->blocks_per_sm = hit.bps;
      p->best_ms = hit.ms;
      p->source = FV_TUNE_CACHED;
    } else {
      // time every variant at all its resident blocks and at half of them
      double best = 1e300;
      TuneEntry win{p->block, p->qpt, p->blocks_per_sm, 0.0};
      for (int k = 0; k < fvk::chains_variant_count(); k++) {
        int block, qpt;
        fvk::chains_variant(k, &block, &qpt);
        build_tiles(p, block, qpt, tiles);
        if ((e = upload_tiles(p, tiles, st)) != FV_SUCCESS) return cleanup(e);
        const int maxb = fvk::chains_max_blocks_per_sm(block, qpt);
        const int bps_cand[2] = {maxb, maxb / 2};
        for (int j = 0; j < 2; j++) {
          const int bps = bps_cand[j];
          if (bps < 1 || (j == 1 && bps == maxb)) continue;
          double ms = 0.0;
          if ((e = time_shape(p, block, qpt, plan_grid(bps, p->n_tiles), st, 3, &ms)) != FV_SUCCESS)
            return cleanup(e);
          p->candidates++;
          if (ms < best) {
            best = ms;
            win = TuneEntry{block, qpt, bps, ms};
          }
        }
      }
      p->block = win.block;
      p->qpt = win.qpt;
      p->blocks_per_sm = win.bps;
      p->best_ms = win.ms;
      p->source = FV_TUNE_TIMED;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_mem[p->key] = win;
      if (path && *path && (e = cache_store(path, p->key, win)) != FV_SUCCESS) return cleanup(e);
    }
  }
  build_tiles(p, p->block, p->qpt, tiles);
  if ((e = upload_tiles(p, tiles, st)) != FV_SUCCESS) return cleanup(e);
  p->grid = plan_grid(p->blocks_per_sm, p->n_tiles);
  // capture the counter reset and the persistent launch into a graph on a
  // private stream
  if (p->n_tiles > 0) {
    cudaStream_t cs;
    ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cleanup(cuda_result(ce, "fv_chains_plan_create: stream"));
    ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const cudaError_t le = fvk::launch_chains(model, p->d_chains, p->d_tiles, p->n_tiles,
                                                p->d_counter, p->block, p->qpt, p->grid, cs);
      ce = cudaStreamEndCapture(cs, &p->graph);
      if (ce == cudaSuccess) ce = le;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) return cleanup(cuda_result(ce, "fv_chains_plan_create: graph capture"));
  }
  *plan = p;
  return FV_SUCCESS;
}

fv_err fv_implied_vol_chains(fv_chains_plan* plan, void* stream) {
  const char* fn = "fv_implied_vol_chains";
  Trace tr(fn, plan ? plan->n_quotes : 0);
  FV_REQUIRE(plan, "plan", fn);
  if (plan->n_tiles == 0) return FV_SUCCESS;
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)), fn);
}

fv_err fv_implied_vol_chains_direct(fv_chains_plan* plan, void* stream) {
  const char* fn = "fv_implied_vol_chains_direct";
  Trace tr(fn, plan ? plan->n_quotes : 0);
  FV_REQUIRE(plan, "plan", fn);
  if (plan->n_tiles == 0) return FV_SUCCESS;
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  return cuda_result(fvk::launch_chains(plan->model, plan->d_chains, plan->d_tiles, plan->n_tiles,
                                        plan->d_counter, plan->block, plan->qpt, plan->grid,
                                        static_cast<cudaStream_t>(stream)),
                     fn);
}

fv_err fv_chains_plan_info(const fv_chains_plan* plan, int* block, int* quotes_per_thread,
                           int* grid, int64_t* tiles, int64_t* quotes) {
  const char* fn = "fv_chains_plan_info";
  FV_REQUIRE(plan, "plan", fn);
  if (block) *block = plan->block;
  if (quotes_per_thread) *quotes_per_thread = plan->qpt;
  if (grid) *grid = plan->grid;
  if (tiles) *tiles = plan->n_tiles;
  if (quotes) *quotes = plan->n_quotes;
  return FV_SUCCESS;
}

fv_err fv_chains_plan_tuning(const fv_chains_plan* plan, int* blocks_per_sm, int* source,
                             int* candidates, double* best_ms, char* key, size_t key_bytes) {
  const char* fn = "fv_chains_plan_tuning";
  FV_REQUIRE(plan, "plan", fn);
  if (blocks_per_sm) *blocks_per_sm = plan->blocks_per_sm;
  if (source) *source = plan->source;
  if (candidates) *candidates = plan->candidates;
  if (best_ms) *best_ms = plan->best_ms;
  if (key && key_bytes > 0) snprintf(key, key_bytes, "%s", plan->key.c_str());
  return FV_SUCCESS;
}

fv_err fv_autotune_cache_get(const char* path, const char* key, int* block, int* quotes_per_thread,
                             int* blocks_per_sm, double* ms) {
  const char* fn = "fv_autotune_cache_get";
  FV_REQUIRE(path, "path", fn);
  if (!key_ok(key)) return fail(FV_ERR_ARG, "%s: empty key or a key with quotes or newlines", fn);
  const auto all = cache_load(path);
  const auto it = all.find(key);
  const TuneEntry t = it == all.end() ? TuneEntry{0, 0, 0, 0.0} : it->second;
  if (block) *block = t.block;
  if (quotes_per_thread) *quotes_per_thread = t.qpt;
  if (blocks_per_sm) *blocks_per_sm = t.bps;
  if (ms) *ms = t.ms;
  return FV_SUCCESS;
}

fv_err fv_autotune_cache_put(const char* path, const char* key, int block, int quotes_per_thread,
                             int blocks_per_sm, double ms) {
  const char* fn = "fv_autotune_cache_put";
  FV_REQUIRE(path, "path", fn);
  if (!key_ok(key)) return fail(FV_ERR_ARG, "%s: empty key or a key with quotes or newlines", fn);
  if (block <= 0 || quotes_per_thread <= 0 || blocks_per_sm <= 0)
    return fail(FV_ERR_ARG, "%s: block, quotes per thread and blocks per SM must be positive", fn);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return cache_store(path, key, TuneEntry{block, quotes_per_thread, blocks_per_sm, ms});
}

}  // extern "C"

struct fv_stream_plan {
  int64_t chunk;
  void* in[2][6];
  int8_t* flag[2];
  double* sigma[2];
  uint8_t* status[2];
  cudaStream_t st[2];
  cudaEvent_t ev_start, ev_end[2];
  unsigned long long* ctr;  // the direct mode's two tile counters
  int transfer;             // fv_transfer
  int last_transfer;
};

extern "C" {

fv_err fv_stream_plan_destroy(fv_stream_plan* p) {
  if (!p) return FV_SUCCESS;
  for (int b = 0; b < 2; b++) {
    if (p->st[b]) cudaStreamSynchronize(p->st[b]);
    for (int j = 0; j < 6; j++)
      if (p->in[b][j]) cudaFree(p->in[b][j]);
    if (p->flag[b]) cudaFree(p->flag[b]);
    if (p->sigma[b]) cudaFree(p->sigma[b]);
    if (p->status[b]) cudaFree(p->status[b]);
    if (p->st[b]) cudaStreamDestroy(p->st[b]);
    if (p->ev_end[b]) cudaEventDestroy(p->ev_end[b]);
  }
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ctr) cudaFree(p->ctr);
  delete p;
  return FV_SUCCESS;
}

fv_err fv_stream_plan_create(int64_t chunk_quotes, fv_stream_plan** plan) {
  const char* fn = "fv_stream_plan_create";
  Trace tr(fn, chunk_quotes);
  FV_REQUIRE(plan, "plan", fn);
  *plan = nullptr;
  if (chunk_quotes <= 0) return fail(FV_ERR_ARG, "%s: chunk_quotes must be positive", fn);
  fv_err e = pending_error(fn);
  if (e != FV_SUCCESS) return e;
  fv_stream_plan* p = new fv_stream_plan();
  memset(p, 0, sizeof(*p));
  p->chunk = chunk_quotes;
  const size_t c = (size_t)chunk_quotes;
  cudaError_t ce = cudaSuccess;
  for (int b = 0; b < 2 && ce == cudaSuccess; b++) {
    for (int j = 0; j < 6 && ce == cudaSuccess; j++) ce = cudaMalloc(&p->in[b][j], c * 8);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->flag[b], c);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->sigma[b], c * 8);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->status[b], c);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&p->st[b], cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_end[b], cudaEventDisableTiming);
  }
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaMalloc(&p->ctr, 2 * sizeof(unsigned long long));
  if (ce != cudaSuccess) {
    cudaGetLastError();
    fv_stream_plan_destroy(p);
    return fail(FV_ERR_NOMEM, "%s: %s", fn, cudaGetErrorString(ce));
  }
  p->transfer = FV_TRANSFER_AUTO;
  p->last_transfer = FV_TRANSFER_AUTO;
  *plan = p;
  return FV_SUCCESS;
}

fv_err fv_stream_plan_set_transfer(fv_stream_plan* plan, int mode) {
  const char* fn = "fv_stream_plan_set_transfer";
  FV_REQUIRE(plan, "plan", fn);
  if (mode != FV_TRANSFER_AUTO && mode != FV_TRANSFER_STAGED && mode != FV_TRANSFER_DIRECT)
    return fail(FV_ERR_ARG, "%s: unknown transfer mode %d", fn, mode);
  plan->transfer = mode;
  return FV_SUCCESS;
}

fv_err fv_stream_plan_last_transfer(const fv_stream_plan* plan, int* mode) {
  const char* fn = "fv_stream_plan_last_transfer";
  FV_REQUIRE(plan, "plan", fn);
  FV_REQUIRE(mode, "mode", fn);
  *mode = plan->last_transfer;
  return FV_SUCCESS;
}

}  // extern "C"

// The address at which the GPU reads and writes host memory in place:
// page-locked memory (cudaHostAlloc, cudaHostRegister) under unified
// addressing.  nullptr for pageable, managed or device memory.
static void* mapped_view(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// one solver launch over a batch whose arrays the device addresses
static cudaError_t launch_solver(const fvk::IvArgs& a, int solver, int precision, cudaStream_t s) {
  if (solver == FV_LBR) return fvk::launch_iv_lbr(a, precision, s);
  if (precision == FV_FP32) return fvk::launch_iv_halley32(a, s);
  return fvk::launch_iv_halley(a, s);
}

// Quotes in chunk k of a host batch with `remaining` quotes left and chunks of
// up to C: the first three ramp up (C/8, C/4, C/2) so that the first solve
// starts after a short copy; once at most 2C remain the chunks halve (down to
// C/8, then the rest) so that the last solve and copy-out are short.
static int64_t host_chunk(int64_t k, int64_t remaining, int64_t C) {
  int64_t m = k < 3 ? std::max<int64_t>(C >> (3 - k), 1) : C;
  if (remaining <= 2 * C && C >= 8) {
    const int64_t half = (remaining + 1) / 2;
    m = std::min(m, half > C / 8 ? half : remaining);
  }
  return std::min(m, remaining);
}

extern "C" {

fv_err fv_implied_vol_host(fv_stream_plan* plan, fv_model model, fv_solver solver,
                           fv_precision precision, fv_dtype in_dtype, const void* price,
                           const void* S_or_F, const void* K, const void* T, const void* r,
                           const void* q, const int8_t* flag, int64_t n, double* out_sigma,
                           uint8_t* status, void* stream) {
  const char* fn = "fv_implied_vol_host";
  Trace tr(fn, n);
  FV_REQUIRE(plan, "plan", fn);
  if (precision != FV_FP64 && precision != FV_MIXED && precision != FV_FP32)
    return fail(FV_ERR_ARG, "%s: unknown precision %d", fn, (int)precision);
  if (in_dtype != FV_DTYPE_F64 && in_dtype != FV_DTYPE_F32)
    return fail(FV_ERR_ARG, "%s: unknown input dtype %d", fn, (int)in_dtype);
  fv_err e = check_iv_args(fn, model, solver, price, S_or_F, K, T, r, q, flag, n, out_sigma, status);
  if (e != FV_SUCCESS || n == 0) return e;
  if (solver == FV_HALLEY && precision == FV_MIXED)
    return fail(FV_ERR_UNSUPPORTED, "%s: the Halley solver runs in FP64 or FP32", fn);
  if ((e = pending_error(fn)) != FV_SUCCESS) return e;
  const size_t es = in_dtype == FV_DTYPE_F32 ? 4 : 8;
  const void* host_in[6] = {price, S_or_F, K, T, r, model == FV_BSM ? q : nullptr};
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (plan->transfer != FV_TRANSFER_STAGED) {
    // direct: the solver works on the host arrays in place, if the GPU maps
    // every one of them
    void* dv[6] = {};
    bool mapped = true;
    for (int j = 0; j < 6 && mapped; j++)
      if (host_in[j]) mapped = (dv[j] = mapped_view(host_in[j])) != nullptr;
    void* dflag = mapped ? mapped_view(flag) : nullptr;
    void* dsig = dflag ? mapped_view(out_sigma) : nullptr;
    void* dst = dsig ? mapped_view(status) : nullptr;
    if (dst) {
      fvk::IvArgs a;
      a.model = model;
      a.f32_inputs = in_dtype == FV_DTYPE_F32;
      a.P = dv[0];
      a.SF = dv[1];
      a.K = dv[2];
      a.T = dv[3];
      a.r = dv[4];
      a.q = dv[5];
      a.flag = static_cast<const int8_t*>(dflag);
      a.n = n;
      a.sigma = static_cast<double*>(dsig);
      a.status = static_cast<uint8_t*>(dst);
      for (int j = 0; j < 7; j++) a.st[j] = 1;
      a.ctr = plan->ctr;
      plan->last_transfer = FV_TRANSFER_DIRECT;
      return cuda_result(launch_solver(a, solver, precision, caller), fn);
    }
    if (plan->transfer == FV_TRANSFER_DIRECT)
      return fail(FV_ERR_ARG, "%s: FV_TRANSFER_DIRECT needs every array in page-locked host memory",
                  fn);
  }
  plan->last_transfer = FV_TRANSFER_STAGED;
  cudaError_t ce = cudaEventRecord(plan->ev_start, caller);
  for (int b = 0; b < 2 && ce == cudaSuccess; b++) ce = cudaStreamWaitEvent(plan->st[b], plan->ev_start, 0);
  const int64_t C = plan->chunk;
  for (int64_t k = 0, off = 0, m = 0; off < n && ce == cudaSuccess; k++, off += m) {
    const int b = (int)(k & 1);
    cudaStream_t s = plan->st[b];
    m = host_chunk(k, n - off, C);
    // buffer b's previous chunk finished on this same stream: stream order
    // keeps its outputs' copies ahead of this chunk's inputs
    for (int j = 0; j < 6 && ce == cudaSuccess; j++)
      if (host_in[j])
        ce = cudaMemcpyAsync(plan->in[b][j], static_cast<const char*>(host_in[j]) + off * es, m * es,
                             cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(plan->flag[b], flag + off, m, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) break;
    fvk::IvArgs a;
    a.model = model;
    a.f32_inputs = in_dtype == FV_DTYPE_F32;
    a.P = plan->in[b][0];
    a.SF = plan->in[b][1];
    a.K = plan->in[b][2];
    a.T = plan->in[b][3];
    a.r = plan->in[b][4];
    a.q = host_in[5] ? plan->in[b][5] : nullptr;
    a.flag = plan->flag[b];
    a.n = m;
    a.sigma = plan->sigma[b];
    a.status = plan->status[b];
    for (int j = 0; j < 7; j++) a.st[j] = 1;
    ce = launch_solver(a, solver, precision, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(out_sigma + off, plan->sigma[b], m * 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(status + off, plan->status[b], m, cudaMemcpyDeviceToHost, s);
  }
  for (int b = 0; b < 2 && ce == cudaSuccess; b++) {
    ce = cudaEventRecord(plan->ev_end[b], plan->st[b]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(caller, plan->ev_end[b], 0);
  }
  return cuda_result(ce, fn);
}

fv_err fv_chains_plan_destroy(fv_chains_plan* plan) {
  if (!plan) return FV_SUCCESS;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->d_tiles) cudaFree(plan->d_tiles);
  if (plan->d_chains) cudaFree(plan->d_chains);
  if (plan->d_counter) cudaFree(plan->d_counter);
  delete plan;
  return FV_SUCCESS;
}

}  // extern "C"
