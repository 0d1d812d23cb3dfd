/*
 * fv.h -- C ABI of the GB300 batched implied-volatility library (libfv.so).
 *
 * The library computes, for batches of European quotes held in device memory,
 * the model price, the five Greeks, the implied volatility (Jaeckel's "Let's
 * Be Rational" or the Halley x8 solver) and the gradient of the implied
 * volatility with respect to every market input.  It follows the problem
 * statement of the fast-vollib paper: Section 2.1 (public API), Section 2.2
 * (the two solvers), Section 2.4 (Black-76 convention) and Section 3
 * (pricing models, Greeks, differentiable IV, batching).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Data pointers are DEVICE pointers owned by the caller, structure-of-arrays,
 *    one element per quote, length n.  Inputs are never written.  Any
 *    alignment is accepted.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous: they launch on `stream` and return; they never synchronise
 *    and, except where stated, allocate nothing, so they can be captured into
 *    a CUDA graph.
 *  - The implied-volatility solvers hand out work in tiles: for batches of
 *    131,072 quotes or more, the first two elements of out_sigma serve as
 *    the tile counters while the call runs (a 16-byte memset on `stream`
 *    precedes the kernel) and receive their own results last.
 *  - Models: FV_BLACK76 takes the forward F and a DISCOUNTED price, and uses
 *    the same r for discounting and inversion (Section 2.4).  FV_BLACK_SCHOLES
 *    takes the spot S with q = 0.  FV_BSM takes S and a continuous dividend
 *    yield q.  `q` may be NULL unless the model is FV_BSM.
 *  - Flags: int8, +1 call, -1 put (the "c"/"p" of Section 3); any other value
 *    makes that quote FV_Q_INVALID.
 *  - Per-quote failures never become call errors: they go to the uint8
 *    `status` array (fv_quote_status) and the quote's sigma is NaN.  A price
 *    at the intrinsic value (within a relative band of 64 * 2^-52) is
 *    FV_Q_OK with sigma = 0; a price within that band below its upper bound
 *    is FV_Q_ABOVE_MAX.
 *  - Call errors (fv_err < 0) are for arguments only (NULL required pointer,
 *    n < 0, unknown enum): the call is then rejected before any launch.  A
 *    CUDA error seen at launch, or left pending by earlier asynchronous work,
 *    returns FV_ERR_CUDA.  fv_last_error() describes the last error of the
 *    calling thread.
 *  - n = 0 is valid and launches nothing.
 *  - Every entry point opens an NVTX range named after itself for the call's
 *    duration (visible to Nsight tools; without one attached it costs
 *    nothing).  With the environment variable FV_LOG=1 each call prints its
 *    name and batch size, and each error its message, to stderr.
 */
#ifndef FV_H
#define FV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { FV_BLACK76 = 0, FV_BLACK_SCHOLES = 1, FV_BSM = 2 } fv_model;
typedef enum { FV_LBR = 0, FV_HALLEY = 1 } fv_solver;
typedef enum { FV_FP64 = 0, FV_MIXED = 1, FV_FP32 = 2 } fv_precision;
typedef enum { FV_DTYPE_F64 = 0, FV_DTYPE_F32 = 1 } fv_dtype;
typedef enum {
  FV_Q_OK = 0,              /* converged (or exactly at intrinsic: sigma = 0) */
  FV_Q_BELOW_INTRINSIC = 1, /* price below the discounted intrinsic value      */
  FV_Q_ABOVE_MAX = 2,       /* price at or above the forward / strike bound    */
  FV_Q_INVALID = 3          /* non-finite input, F|S, K, T <= 0, bad flag      */
} fv_quote_status;
typedef enum {
  FV_SUCCESS = 0,
  FV_ERR_ARG = -1,
  FV_ERR_CUDA = -2,
  FV_ERR_UNSUPPORTED = -3,
  FV_ERR_NOMEM = -4
} fv_err;

/* Model price at sigma (Section 3 "Pricing models": fast_black,
 * fast_black_scholes, fast_black_scholes_merton).
 *   P = e^{-rT} sqrt(F K) b(ln(F/K), sigma sqrt(T), flag),
 *   F = forward (Black-76) or S e^{(r-q)T}.
 * sigma = 0 gives the discounted intrinsic value.  Invalid inputs or sigma < 0
 * give NaN.  FP64 in and out. */
fv_err fv_price(fv_model model, const int8_t* flag, const double* S_or_F, const double* K,
                const double* T, const double* r, const double* q, const double* sigma, int64_t n,
                double* out_price, void* stream);

/* Implied volatility (Section 3 "Implied volatility": fast_implied_volatility
 * for BSM quotes, fast_implied_volatility_black for discounted Black-76 mids;
 * Section 2.2 for the solvers).  FP64 inputs; the status decision, every
 * residual and every Newton step in FP64 (their divisions take an FP32
 * reciprocal refined by FP64 Newton steps).
 *   FV_LBR:    normalised coordinates, four-region initial guess (built in
 *              FP32: it is ~1e-2 off and only seeds the iteration),
 *              three-branch objective, Householder(3) iteration (two steps,
 *              plus a third wherever the second still moved sigma; the
 *              step's second-order correction factor in FP32).
 *   FV_HALLEY: Brenner-Subrahmanyam guess, eight Halley sweeps on the
 *              residual, and for the quotes that fail the convergence test a
 *              fallback inside the sweeps' bracket: the LBR's rational
 *              guess, then Householder(3) steps on the LBR's transformed
 *              objective, each replaced by a bisection when it would leave
 *              the bracket.  The failures of each tile of quotes are
 *              compacted in shared memory and solved by the same kernel: no
 *              workspace, no second launch.
 * out_sigma: FP64, NaN where status != FV_Q_OK.  status: uint8 per quote. */
fv_err fv_implied_vol(fv_model model, fv_solver solver, const double* price, const double* S_or_F,
                      const double* K, const double* T, const double* r, const double* q,
                      const int8_t* flag, int64_t n, double* out_sigma, uint8_t* status,
                      void* stream);

/* Bytes of device workspace fv_implied_vol_ws needs for n quotes (0 for
 * FV_LBR). */
size_t fv_workspace_size(fv_solver solver, int64_t n);

/* fv_implied_vol with a caller-owned device workspace of at least
 * fv_workspace_size(solver, n) bytes, 16-byte aligned; allocates nothing.
 * With FV_HALLEY the sweep kernel appends the quotes that fail the
 * convergence test to a compacted list in the workspace (Section 2.2, Halley
 * item) and a second kernel runs the same fallback as fv_implied_vol over the
 * whole list; the results are those of fv_implied_vol.  The workspace's
 * contents are undefined after the call, and two calls in flight must not
 * share it.  With FV_LBR the workspace is not used (its size is 0). */
fv_err fv_implied_vol_ws(fv_model model, fv_solver solver, const double* price,
                         const double* S_or_F, const double* K, const double* T, const double* r,
                         const double* q, const int8_t* flag, int64_t n, double* out_sigma,
                         uint8_t* status, void* workspace, size_t workspace_bytes, void* stream);

/* Implied volatility with a chosen precision and input type.
 *   FV_FP64:  as fv_implied_vol.
 *   FV_MIXED: the LBR bulk in FP32 followed by one FP64 Householder(3)
 *             correction; the normalisation, status decision, intrinsic
 *             subtraction and the final residual are FP64 (result within
 *             1e-12 of the FP64 path where the quote is well conditioned).
 *   FV_FP32:  the LBR in FP32 only (relative error about 1e-5); the
 *             normalisation, status decision and intrinsic subtraction stay
 *             FP64, so the status is the FP64 rule's.
 * FV_HALLEY with FV_FP32 is the paper's throughput path for float32 label
 * pipelines (Section 2.2): eight Halley sweeps in FP32 on the direct residual
 * e^{x/2} Phi(h+t) - e^{-x/2} Phi(h-t) with plain FP32 normal CDFs, and an
 * FP32 bisection fallback on the quotes that fail the convergence test (about
 * five digits where the normalised vega exceeds 1e-8; the plain residual
 * loses the deep wings), its fallback in the same kernel as in
 * fv_implied_vol.  FV_HALLEY with FV_MIXED is FV_ERR_UNSUPPORTED.
 * in_dtype says whether price, S_or_F, K, T, r, q point to double or float.
 * out_sigma is always FP64. */
fv_err fv_implied_vol_ex(fv_model model, fv_solver solver, fv_precision precision,
                         fv_dtype in_dtype, const void* price, const void* S_or_F, const void* K,
                         const void* T, const void* r, const void* q, const int8_t* flag,
                         int64_t n, double* out_sigma, uint8_t* status, void* stream);

/* Implied volatility with strided inputs (Section 2.1: the entry points
 * accept broadcastable arrays).  `strides` is a HOST array of 7 element
 * strides for price, S_or_F, K, T, r, q and flag, in that order: quote i reads
 * element i * stride, so 0 broadcasts one value (a scalar spot, rate or
 * maturity for a whole strip) and 1 is a contiguous array.  Negative strides
 * are FV_ERR_ARG.  Outputs stay contiguous.  Otherwise as fv_implied_vol_ex. */
fv_err fv_implied_vol_strided(fv_model model, fv_solver solver, fv_precision precision,
                              fv_dtype in_dtype, const void* price, const void* S_or_F,
                              const void* K, const void* T, const void* r, const void* q,
                              const int8_t* flag, const int64_t* strides, int64_t n,
                              double* out_sigma, uint8_t* status, void* stream);

/* The five Greeks (Section 3 "Greeks": vectorized_{delta,gamma,theta,rho,vega}
 * and get_all_greeks, computed in one pass sharing d1/d2).  py_vollib scaling:
 * delta, gamma, vega per 1% of volatility, theta per calendar day (dV/dt over
 * 365), rho per 1% of rate.  Black-76 Greeks are with respect to F.  Any
 * output pointer may be NULL.  NaN unless the inputs are valid and sigma > 0. */
fv_err fv_greeks(fv_model model, const int8_t* flag, const double* S_or_F, const double* K,
                 const double* T, const double* r, const double* q, const double* sigma,
                 int64_t n, double* delta, double* gamma, double* vega, double* theta,
                 double* rho, void* stream);

/* Adjoint of the implied volatility (Section 3 "Differentiable IV"): by the
 * implicit-function theorem, d sigma / d P = 1 / vega and
 * d sigma / d x_i = -(dV/d x_i) / vega for x_i in {S|F, K, T, r, q}, with
 * vega = dV/d sigma at the given sigma (no solver iterations are stored).
 * Each output is grad_sigma times that derivative; gq is 0 unless the model is
 * FV_BSM.  All outputs are 0 where status != FV_Q_OK, sigma <= 0 or vega = 0.
 * Any output pointer may be NULL; price is read only for the Black-76 T and r
 * partials (where V = price at the root). */
fv_err fv_iv_adjoint(fv_model model, const double* price, const double* S_or_F, const double* K,
                     const double* T, const double* r, const double* q, const int8_t* flag,
                     const double* sigma, const uint8_t* status, const double* grad_sigma,
                     int64_t n, double* gP, double* gS, double* gK, double* gT, double* gr,
                     double* gq, void* stream);

/* Normalised Black function b(x, s, theta) =
 *   theta [e^{x/2} Phi(theta(x/s + s/2)) - e^{-x/2} Phi(theta(x/s - s/2))]
 * in FP64 (the evaluation of Section 2.2: erfcx form, small-t expansion); the
 * device function the solvers use.  s <= 0 gives the intrinsic value. */
fv_err fv_normalised_black(const double* x, const double* s, const int8_t* theta, int64_t n,
                           double* out, void* stream);

/* The kernels' own FP64 special functions, evaluated elementwise:
 *   FV_MATH_ERFCX  erfcx(z) = exp(z^2) erfc(z), the function the normalised
 *                  Black evaluation is built on (erfcx branch of Section 2.2);
 *                  any z (erfcx(-inf) = +inf, erfcx(+inf) = 0);
 *   FV_MATH_LOG    ln z, the logarithm of the wing objectives (Section 2.2);
 *                  ln 0 = -inf, negative z gives NaN;
 *   FV_MATH_EXP    e^z, the exponential of every normalised-Black evaluation;
 *                  0 below z = -745.2, +inf above 709.78;
 *   FV_MATH_EXPM1  e^z - 1 from the same reduction as e^z (the status rule
 *                  takes both for z = -|x|/2: bound and intrinsic value);
 *                  -1 below z = -708.3, +inf above 709.78;
 *   FV_MATH_LOG1P  ln(1 + z) as the logarithm of the exact sum 1 + z, the
 *                  form the status rule gives x = ln(F/K) near the money;
 *                  -inf at z = -1, NaN below;
 *   FV_MATH_ERFCX_SQRT2  erfcx(z/sqrt2), the form the solvers and Greeks call
 *                  (their arguments are h + t, t - h, h and |d|): the piece
 *                  index from an FP32 view of z/sqrt2, v = z/sqrt2 - c by one
 *                  FMA; any z.
 * The paper has no counterpart entry point: this exposes what the kernels
 * compute so that it can be checked on its own.  z, out: device arrays of n
 * doubles (caller-owned); NaN gives NaN.  Errors: unknown function, n < 0 or
 * a NULL pointer with n > 0 -> FV_ERR_ARG before any launch. */
typedef enum {
  FV_MATH_ERFCX = 0,
  FV_MATH_LOG = 1,
  FV_MATH_EXP = 2,
  FV_MATH_EXPM1 = 3,
  FV_MATH_LOG1P = 4,
  FV_MATH_ERFCX_SQRT2 = 5
} fv_math_fn;
fv_err fv_math(fv_math_fn which, const double* z, int64_t n, double* out, void* stream);

/* ---- batches of option chains (one persistent launch) ------------------ */
/* One chain: device arrays of n quotes sharing one forward (Black-76) or spot
 * (BSM / Black-Scholes), one maturity and one rate.  Each chain may live in
 * its own allocation. */
typedef struct {
  const double* price;  /* n discounted prices (Black-76) or prices     */
  const double* K;      /* n strikes                                    */
  const int8_t* flag;   /* n flags                                      */
  double* sigma;        /* n outputs                                    */
  uint8_t* status;      /* n outputs                                    */
  int64_t n;            /* quotes in the chain (0 allowed)              */
  double S_or_F;        /* forward (Black-76) or spot                   */
  double T;             /* maturity in years                            */
  double r;             /* rate                                         */
  double q;             /* dividend yield (FV_BSM only)                 */
} fv_chain;

typedef struct fv_chains_plan fv_chains_plan;

/* Build a plan for one batch of chains (Section 3, batching): copy the
 * descriptors and a tile table (tile -> chain, offset) to the device, choose
 * the launch shape, and capture the persistent launch (a memset of the tile
 * counter, then the kernel) into a CUDA graph.  Allocates device memory and
 * synchronises `stream`; owned by the plan.  Only FV_LBR in FP64 is
 * supported.  The chains' arrays must stay valid while the plan is used.
 *
 * Launch shape: block size x quotes per thread (64 x {1,2,4}, 128 x {1,2,4},
 * 256 x {1,2,4}, 512 x {1,2}) and resident blocks per SM (every block that
 * fits, or half of them).  autotune = 0 takes 256 x 4 at every resident
 * block.  autotune = 1 looks the workload's key up in the tuning cache (this
 * process's winners, then the file named by the environment variable
 * FV_AUTOTUNE_CACHE if set) and otherwise times every candidate on `stream`
 * (the median of three launches after one untimed launch; a few seconds on
 * tens of millions of quotes) and records the winner in both.  The
 * environment variable FV_AUTOTUNE = 0 or 1 overrides the argument.  The key
 * names the device (name, SM count), the model and floor(log2) of the chain
 * count, the quote count and the mean chain length. */
fv_err fv_chains_plan_create(fv_model model, fv_solver solver, const fv_chain* chains,
                             int64_t n_chains, int autotune, void* stream, fv_chains_plan** plan);

/* Launch the plan's graph on `stream` (one persistent launch over every
 * chain).  Allocates nothing. */
fv_err fv_implied_vol_chains(fv_chains_plan* plan, void* stream);

/* Same work without the graph: one launch of the persistent kernel. */
fv_err fv_implied_vol_chains_direct(fv_chains_plan* plan, void* stream);

/* Block size, quotes per thread, grid size and tile count the plan uses. */
fv_err fv_chains_plan_info(const fv_chains_plan* plan, int* block, int* quotes_per_thread,
                           int* grid, int64_t* tiles, int64_t* quotes);

/* How the plan's launch shape was chosen: resident blocks per SM, the source
 * (FV_TUNE_DEFAULT, FV_TUNE_TIMED, FV_TUNE_CACHED), the number of candidates
 * timed (0 unless timed), the median launch time of the chosen shape in ms
 * (as timed, or as recorded in the cache; 0 for the default) and the tuning
 * key (written to `key`, at most key_bytes bytes with the terminating NUL;
 * NULL skips it).  Any output may be NULL. */
typedef enum { FV_TUNE_DEFAULT = 0, FV_TUNE_TIMED = 1, FV_TUNE_CACHED = 2 } fv_tune_source;
fv_err fv_chains_plan_tuning(const fv_chains_plan* plan, int* blocks_per_sm, int* source,
                             int* candidates, double* best_ms, char* key, size_t key_bytes);

/* The tuning cache file (host only; no GPU needed), so that a deployment can
 * inspect it or seed it with shapes tuned elsewhere.  get: the entry for
 * `key`, or block = quotes_per_thread = blocks_per_sm = 0 and ms = 0 when the
 * file or the entry is absent.  put: adds or replaces the entry (the file is
 * rewritten through a temporary file and a rename).  Keys may not be empty
 * or hold quotes, backslashes or line breaks (FV_ERR_ARG); put also rejects
 * non-positive shapes.  A plan ignores an entry that names no compiled
 * variant and times the candidates instead. */
fv_err fv_autotune_cache_get(const char* path, const char* key, int* block, int* quotes_per_thread,
                             int* blocks_per_sm, double* ms);
fv_err fv_autotune_cache_put(const char* path, const char* key, int block, int quotes_per_thread,
                             int blocks_per_sm, double ms);

fv_err fv_chains_plan_destroy(fv_chains_plan* plan);

/* ---- host-resident batches ------------------------------------------- */
/* Section 2.1: the paper's entry points take host arrays (NumPy arrays,
 * lists, pandas columns); these calls are their form for host memory on this
 * GPU.  A stream plan holds device staging for two chunks of up to chunk_quotes
 * quotes (inputs and outputs), two CUDA streams and a 16-byte device tile
 * counter.  Created once (allocates device memory); used by
 * fv_implied_vol_host.  One call at a time per plan. */
typedef struct fv_stream_plan fv_stream_plan;
fv_err fv_stream_plan_create(int64_t chunk_quotes, fv_stream_plan** plan);
fv_err fv_stream_plan_destroy(fv_stream_plan* plan);

/* How fv_implied_vol_host moves a batch between host and GPU.
 *  - FV_TRANSFER_DIRECT: the solver reads the inputs and writes sigma and
 *    status in host memory itself, over the CPU-GPU link (NVLink-C2C on a
 *    Grace-Blackwell node), in one launch on `stream` with no staging copy.
 *    Every array must be page-locked host memory the GPU maps
 *    (cudaHostAlloc, cudaHostRegister, torch's pin_memory()); otherwise the
 *    call fails with FV_ERR_ARG before any work is queued.
 *  - FV_TRANSFER_STAGED: chunked copies through the plan's device staging,
 *    overlapped with the solve on the plan's two streams (below).
 *  - FV_TRANSFER_AUTO (a new plan's mode): DIRECT when every array is such
 *    page-locked memory, STAGED otherwise (pageable memory).
 * The solver's per-quote arithmetic is the same in both modes, so are the
 * results.  set_transfer: FV_ERR_ARG for an unknown mode.  last_transfer:
 * the mode the plan's last call took (DIRECT or STAGED; AUTO before the first
 * call), in *mode. */
typedef enum { FV_TRANSFER_AUTO = 0, FV_TRANSFER_STAGED = 1, FV_TRANSFER_DIRECT = 2 } fv_transfer;
fv_err fv_stream_plan_set_transfer(fv_stream_plan* plan, int mode);
fv_err fv_stream_plan_last_transfer(const fv_stream_plan* plan, int* mode);

/* Implied volatility of n quotes whose inputs and outputs are HOST arrays.
 * Direct mode: one launch of the solver on `stream` over the host arrays
 * (the dynamic tile counter in the plan's device memory, since the outputs
 * are not device memory).  Staged mode: the batch is cut into chunks that
 * alternate between the plan's two streams: while chunk k solves, chunk
 * k+1's inputs travel to the device and chunk k-1's sigma and status travel
 * back (page-locked memory lets the copies run concurrently with the solve;
 * pageable memory works but serialises them).  Chunks hold chunk_quotes
 * quotes except at the ends: the first three ramp up (1/8, 1/4, 1/2 of it)
 * so that the first solve starts after a short copy, and the last ones halve
 * so that the last solve and copy-out are short.  The staged pipeline starts
 * after the work already queued on `stream`, and `stream` waits for it.  In
 * both modes the outputs are in place once `stream` has completed.
 * Arguments as fv_implied_vol_ex (contiguous arrays, q may be NULL unless
 * FV_BSM). */
fv_err fv_implied_vol_host(fv_stream_plan* plan, fv_model model, fv_solver solver,
                           fv_precision precision, fv_dtype in_dtype, const void* price,
                           const void* S_or_F, const void* K, const void* T, const void* r,
                           const void* q, const int8_t* flag, int64_t n, double* out_sigma,
                           uint8_t* status, void* stream);

/* ---- implied volatility without any device allocation ----------------- */
/* The paper has no counterpart to this entry point; it serves callers that
 * may not allocate device memory (a host process that pre-reserves all of it,
 * an allocator that forbids raw cudaMalloc, a latency-critical path that
 * cannot take a first-call allocation or the synchronisation of freeing one)
 * and that want the Halley solver in its compacted-list arrangement.  It
 * runs the Halley x8 solver with its fallback exactly as fv_implied_vol_ws
 * does (the same results as fv_implied_vol), but the fallback list lives in
 * a scratch array compiled into the library: device global memory of about
 * 20 bytes per quote of capacity (about 5 MiB), held by every GPU that loads
 * the library until the process exits.
 *  - n may not exceed FV_NOALLOC_MAX_QUOTES (FV_ERR_ARG otherwise, nothing
 *    launched); split larger batches.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before capturing the stream into a CUDA graph.
 *  - Each call clears the scratch's fallback counter on `stream` before use.
 *    All calls on a device share the one array, so two calls whose GPU work
 *    overlaps (different streams, or different threads) race and give wrong
 *    results: serialise them on one stream.
 *  - Calls no cudaMalloc, no cudaFree and no other allocating routine.
 * Arguments, outputs and errors as fv_implied_vol with FV_HALLEY. */
#define FV_NOALLOC_MAX_QUOTES 262144
fv_err fv_implied_vol_halley_noalloc(fv_model model, const double* price, const double* S_or_F,
                                     const double* K, const double* T, const double* r,
                                     const double* q, const int8_t* flag, int64_t n,
                                     double* out_sigma, uint8_t* status, void* stream);

/* Error reporting. */
const char* fv_status_string(fv_err err);
const char* fv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FV_H */
