/*
 * love.h -- C ABI of the GB300 (sm_103a) implementation of LOVE
 * (LanczOs Variance Estimates) for KISS-GP.
 *
 * Paper: Pleiss, Gardner, Weinberger, Wilson, "Constant-Time Predictive
 * Distributions for Gaussian Processes", ICML 2018.
 *
 * Phases follow the paper's pre-compute / test split (Sec. 3, "pre-compute
 * phase and test phase"):
 *   ski_build              KISS-GP structure of the training set (Sec. 2.3, eq. ski)
 *   love_precompute        Lanczos on W^T K_UU W + s^2 I, caches (Sec. 3.2, Algorithm 1)
 *   love_predict_mean_var  O(k) predictive mean and variance (eqs. pred_mean_ski,
 *                          pred_covar_ski_fast; Algorithm 1)
 *   love_sample            posterior samples via the low-rank root (Sec. 3.3, eq. sample)
 *   love_var_backward      vector-Jacobian product of the variances (not in the
 *                          paper; derived from eq. pred_covar_ski_cache)
 *
 * Conventions shared by every entry point
 *   - Pointers named x_*, y_*, v, out, mean, var, grad_* are DEVICE pointers
 *     owned by the caller unless the comment says "host".  They must stay valid
 *     until the work enqueued on `stream` has finished.
 *   - Arrays are dense, row-major, with the element type of the handle's dtype
 *     (LOVE_F32 -> float, LOVE_F64 -> double).  Point sets are t x d (d = dim).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     stream-ordered and asynchronous unless stated.
 *   - Every call returns a love_status; no C++ exception crosses the ABI.
 *     Argument and launch errors are returned synchronously.  Errors found by
 *     a kernel (a point outside the interpolable grid, a NaN, a non-positive
 *     Cholesky pivot, an expired bounded wait) are recorded in the handle's
 *     device status word, read by love_get_device_status().
 *   - Handles are not safe for concurrent use from several host threads.
 */
#ifndef LOVE_H_
#define LOVE_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LOVE_API __attribute__((visibility("default")))
#else
#define LOVE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* love_stream_t;   /* == cudaStream_t */

typedef enum {
  LOVE_OK = 0,
  LOVE_ERR_ARG = 1,        /* invalid argument (NULL, size, dim, dtype)            */
  LOVE_ERR_DOMAIN = 2,     /* a point whose 4-point stencil leaves the grid, or NaN */
  LOVE_ERR_NOT_PD = 3,     /* non-positive pivot in the tridiagonal Cholesky        */
  LOVE_ERR_NAN = 4,        /* NaN/Inf met in a reduction                            */
  LOVE_ERR_OOM = 5,        /* allocation failed (device or host memory, host thread) */
  LOVE_ERR_CUDA = 6,       /* a CUDA runtime error (see love_last_cuda_error)       */
  LOVE_ERR_TIMEOUT = 7,    /* a bounded device wait expired                         */
  LOVE_ERR_STATE = 8,      /* the handle lacks what the call needs                  */
  LOVE_ERR_UNSUPPORTED = 9 /* configuration outside what this library implements    */
} love_status;

typedef enum { LOVE_F32 = 0, LOVE_F64 = 1, LOVE_BF16 = 2 } love_dtype;

/* Device-memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes usable on `stream` (NULL on failure -> LOVE_ERR_OOM); free releases it.
 * With a NULL allocator the library uses cudaMallocAsync / cudaFreeAsync. */
typedef struct {
  void* (*alloc)(void* ctx, size_t bytes, love_stream_t stream);
  void (*free)(void* ctx, void* ptr, size_t bytes, love_stream_t stream);
  void* ctx;
} love_allocator;

/* KISS-GP description (Sec. 2.3).  The grid of dimension e has grid_size[e]
 * points at grid_lo[e] + j h_e, h_e = (grid_hi[e] - grid_lo[e]) / (grid_size[e]-1);
 * the grid linear index is row-major over dimensions (last fastest).  The
 * kernel is the product RBF  outputscale * prod_e exp(-(x_e - x'_e)^2 / (2 l_e^2)),
 * so K_UU is a Kronecker product of symmetric Toeplitz factors. */
typedef struct {
  int dim;                    /* 1..3                                        */
  int64_t n;                  /* training points (>= 1)                      */
  int64_t grid_size[3];       /* points per dimension (>= 4)                 */
  double grid_lo[3];
  double grid_hi[3];
  double outputscale;         /* s_f > 0                                     */
  double lengthscale[3];      /* l_e > 0                                     */
  double noise;               /* sigma^2 > 0                                 */
  love_dtype dtype;           /* LOVE_F32 or LOVE_F64: x, y and the Lanczos  */
  const love_allocator* allocator;  /* NULL -> cudaMallocAsync             */
  int additive;               /* 0: the product kernel above.  1: the additive
                                 composition of the paper's Sec. 3 extension,
                                 sum_e outputscale exp(-(x_e - x'_e)^2 / (2 l_e^2)):
                                 one 1-D grid per dimension, stacked
                                 interpolation vectors (4 nonzeros per
                                 dimension) and a block-diagonal K_UU,
                                 m = sum_e grid_size[e].  Supported by ski_mvm,
                                 ski_mvm_kuu, love_precompute (variance and mean
                                 caches, sampler), love_predict_mean_var,
                                 love_predict_var_root and love_sample; the
                                 other calls return LOVE_ERR_UNSUPPORTED. */
} love_ski_desc;

typedef struct love_ski* love_ski_t;
typedef struct love_cache* love_cache_t;

/* ski_build -- sort the training set by interpolation cell and prepare K_UU.
 * (Sec. 2.3, eq. ski: W_X holds the cubic interpolation weights of each x;
 * K_UU is Toeplitz / Kronecker-Toeplitz on the regular grid.)
 * x_train: n x dim device array (dtype); y_train: n device array or NULL.
 * Copies what it needs; the caller may free x_train/y_train on return.
 * Synchronises `stream` once.  Returns LOVE_ERR_DOMAIN if a training point's
 * stencil leaves the grid or is NaN.  *out is owned by the caller and freed
 * with ski_destroy. */
LOVE_API love_status ski_build(const love_ski_desc* desc, const void* x_train,
                      const void* y_train, love_stream_t stream, love_ski_t* out);
LOVE_API love_status ski_destroy(love_ski_t ski);

/* ski_mvm -- out = (W^T K_UU W + sigma^2 I) v   (Algorithm 1's mvm_K_XX).
 * v, out: n device arrays in the caller's training-point order.  May not alias. */
LOVE_API love_status ski_mvm(love_ski_t ski, const void* v, void* out, love_stream_t stream);

/* ski_mvm_kuu -- out = K_UU v for m = prod(grid_size) grid values (Sec. 2.3,
 * Toeplitz/Kronecker MVM by FFT).  v, out: m device arrays (dtype). */
LOVE_API love_status ski_mvm_kuu(love_ski_t ski, const void* v, void* out, love_stream_t stream);

/* Flags of love_precompute_opts.flags */
#define LOVE_WANT_MEAN 0x1u     /* solve K^ z = y by CG, cache a = K_UU W z   */
#define LOVE_WANT_SAMPLER 0x2u  /* Lanczos on K_UU - R^T R', cache S          */
#define LOVE_WANT_GRAD 0x4u     /* keep P = W Q L^{-T} for love_var_backward  */
#define LOVE_PRIOR_EXACT 0x8u   /* prior k(x*,x*) = s_f instead of w^T K_UU w */
#define LOVE_TIME_REORTH 0x10u  /* time the reorthogonalisation sweeps (love_cache_info.reorth_ms) */
#define LOVE_BATCH_STREAMS 0x20u /* love_precompute_batched: one love_precompute per GP on a pool
                                    stream instead of the batched Lanczos kernels */

typedef struct {
  int k;                   /* Lanczos steps (1..200)                           */
  love_dtype cache_dtype;  /* F32, BF16 (with an F32 ski) or F64 (F64 ski)     */
  unsigned flags;
  double breakdown_tol;    /* stop when beta_j <= tol * max|alpha|; <=0: 1e-12 (F64) / 1e-8 (F32) */
  double cg_tol;           /* relative residual of the FP64 CG; <=0: 1e-12 (F64 ski) / 1e-6 (F32 ski) */
  int cg_max_iter;         /* <=0: 4000                                        */
  int sampler_k;           /* Lanczos steps for S; <=0: k                      */
  uint64_t sampler_seed;   /* SplitMix64 seed of the Rademacher probe          */
  int reorth;              /* LOVE_REORTH_ALWAYS (0), _DETECT (1) or _LOWSYNC (2) */
  double reorth_eta;       /* DETECT threshold on |Q_j^T y'| / |y'|; <=0: 2^-22 (F32) / 2^-51 (F64) */
  int cg_plain;            /* 1: the mean CG without preconditioner (Sec. 2.1); 0: on a 1-D grid
                              the grid-space CG is preconditioned by the spectral inverse of
                              B K_UU + s^2 I (B the averaged stencil of W W^T); same stopping rule */
} love_precompute_opts;

/* Reorthogonalisation of the Lanczos runs over K^ (love_precompute.reorth).
 * ALWAYS: classical Gram-Schmidt twice at every step (Sec. 5).  DETECT: the
 * second pass runs only where the first one left a measurable component,
 * |Q_j^T y'| > eta |y'| with y' = y - Q_j Q_j^T y (measured in the same sweep
 * that applies the first pass), so a healthy step reads Q_j twice instead of
 * three times; the number of steps that skipped it is reported by
 * love_cache_info.  LOWSYNC: the second pass folded into the first through
 * the Gram matrix G = Q_j^T Q_j (kept from the measured dots of each new
 * vector): c = c1 + (c1 - G c1) with c1 = Q_j^T y, so one update sweep
 * y - Q_j c (which also measures Q_j^T y' for the next row of G) replaces the
 * two; the DETECT test then decides whether a real second pass is still
 * needed.  Two reads of Q_j per step instead of three.  The sampler's Lanczos
 * run always takes both passes. */
#define LOVE_REORTH_ALWAYS 0
#define LOVE_REORTH_DETECT 1
#define LOVE_REORTH_LOWSYNC 2

/* love_precompute -- the LOVE pre-compute phase (Sec. 3.2, Algorithm 1):
 * k Lanczos steps with full reorthogonalisation (Sec. 5) on K^ from the probe
 * b = (1/m) W^T K_UU 1; T = L L^T; the variance cache Rt = K_UU W Q L^{-T}
 * (so Rt Rt^T = R^T R'), the mean cache a (eq. pred_mean_ski) and optionally
 * the sampler root S (Sec. 3.3).  Synchronises `stream` once at the end and
 * writes the number of steps kept (<= k, fewer after a Lanczos breakdown) to
 * *k_eff (host pointer, may be NULL).  Returns LOVE_ERR_NOT_PD if T is not
 * positive definite.  *out is freed with love_cache_destroy.  The ski handle
 * may be destroyed afterwards; the cache does not reference it. */
LOVE_API love_status love_precompute(love_ski_t ski, const love_precompute_opts* opts,
                            love_stream_t stream, love_cache_t* out, int* k_eff);
LOVE_API love_status love_cache_destroy(love_cache_t cache);

/* love_predict_mean_var -- for each of t test points (t x dim device array,
 * the ski dtype): mean = w*^T a (eq. pred_mean_ski; requires LOVE_WANT_MEAN,
 * else pass mean = NULL) and var = p(x*) - |Rt^T w*|^2 (eq. pred_covar_ski_fast
 * with i = j; Algorithm 1), p the SKI prior w*^T K_UU w* (or s_f with
 * LOVE_PRIOR_EXACT).  Outputs are t device arrays in the ski dtype.  var is
 * clamped at 0 (the clamp count is in the device status).  A point whose stencil
 * leaves the grid gets NaN and sets LOVE_ERR_DOMAIN in the device status.
 * t = 0 is a no-op. */
LOVE_API love_status love_predict_mean_var(love_cache_t cache, int64_t t, const void* x_test,
                                  void* mean, void* var, love_stream_t stream);

/* love_predict_mean_var_host -- love_predict_mean_var on HOST buffers: x_test
 * (t x dim), mean (t, or NULL) and var (t) in host memory, ski dtype.  Page-
 * locked buffers (cudaHostAlloc, cudaHostRegister, torch pin_memory) are read
 * and written by the predict kernel itself through their device mapping, over
 * the CPU-GPU link, with no separate copies; any other host buffer goes
 * through device staging buffers in chunks of 2^20 points (taken from the
 * cache's allocator and released before returning).  Synchronises `stream`:
 * the results are in the host buffers when the call returns.  t = 0 is a
 * no-op; errors as love_predict_mean_var. */
LOVE_API love_status love_predict_mean_var_host(love_cache_t cache, int64_t t, const void* x_test, void* mean,
                                                void* var, love_stream_t stream);

/* love_predict_covariance -- posterior cross-covariances between two sets of
 * test points (Sec. 3: eq. pred_covar_ski_fast for i != j, Algorithm 1 with
 * two point sets):  cov[i, j] = p(x1_i, x2_j) - (Rt^T w1_i) . (Rt^T w2_j), with
 * p the SKI prior w1_i^T K_UU w2_j (or outputscale * k(x1_i, x2_j) with
 * LOVE_PRIOR_EXACT).  x1: t1 x dim, x2: t2 x dim device arrays; cov: t1 x t2
 * row-major device array; all in the ski dtype.  Entries of a point whose
 * stencil leaves the grid are NaN (and LOVE_ERR_DOMAIN is recorded).  Takes
 * temporary device memory from the cache's allocator (O((t1 + t2) k)).  With
 * x1 = x2 the diagonal is the variance of love_predict_mean_var (up to
 * rounding). */
LOVE_API love_status love_predict_covariance(love_cache_t cache, int64_t t1, const void* x1, int64_t t2,
                                             const void* x2, void* cov, love_stream_t stream);

/* love_predict_var_root -- predictive variance from the posterior root S of
 * Sec. 3.3 (S S^T ~ K_UU - Rt Rt^T, the sampler cache): var = |S^T w*|^2 at
 * each of t test points.  A sum of squares, so no cancellation against the
 * prior (relative accuracy where p - |Rt^T w*|^2 loses it), but a rank-k_s
 * truncation of the posterior covariance (exact at Krylov exhaustion).
 * Requires LOVE_WANT_SAMPLER, else LOVE_ERR_STATE.  x_test: t x dim device
 * array; var: t device array; both in the ski dtype.  t = 0 is a no-op. */
LOVE_API love_status love_predict_var_root(love_cache_t cache, int64_t t, const void* x_test, void* var,
                                           love_stream_t stream);

/* love_sample -- s posterior samples at t test points (Sec. 3.3, eq. sample):
 * out[j, i] = mean_i + (W*^T S z)_{i j}, out an s x t device array (sample-major,
 * ski dtype).  z: k_s x s device array of standard normals (row-major, float for
 * an F32 ski, double for F64), or NULL to draw them on the device from
 * Philox4x32-10 with `seed` (Box-Muller).  Requires LOVE_WANT_SAMPLER. */
LOVE_API love_status love_sample(love_cache_t cache, int64_t t, const void* x_test, int s,
                        const void* z, uint64_t seed, void* out, love_stream_t stream);

/* love_sampler_precompute -- the sampler pre-compute of Sec. 3.3 (eqs.
 * lancapprox, sampling_pre_cholesky, pred_covar_ski_interp_form) on an
 * existing cache: ks Lanczos steps (0 -> k_eff; at most 200 and m) with full
 * reorthogonalisation on M = K_UU - Rt Rt^T from the SplitMix64 Rademacher probe
 * of `seed`, T' = L' L'^T and the root S = Q' L' (m x ks'), exactly the
 * sampler run that love_precompute makes with LOVE_WANT_SAMPLER, but on the Rt
 * the cache holds -- one made by love_precompute, love_cache_import or
 * love_cache_load -- with the cache's own grid and kernel (K_UU's plans are
 * built for the call and released).  For a BF16 cache Rt is read as stored
 * (BF16-rounded); love_precompute's sampler uses Rt before that rounding.  A
 * root the cache held before is replaced; afterwards the cache has
 * LOVE_WANT_SAMPLER, love_cache_info reports sampler_k, sampler_fallback and
 * phase_ms[3].  Work space and the root come from the cache's allocator.
 * Synchronises `stream`.  Errors: LOVE_ERR_ARG (NULL cache, ks < 0 or > 200),
 * LOVE_ERR_NAN (no Lanczos step survived), LOVE_ERR_OOM. */
LOVE_API love_status love_sampler_precompute(love_cache_t cache, int ks, uint64_t seed, love_stream_t stream);

/* love_var_backward -- vector-Jacobian product of L = sum_i g_i var_i (not in
 * the paper; derived from eq. pred_covar_ski_cache with K^^{-1} ~ Q T^{-1} Q^T,
 * Q held fixed):
 *   grad_x[i, e]      = g_i d var_i / d x*_{i,e}                (t x dim, may be NULL)
 *   grad_lengthscale  = dL / d l_e  (HOST array of dim doubles, may be NULL)
 *   grad_noise        = dL / d sigma^2 (HOST double, may be NULL)
 * grad_var: t device array (ski dtype).  Requires LOVE_WANT_GRAD.  Synchronises
 * `stream` when a host output is requested. */
LOVE_API love_status love_var_backward(love_cache_t cache, int64_t t, const void* x_test,
                              const void* grad_var, void* grad_x,
                              double* grad_lengthscale, double* grad_noise,
                              love_stream_t stream);

/* Cache description, filled by love_cache_info (host struct). */
typedef struct {
  int dim;
  int64_t grid_size[3];
  int64_t m;
  int k_eff;               /* columns of Rt                                   */
  int ld;                  /* row stride (elements) of the predict cache      */
  int sampler_k;           /* columns of S (0 if absent)                      */
  int cg_iters;            /* CG iterations used for the mean (0 if absent)   */
  int sampler_fallback;    /* 1 if T' was not PD and S came from its eigenpairs */
  love_dtype dtype;        /* ski dtype                                       */
  love_dtype cache_dtype;
  unsigned flags;
  /* device time (ms, CUDA events) of the pre-compute phases: [0] Lanczos with
   * reorthogonalisation (incl. probe), [1] mean CG, [2] cache build (and the
   * gradient tables), [3] sampler; 0 for a cache that was imported or loaded */
  float phase_ms[4];
  int reorth_skipped;      /* Lanczos steps that skipped the second pass (DETECT) */
  float reorth_ms;         /* device time of the reorthogonalisation sweeps within phase_ms[0]
                              (CUDA events around each step's sweeps; LOVE_TIME_REORTH, else 0) */
  int batched_rows;        /* made by love_precompute_batched's batched Lanczos run: the rows of
                              its sweep chunks (phase_ms[0] is then the device time of the whole
                              batch's run, reorth_ms 0); else 0 */
} love_cache_info_t;

LOVE_API love_status love_cache_info(love_cache_t cache, love_cache_info_t* info);

/* love_cache_import -- build a cache from HOST arrays instead of running the
 * pre-compute (used to check the test-phase kernels against an independently
 * computed cache).  Rt: m x k row-major doubles; a: m doubles or NULL; S: m x ks
 * doubles or NULL; alpha (k), beta (k-1): the tridiagonal T (for gradients and
 * the noise derivative), P: m x k doubles or NULL.  Values are rounded to
 * cache_dtype.  The grid and kernel come from `desc` (n is ignored). */
LOVE_API love_status love_cache_import(const love_ski_desc* desc, int k, love_dtype cache_dtype,
                              unsigned flags, const double* Rt, const double* a,
                              int ks, const double* S, const double* alpha,
                              const double* beta, const double* P,
                              love_stream_t stream, love_cache_t* out);

/* love_cache_export -- copy cache contents to HOST arrays (any may be NULL):
 * Rt (m x k_eff), a (m), S (m x sampler_k), P (m x k_eff) as doubles, row-major;
 * alpha (k_eff), beta (k_eff - 1).  Synchronises `stream`. */
LOVE_API love_status love_cache_export(love_cache_t cache, double* Rt, double* a, double* S,
                              double* P, double* alpha, double* beta,
                              love_stream_t stream);

/* love_cache_save / love_cache_load -- a versioned, self-describing binary file
 * holding the grid, hyperparameters, alpha, beta and the cached matrices
 * (checkpoint of the pre-compute, which the paper runs as part of training).
 * Save/load round-trips bit-exactly.  Both synchronise `stream`.  load
 * returns LOVE_ERR_ARG, before allocating or copying anything, for a missing
 * file or one whose header does not describe exactly the buffers the library
 * writes for such a cache (grid, dtypes, k_eff and every buffer's size, the
 * gradient tables all present or all absent) or whose length differs from the
 * header's total; an allocation failure returns LOVE_ERR_OOM. */
LOVE_API love_status love_cache_save(love_cache_t cache, const char* path, love_stream_t stream);
LOVE_API love_status love_cache_load(const char* path, const love_allocator* allocator,
                            love_stream_t stream, love_cache_t* out);

/* Device status: bit (1 << status) for each error a kernel recorded since the
 * last reset, plus the count of points with a domain error and of clamped
 * negative variances.  Synchronises `stream`.  reset != 0 clears them. */
typedef struct {
  uint32_t bits;
  int64_t domain_errors;
  int64_t clamped;
} love_device_status_t;

LOVE_API love_status love_get_device_status(love_cache_t cache, int reset, love_device_status_t* st,
                                   love_stream_t stream);

/* ski_mvm_kuu_noalloc -- out = K_UU v, like ski_mvm_kuu, for callers that may
 * not allocate device memory.  The paper has no counterpart; it exists for
 * callers such as real-time loops that forbid allocator calls (an allocation
 * can block on the allocator's lock or synchronise the device), host
 * frameworks that own and have already reserved all device memory (a
 * cudaMalloc would fail or compete with their pool), and code running inside
 * the caching allocator's own callbacks, which cannot re-enter it.  ski_mvm_kuu takes
 * its FFT work area from the handle's allocator; this entry point instead uses
 * a fixed file-scope device array of 4 MiB, present on every GPU that loads the
 * library until the process exits, and calls no allocator (no cudaMalloc,
 * cudaFree or allocating library routine).  It accepts grids whose longest
 * mode with more than 2048 points needs at most 4 MiB of FFT work (a 1-D grid
 * of up to 131,072 points); larger grids return LOVE_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents (every call overwrites the part it reads, so nothing needs
 * clearing); calls whose work overlaps on the GPU, on different streams or
 * from different threads, race on it.  v, out: m device arrays (dtype). */
LOVE_API love_status ski_mvm_kuu_noalloc(love_ski_t ski, const void* v, void* out, love_stream_t stream);

/* ---- Batches of independent GPs ------------------------------------------
 * Not in the paper: a serving form of the same method for B independent
 * KISS-GPs of uneven n, m and test-set size.  Each GP's results are those of
 * the single-GP calls on its own handles (up to summation order). */

/* love_precompute_batched -- love_precompute for skis[0..B) with shared opts.
 * When every ski is 1-D, FP32 and not additive (and LOVE_BATCH_STREAMS is not
 * set), the B Lanczos runs are ONE batched run: each step is one launch per
 * phase (scatter, K_UU, gather, three reorthogonalisation sweeps) over a ragged
 * list of chunks of all GPs, the k steps captured into one CUDA graph, and the
 * sweep chunk size picked by timing the batch's own dot sweep.  Its
 * reorthogonalisation is the detection form (LOVE_REORTH_DETECT; LOWSYNC is
 * read as DETECT), so each GP's cache equals the single-GP cache to the FP32
 * tolerance, not bitwise.  The remaining phases (mean, cache, sampler) and
 * every other batch run as love_precompute per GP: up to `workers` at the
 * same time (0 -> 8; at most 32), each on a stream of a pool the library
 * owns, ordered after the work already queued on `stream`; the call returns
 * when all are done (like love_precompute, it synchronises).  caches[b] receives GP b's handle and
 * k_eff[b] (may be NULL) its Lanczos steps.  On failure every cache this call
 * created is destroyed, caches[] is all NULL and the status of the lowest
 * failing b is returned. */
LOVE_API love_status love_precompute_batched(int B, const love_ski_t* skis, const love_precompute_opts* opts,
                                             int workers, love_stream_t stream, love_cache_t* caches,
                                             int* k_eff);

typedef struct love_batch* love_batch_t;

/* love_batch_create -- serve caches[0..B) together.  t_off: HOST array of
 * B + 1 non-decreasing row offsets, t_off[0] = 0; rows t_off[b] ..
 * t_off[b+1] - 1 of the concatenated test inputs belong to GP b.  All caches
 * share dim, data dtype and cache dtype and must outlive the batch.  Uploads a
 * descriptor table (one entry per GP, plus a list of row chunks that never
 * straddle two GPs) and autotunes the launch shape of love_predict_batched
 * (lanes per test point, CTAs per SM) by timing the candidates on synthetic
 * in-domain points of the same sizes; synchronises `stream`.  Freed with
 * love_batch_destroy. */
LOVE_API love_status love_batch_create(int B, const love_cache_t* caches, const int64_t* t_off,
                                       love_stream_t stream, love_batch_t* out);
LOVE_API love_status love_batch_destroy(love_batch_t batch);

/* love_predict_batched -- love_predict_mean_var for every GP of the batch in
 * one kernel launch (a persistent grid walks the chunk list).  x: t_off[B] x
 * dim device array; mean (NULL, or every cache has LOVE_WANT_MEAN) and var:
 * t_off[B] device arrays; all in the data dtype.  No allocation, no
 * synchronisation: it may be captured into a CUDA graph. */
LOVE_API love_status love_predict_batched(love_batch_t batch, const void* x, void* mean, void* var,
                                          love_stream_t stream);

/* love_sample_batched -- love_sample for every GP: s samples per GP at its own
 * rows of x, normals drawn on the device (Philox4x32-10, GP b uses seed + b).
 * out: GP b's s x t_b sample-major block starts at element s * t_off[b].  Every
 * cache needs LOVE_WANT_SAMPLER.  Work space comes from the batch (allocated
 * on the first call for a given s, before any capture). */
LOVE_API love_status love_sample_batched(love_batch_t batch, const void* x, int s, uint64_t seed, void* out,
                                         love_stream_t stream);

/* love_batch_serve -- love_predict_batched then (if s > 0) love_sample_batched
 * on one stream.  With use_graph != 0 the launches are captured into a CUDA
 * graph the first time a given (x, mean, var, s, seed, samples) is seen (after
 * one eager call that sets up the work space) and the graph is replayed on
 * later calls with the same arguments.  A love_sample_batched call that has to
 * grow the batch's work space waits for a replay in flight and drops the graph,
 * so the next serve call captures again. */
LOVE_API love_status love_batch_serve(love_batch_t batch, const void* x, void* mean, void* var, int s,
                                      uint64_t seed, void* samples, int use_graph, love_stream_t stream);

/* Launch shape chosen by the autotuner and the candidates' times (host). */
typedef struct {
  int lanes_per_point;      /* threads cooperating on one test point */
  int ctas_per_sm;          /* persistent grid = ctas_per_sm x SMs (capped by chunks) */
  int n_candidates;
  float candidate_ms[16];   /* in the order lanes {small..large} x ctas {4, 8, 16} */
  int64_t chunks;
  int64_t graph_captures;          /* CUDA graphs captured by love_batch_serve so far */
  int64_t graph_captures_dropped;  /* of them, dropped because love_sample_batched needed a larger
                                      work space (the next serve call captures again) */
} love_batch_info_t;
LOVE_API love_status love_batch_info(love_batch_t batch, love_batch_info_t* info);

/* Host-side helpers. */
LOVE_API const char* love_status_string(love_status s);
LOVE_API int love_last_cuda_error(void);            /* last cudaError_t seen by the library */
/* Number of kernels this library has launched in this process (all entry
 * points, all devices); a host-side counter, no synchronisation. */
LOVE_API uint64_t love_launch_count(void);
LOVE_API const char* love_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LOVE_H_ */
