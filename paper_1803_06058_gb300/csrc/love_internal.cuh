// love_internal.cuh -- shared definitions of the GB300 LOVE library.
//
// Device-side building blocks used by every kernel file:
//   * double-float ("df") arithmetic: a value hi + lo of two floats, built from
//     the error-free transformations TwoSum (Knuth) and TwoProduct via FMA.
//     GB300 runs FP64 at a small fraction of its FP32 rate, so sums whose
//     cancellation needs more than 24 bits (reorthogonalisation dots, the
//     predictive variance p - |v|^2) are accumulated in df (~48-bit) instead
//     of native doubles (Dot2 of Ogita, Rump & Oishi 2005).
//   * Keys cubic-convolution weights (Sec. 2.3; a = -1/2).
//   * bounded mbarrier waits and 1-D bulk async copies (TMA) in inline PTX.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "../../include/love.h"

#define LOVE_MAX_DIM 3
#define LOVE_MAX_K 200

// ---------------------------------------------------------------------------
// device status word (one per handle)
struct DevStatus {
  unsigned int bits;
  unsigned int pad;
  unsigned long long domain_errors;
  unsigned long long clamped;
};

__device__ __forceinline__ void dev_flag(DevStatus* st, love_status s) {
  if (st) atomicOr(&st->bits, 1u << (unsigned)s);
}

// ---------------------------------------------------------------------------
// grid description passed by value to kernels
struct GridDev {
  int dim;
  int g[LOVE_MAX_DIM];          // points per dimension
  int stride[LOVE_MAX_DIM];     // linear-index stride of each dimension
  float lo_f[LOVE_MAX_DIM];
  float inv_h_f[LOVE_MAX_DIM];
  double lo_d[LOVE_MAX_DIM];
  double inv_h_d[LOVE_MAX_DIM];
  double h_d[LOVE_MAX_DIM];
  int m;
  int additive;                 // additive composition: block-diagonal K_UU
  int off[LOVE_MAX_DIM];        // (additive) first grid index of each block
};

// grid coordinate s = (x - lo)/h in the arithmetic of T.  The same function
// is used to bucket training points and to evaluate their weights, so the
// cell of a point and its stencil always agree.
__device__ __forceinline__ float grid_coord(float x, const GridDev& g, int e) {
  return (x - g.lo_f[e]) * g.inv_h_f[e];
}
__device__ __forceinline__ double grid_coord(double x, const GridDev& g, int e) {
  return (x - g.lo_d[e]) * g.inv_h_d[e];
}

// Keys kernel u(s) with a = -1/2:
//   |s| <= 1 : 3/2 |s|^3 - 5/2 |s|^2 + 1
//   1 < |s| < 2 : -1/2 |s|^3 + 5/2 |s|^2 - 4 |s| + 2
template <typename T>
__device__ __forceinline__ T keys_u(T s) {
  T a = s < T(0) ? -s : s;
  if (a <= T(1)) return (T(1.5) * a - T(2.5)) * a * a + T(1);
  if (a < T(2)) return ((T(-0.5) * a + T(2.5)) * a - T(4)) * a + T(2);
  return T(0);
}
// derivative u'(s) (odd)
template <typename T>
__device__ __forceinline__ T keys_du(T s) {
  T a = s < T(0) ? -s : s;
  T r;
  if (a <= T(1)) r = (T(4.5) * a - T(5)) * a;
  else if (a < T(2)) r = (T(-1.5) * a + T(5)) * a - T(4);
  else r = T(0);
  return s < T(0) ? -r : r;
}

// base index and the 4 weights of one coordinate: nodes i-1..i+2,
// w_r = u(f + 1 - r), f = s - i.  Returns false if the stencil leaves [0, g).
template <typename T>
__device__ __forceinline__ bool keys_weights(T s, int g, int& base, T w[4]) {
  if (!(s >= T(1)) || !(s < T(g - 2))) {  // also rejects NaN
    base = 1;
    w[0] = w[1] = w[2] = w[3] = T(0);
    return false;
  }
  int i = (int)floor(s);
  if (i > g - 3) i = g - 3;
  T f = s - T(i);
  base = i;
  w[0] = keys_u(f + T(1));
  w[1] = keys_u(f);
  w[2] = keys_u(T(1) - f);
  w[3] = keys_u(T(2) - f);
  return true;
}
template <typename T>
__device__ __forceinline__ void keys_dweights(T s, int base, T inv_h, T dw[4]) {
  T f = s - T(base);
  dw[0] = keys_du(f + T(1)) * inv_h;
  dw[1] = keys_du(f) * inv_h;
  dw[2] = keys_du(f - T(1)) * inv_h;
  dw[3] = keys_du(f - T(2)) * inv_h;
}

// ---------------------------------------------------------------------------
// double-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2)
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float err = (a - (s - bb)) + (b - bb);
  return {s, err};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, p.lo);
  p.lo = fmaf(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_from_double(double x) {
  float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// Dot2 accumulator: sum of exact products a*b (Ogita, Rump, Oishi 2005)
struct DotAccF {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float t = s + p;
    float z = t - s;
    float err = (s - (t - z)) + (p - z);
    s = t;
    c += pe + err;
  }
  __device__ __forceinline__ void add(float p) {
    float t = s + p;
    float z = t - s;
    c += (s - (t - z)) + (p - z);
    s = t;
  }
  __device__ __forceinline__ void merge(float s2, float c2) {
    float t = s + s2;
    float z = t - s;
    float err = (s - (t - z)) + (s2 - z);
    s = t;
    c += c2 + err;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
struct DotAccD {
  double s;
  static constexpr double c = 0.0;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add(double p) { s += p; }
  __device__ __forceinline__ void merge(double s2, double c2) { s += s2 + c2; }
  __device__ __forceinline__ double value() const { return s; }
};
template <typename T> struct DotAcc;
template <> struct DotAcc<float> { using type = DotAccF; };
template <> struct DotAcc<double> { using type = DotAccD; };

// warp-level merge of a DotAcc (deterministic butterfly)
__device__ __forceinline__ void warp_merge(DotAccF& a, unsigned mask = 0xffffffffu, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) {
    float s2 = __shfl_xor_sync(mask, a.s, o, width);
    float c2 = __shfl_xor_sync(mask, a.c, o, width);
    a.merge(s2, c2);
  }
}
__device__ __forceinline__ void warp_merge(DotAccD& a, unsigned mask = 0xffffffffu, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) a.s += __shfl_xor_sync(mask, a.s, o, width);
}

// ---------------------------------------------------------------------------
// mbarrier + bulk async copy (TMA, 1-D form) helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// programmatic dependent launch: wait for the preceding grid (and its memory)
// before reading what it wrote; let the next grid launch early
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of `bar`, giving up after ~1 s.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > 1000000000ull) return false;
  }
}

// ---------------------------------------------------------------------------
// grid-wide barrier of a cooperative launch (all CTAs co-resident), bounded
// like every other wait: after ~1 s a CTA flags LOVE_ERR_TIMEOUT, raises the
// abort word (so the others stop waiting too) and the call returns false; the
// kernel must then return without entering another barrier.  The arrival
// counter lives in global memory, zeroed before the first barrier of a run, and
// only grows: barrier number `gen` (counted from 0 over the run) is passed when
// it reaches (gen + 1) x gridDim.x.  After the CTA's bar.sync, thread 0 arrives
// with a release add (red.release: cumulative over the CTA's writes) and polls
// with acquire loads, which read the last add of a release sequence holding
// every arrival: every global write made before the barrier by any CTA is
// visible after it (data other CTAs wrote must still be read past L1,
// ld.global.cg).
struct GridSync {
  unsigned int count;   // arrivals since the run's first barrier
  unsigned int gen;     // unused (layout kept)
  unsigned int abort;   // a CTA gave up waiting
  unsigned int pad;
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// `gen` is the caller's count of barriers passed (the same in every CTA)
__device__ __forceinline__ bool grid_barrier(GridSync* gs, unsigned int& gen, DevStatus* status) {
  __shared__ int gb_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = (gen + 1u) * gridDim.x;
    red_release_add_gpu(&gs->count, 1u);
    if ((int)(ld_acquire_gpu(&gs->count) - target) < 0) {
      const uint64_t t0 = global_timer_ns();
      while ((int)(ld_acquire_gpu(&gs->count) - target) < 0) {
        if (ld_acquire_gpu(&gs->abort)) {
          ok = 0;
          break;
        }
        if (global_timer_ns() - t0 > 1000000000ull) {
          atomicExch(&gs->abort, 1u);
          dev_flag(status, LOVE_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    gb_ok = ok;
  }
  __syncthreads();
  gen += 1u;
  return gb_ok != 0;
}

// ---------------------------------------------------------------------------
// host-side handle definitions
struct FftPlan {
  int64_t g = 0;       // Toeplitz size along this mode
  int64_t N = 0;       // circulant length (power of two, >= 2g - 1)
  int N1 = 0, N2 = 0;  // four-step split (N1 = N, N2 = 1: single-CTA path)
  void* lam_f = nullptr;  // N floats: spectrum / N (outputscale folded into mode 0)
  void* lam_d = nullptr;  // N doubles
  void* tw_f = nullptr;   // N float2: exp(-2 pi i j / N)
  void* tw_d = nullptr;   // N double2
  void* lamdl_f = nullptr;  // spectrum of dT/dl (for gradients), / N
  void* lamdl_d = nullptr;
  // short modes (g <= TOEP_DENSE_MAX): the first column of T (and of dT/dl),
  // outputscale folded in like the spectrum, as float pairs (hi, lo) for the
  // dense double-float product; nullptr: the mode always takes the FFT
  void* col2 = nullptr;    // g float2
  void* coldl2 = nullptr;  // g float2
};
// modes up to this length apply T by a dense double-float product on the
// FP32 pipes instead of the FFT (whose FP64 butterflies run at the part's
// low FP64 rate)
constexpr int64_t TOEP_DENSE_MAX = 384;

struct Allocator {
  love_allocator a{};
  bool user = false;
  void* alloc(size_t bytes, cudaStream_t s) const;
  void free(void* p, size_t bytes, cudaStream_t s) const;
};

// Work buffers of one host thread kept for reuse: while a thread has one
// installed (love_precompute_batched's workers and their mean-solve threads),
// scratch_alloc / scratch_free hand a freed buffer back to the next request
// of the same allocator and stream that fits it (sizes rounded up to powers of
// two), so B pre-computes in a row call the allocator (for the torch binding,
// a Python callback per call) about as often as one.  Reuse on the same stream
// only, so the stream orders a buffer's earlier work before its next use.
// release() returns every buffer to its allocator.
struct ScratchCache {
  struct Blk {
    Allocator al;
    cudaStream_t s;
    void* p;
    size_t bytes;
  };
  std::vector<Blk> idle, busy;
  ~ScratchCache() { release(); }
  void* take(const Allocator& al, size_t bytes, cudaStream_t s);
  bool give(void* p);
  void release();
};
ScratchCache*& thread_scratch();        // this thread's cache, or nullptr
ScratchCache*& thread_mean_scratch();   // the cache a mean-solve thread started here adopts
void* scratch_alloc(const Allocator& al, size_t bytes, cudaStream_t s);
void scratch_free(const Allocator& al, void* p, size_t bytes, cudaStream_t s);

struct GridHost {
  int dim = 1;
  bool additive = false;                 // block-diagonal K_UU of 1-D blocks
  int64_t off[LOVE_MAX_DIM] = {0, 0, 0};  // (additive) first index of block e
  int64_t g[LOVE_MAX_DIM] = {1, 1, 1};
  int64_t stride[LOVE_MAX_DIM] = {1, 1, 1};
  int64_t m = 1;
  double lo[LOVE_MAX_DIM] = {0, 0, 0};
  double h[LOVE_MAX_DIM] = {1, 1, 1};
  double ls[LOVE_MAX_DIM] = {1, 1, 1};
  double sf = 1.0;
  double noise = 1.0;
  double cloc[LOVE_MAX_DIM][4] = {};     // T_e[0..3] (first Toeplitz entries)
  double cloc_dl[LOVE_MAX_DIM][4] = {};  // dT_e/dl_e [0..3]
  GridDev dev() const;
};

// one 1-D component (block e) of an additive grid, as a 1-D grid of its own
inline GridDev component_dev(const GridHost& gh, int e) {
  GridDev d = gh.dev();
  GridDev c{};
  c.dim = 1;
  c.g[0] = d.g[e];
  c.stride[0] = 1;
  c.lo_f[0] = d.lo_f[e];
  c.inv_h_f[0] = d.inv_h_f[e];
  c.lo_d[0] = d.lo_d[e];
  c.inv_h_d[0] = d.inv_h_d[e];
  c.h_d[0] = d.h_d[e];
  for (int q = 1; q < LOVE_MAX_DIM; ++q) {
    c.g[q] = 1;
    c.stride[q] = 1;
  }
  c.m = d.g[e];
  c.additive = 0;
  return c;
}

struct love_ski {
  GridHost grid;
  love_dtype dtype = LOVE_F32;
  int64_t n = 0, n_pad = 0;
  Allocator alloc;
  int device = 0;
  void* xs = nullptr;          // n_pad x dim, sorted by cell (dtype)
  void* ys = nullptr;          // n_pad (dtype) or null
  int32_t* perm = nullptr;     // sorted position -> caller index (n)
  int32_t* cell_start = nullptr;  // m + 1
  FftPlan fft[LOVE_MAX_DIM];
  DevStatus* status = nullptr;
  // additive composition: per dimension e, the points sorted by their cell in
  // dimension e: 1-D coordinates, cell starts (g_e + 1) and the position of
  // each in the primary (dimension-0) order (null for e = 0)
  void* xs1[LOVE_MAX_DIM] = {nullptr, nullptr, nullptr};
  int32_t* cs1[LOVE_MAX_DIM] = {nullptr, nullptr, nullptr};
  int32_t* map1[LOVE_MAX_DIM] = {nullptr, nullptr, nullptr};
};

struct love_cache {
  GridHost grid;
  love_dtype dtype = LOVE_F32, cache_dtype = LOVE_F32;
  unsigned flags = 0;
  int k_eff = 0, ld = 0;       // Rc: m x ld, columns [0,k) = Rt, column k = a
  Allocator alloc;
  void* Rc = nullptr;
  int ks = 0, ld_s = 0;        // S: m x ld_s (dtype), columns [0, ks)
  void* S = nullptr;
  int ld_g = 0;                // backward tables: KdP_e: m x ld_g per dimension
  void* KdP = nullptr;         // dim x m x ld_g (dtype): (dK/dl_e) P
  void* B = nullptr;           // dim x k x k (float/double): P^T (dK/dl_e) P
  void* Minv = nullptr;        // k x k: L^{-1} L^{-T}
  double* alpha = nullptr;     // host copies
  double* beta = nullptr;
  void* P = nullptr;           // m x k_eff column-major (dtype), kept for export
  int cg_iters = 0;
  int reorth_skipped = 0;
  float reorth_ms = 0.f;
  int batched_rows = 0;        // sweep chunk rows of the batched Lanczos run that made it (0: single)
  int sampler_fallback = 0;
  float phase_ms[4] = {0, 0, 0, 0};
  DevStatus* status = nullptr;
  void* sws = nullptr;         // love_sample work space (grown on demand, kept)
  size_t sws_bytes = 0;
};

// ---------------------------------------------------------------------------
// launchers (defined in the kernel .cu files)
namespace love {

// k_sort.cu
love_status sort_training_points(love_ski* ski, const void* x_in, const void* y_in, cudaStream_t s);
// additive composition: the per-dimension orders (xs1, cs1, map1) from the primary order
love_status sort_additive_dims(love_ski* ski, cudaStream_t s);

// k_fft.cu
// dense: allow the double-float dense product on modes of up to TOEP_DENSE_MAX
// (FP32 data; FP64 data keeps the FP64 FFT, whose rounding is ~100x smaller)
love_status fft_plan_create(FftPlan& p, const GridHost& g, int e, const Allocator& al, cudaStream_t s,
                            bool dense);
void fft_plan_destroy(FftPlan& p, const Allocator& al, cudaStream_t s);
// out = K_UU v (all modes) for `ncol` columns (column stride ldc elements); work
// must hold fft_work_elems() complex values.  deriv_dim >= 0 selects dK/dl_e.
size_t fft_work_bytes(const GridHost& g, const FftPlan* plans, int ncol, bool dbl);
template <typename T>
love_status kuu_apply(const GridHost& g, const FftPlan* plans, const T* v, T* out, int ncol,
                      int64_t ldc, void* work, int deriv_dim, cudaStream_t s);

// k_lanczos.cu
struct LanczosWork;
template <typename T>
love_status lanczos_run(love_ski* ski, int k, double tau, double eta, T* Q, int64_t ldq, double* alpha_h,
                        double* beta_h, int* k_eff, int* skipped, cudaStream_t s, float* reorth_ms = nullptr,
                        bool lowsync = false);
template <typename T>
love_status ski_mvm_sorted(love_ski* ski, const T* v, T* out, void* work, cudaStream_t s);
template <typename T>
love_status scatter_multi(love_ski* ski, const T* Q, int64_t ldq, int ncol, T* out, int64_t ldo,
                          cudaStream_t s);
template <typename T>
love_status cg_solve(love_ski* ski, const T* b, double* x, double tol, int max_iter, int* iters,
                     cudaStream_t s);
// mean weights a = K_UU W K^^-1 y (m-vector, FP64) by CG on the grid system
// (G K_UU + s^2 I) z = W y with G = W W^T; dimensions 1 and 2
bool mean_grid_cg_supported(const love_ski* ski);
template <typename T>
love_status mean_grid_cg(love_ski* ski, double tol, int max_iter, double* a, int* iters, cudaStream_t s,
                         bool precond);
// write mean weights a (m, FP64) into the cache's mean column
love_status cache_set_mean(love_cache* c, const double* a, cudaStream_t s);
// zmean: K^^-1 y (n-vector, cell-sorted) or amean: the mean weights themselves
template <typename T>
love_status build_cache(love_ski* ski, love_cache* c, const T* Q, int64_t ldq, const double* zmean,
                        cudaStream_t s, T* keep_rt, const double* amean = nullptr);
// sampler Lanczos on M = K_UU - Rt Rt^T, FP64 vectors Q (m_pad x ks, column-major);
// Rt: m x k column-major (ldr) of the data dtype
template <typename T>
love_status sampler_lanczos(const GridHost& gh, const FftPlan* fft, const Allocator& al, const T* Rt, int64_t ldr,
                            int k, int ks, uint64_t seed, double tau, double* Q, int64_t ldq, double* alpha_h,
                            double* beta_h, int* ks_eff, DevStatus* status, cudaStream_t s);
// k_mvm.cu: the SKI product of one Lanczos step (1-D grid, FP32 data) as one
// cooperative kernel: y = W^T K_UU W q_j + s^2 q_j, q_j scaled by *scal in place;
// a no-op once *done.  work: ski_mvm_fused_work_bytes(ski) bytes, set up once per
// run by ski_mvm_fused_reset (df twiddle and spectrum tables, zeroed barrier
// counters); gen0: the barriers the run's
// earlier products completed (4 per product).  LOVE_ERR_UNSUPPORTED where the
// grid or the device does not allow it.
// k_lanczos_batched.cu: the n-space Lanczos runs of B independent GPs on 1-D
// grids (FP32 data, kcols[b] steps each, the detection form of the
// reorthogonalisation with eta), one launch per phase per step for all GPs,
// the steps captured into one CUDA graph on s (a stream that can be captured:
// not the legacy default stream).  Q[b]: n_pad x kcols[b] (ski b's allocator).
// rows: rows per sweep chunk (a multiple of 64 >= 256), or 0 to pick it by
// timing the dot sweep.  LOVE_ERR_UNSUPPORTED where a GP is not of that form.
struct BatchedLanczos {
  struct Gp {
    std::vector<double> alpha, beta;
    int k_eff = 0, skipped = 0;
  };
  std::vector<Gp> gp;
  int rows = 0;                  // the sweep chunk rows used
  float ms = 0.f;                // device time of the batch's probe and k steps (CUDA events)
  std::vector<float> tune_ms;    // dot-sweep time per candidate (256, 512, 1024, 2048 rows)
};
love_status lanczos_batched(int B, love_ski* const* skis, const int* kcols, float* const* Q, double tau, double eta,
                            int rows, cudaStream_t s, BatchedLanczos* out);
// love_api.cu: the option checks and Lanczos parameters of love_precompute, and
// its remaining phases (mean, cache, sampler) on a Lanczos run already made
// (Q: n_pad x precompute_k columns from ski's allocator, owned by the call)
love_status precompute_opts_check(const love_ski* ski, const love_precompute_opts* opts);
int precompute_k(const love_ski* ski, const love_precompute_opts* o);
void precompute_lanczos_params(const love_ski* ski, const love_precompute_opts* o, double* tau, double* eta);
love_status precompute_from_lanczos(love_ski* ski, const love_precompute_opts* opts, cudaStream_t s, float* Q,
                                    const BatchedLanczos::Gp& r, int rows, float lanczos_ms, love_cache** out,
                                    int* k_eff);
// the circulant's twiddles W_N^j and spectrum lambda_j / N as double-float
// tables (twdf: {re.hi, re.lo, im.hi, im.lo}; lamdf: {hi, lo}), N entries each
love_status fft_df_tables(const FftPlan& p, float4* twdf, float2* lamdf, cudaStream_t s);
size_t ski_mvm_fused_work_bytes(const love_ski* ski);
love_status ski_mvm_fused_reset(const love_ski* ski, void* work, cudaStream_t s);
love_status ski_mvm_fused(love_ski* ski, float* qj, const double* scal, const int* done, float* y, void* work,
                          unsigned int gen0, cudaStream_t s);
// k_sampler.cu: the same run as one persistent cooperative kernel (1-D grids
// whose per-CTA share fits in shared memory); LOVE_ERR_UNSUPPORTED otherwise
template <typename T>
love_status sampler_lanczos_fused(const GridHost& gh, const FftPlan* fft, const Allocator& al, const T* Rt,
                                  int64_t ldr, int k, int ks, uint64_t seed, double tau, double* Q, int64_t ldq,
                                  double* alpha_h, double* beta_h, int* ks_eff, DevStatus* status, cudaStream_t s);
// k_sample.cu: S = Q' L' (or the eigen fallback), stored in the cache
// (g, fft: the grid and K_UU plans of the cache's kernel; al: work space)
template <typename T>
love_status sampler_build(const GridHost& g, const FftPlan* fft, const Allocator& al, love_cache* c, const T* Rt,
                          int ks, uint64_t seed, double tau, cudaStream_t s);

template <typename T>
love_status permute_in(const T* v, const int32_t* perm, int64_t n, int64_t n_pad, T* out, cudaStream_t s);
template <typename T>
love_status permute_out(const T* v, const int32_t* perm, int64_t n, T* out, cudaStream_t s);

// k_predict.cu
// batched predict: one entry per GP (an opaque descriptor of predict_desc_bytes()),
// row chunks that never straddle two GPs, one persistent launch
struct PredChunk {
  int gp, pad;
  int64_t begin, end;  // rows [begin, end) of GP gp (GP-local indices)
};
size_t predict_desc_bytes();
void predict_fill_desc(const love_cache* c, void* dst);
int predict_lane_candidates(int dim, int* out);
love_status predict_batched_launch(const void* descs, const int64_t* toff, const PredChunk* chunks, int nchunks,
                                   int dim, love_dtype dtype, love_dtype cache_dtype, int lanes, int ctas_per_sm,
                                   const void* x, void* mean, void* var, cudaStream_t s);
love_status predict_root_launch(love_cache* c, int64_t t, const void* x, void* var, cudaStream_t s);
// k_cov.cu: t1 x t2 posterior cross-covariances (row-major, data dtype)
love_status cov_launch(love_cache* c, int64_t t1, const void* x1, int64_t t2, const void* x2, void* out,
                       cudaStream_t s);
love_status predict_launch(love_cache* c, int64_t t, const void* x, void* mean, void* var,
                           cudaStream_t s);
love_status backward_launch(love_cache* c, int64_t t, const void* x, const void* gv, void* gx,
                            double* gl, double* gn, cudaStream_t s);
love_status backward_tables(love_cache* c, const FftPlan* plans, const void* P, int k,
                            cudaStream_t s);

// k_sample.cu
love_status sample_launch(love_cache* c, int64_t t, const void* x, int s_count, const void* z,
                          uint64_t seed, void* out, cudaStream_t s);
// the same with caller work space (Philox normals, no allocation)
size_t sample_ws_bytes(const love_cache* c, int64_t t, int s_count);
love_status sample_launch_ws(love_cache* c, int64_t t, const void* x, int s_count, uint64_t seed, void* out,
                             void* ws, cudaStream_t s);
love_status sample_launch_z_ws(love_cache* c, int64_t t, const void* x, int s_count, const void* z, uint64_t seed,
                               void* out, void* ws, cudaStream_t s);

// api helpers
extern thread_local int g_last_cuda_error;
// kernels launched by this library in this process (reported by love_launch_count)
void count_launch();
inline love_status cuda_check(cudaError_t e) {
  if (e == cudaSuccess) return LOVE_OK;
  g_last_cuda_error = (int)e;
  return LOVE_ERR_CUDA;
}

// the most dynamic shared memory a kernel can take (the device's opt-in
// maximum less the kernel's static shared memory), looked up once per kernel;
// -1 when the attributes cannot be read
int smem_limit(const void* kernel);

// raise a kernel's dynamic shared-memory limit (above the 48 KB default)
template <typename K>
inline love_status allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return LOVE_OK;
  // always raise the kernel's limit to the most it can take, not to `bytes`:
  // concurrent host threads launching the same kernel with different sizes
  // then never lower the limit under one another
  const int limit = smem_limit(reinterpret_cast<const void*>(kernel));
  if (limit < 0) return LOVE_ERR_CUDA;
  if (bytes > (size_t)limit) return LOVE_ERR_UNSUPPORTED;
  return cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
}
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
int num_sms();

}  // namespace love

// The C-ABI entry points are function-try-blocks closed by LOVE_ENTRY_CATCH:
// the library throws only when host resources run out (std::bad_alloc from a
// container, std::system_error from starting a host thread), and no exception
// may cross the C boundary, so any exception becomes LOVE_ERR_OOM
#define LOVE_ENTRY_CATCH \
  catch (...) {          \
    return LOVE_ERR_OOM; \
  }

#define LOVE_TRY(...)                      \
  do {                                     \
    love_status _st = (__VA_ARGS__);       \
    if (_st != LOVE_OK) return _st;        \
  } while (0)
#define LOVE_CUDA(...) LOVE_TRY(love::cuda_check(__VA_ARGS__))
#define LOVE_LAUNCH_CHECK() LOVE_CUDA(cudaGetLastError())
#define LOVE_COUNT_LAUNCH() love::count_launch()
