// love_api.cu -- the C ABI declared in include/love.h.
//
// Host-side orchestration only: argument checks, handle lifetime, device
// memory (caller allocator or cudaMallocAsync), and the order of the kernel
// phases.  Every arithmetic step of the method runs in the kernels of
// k_sort.cu, k_fft.cu, k_lanczos.cu, k_predict.cu and k_sample.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>
#include <vector>

#include <mutex>
#include <thread>

#include "love_internal.cuh"

namespace love {

thread_local int g_last_cuda_error = 0;
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace love

using namespace love;

// ---------------------------------------------------------------------------
void* Allocator::alloc(size_t bytes, cudaStream_t s) const {
  if (bytes == 0) bytes = 16;
  if (user) return a.alloc(a.ctx, bytes, s);
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    g_last_cuda_error = (int)e;
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void Allocator::free(void* p, size_t bytes, cudaStream_t s) const {
  if (!p) return;
  if (user) {
    a.free(a.ctx, p, bytes ? bytes : 16, s);
    return;
  }
  cudaFreeAsync(p, s);
}

static bool same_allocator(const Allocator& a, const Allocator& b) {
  return a.user == b.user && (!a.user || (a.a.alloc == b.a.alloc && a.a.free == b.a.free && a.a.ctx == b.a.ctx));
}
void* ScratchCache::take(const Allocator& al, size_t bytes, cudaStream_t s) {
  size_t r = 256;
  while (r < bytes) r <<= 1;
  for (size_t i = 0; i < idle.size(); ++i) {
    if (idle[i].s == s && idle[i].bytes == r && same_allocator(idle[i].al, al)) {
      busy.push_back(idle[i]);
      idle.erase(idle.begin() + (std::ptrdiff_t)i);
      return busy.back().p;
    }
  }
  void* p = al.alloc(r, s);
  if (p) busy.push_back(Blk{al, s, p, r});
  return p;
}
bool ScratchCache::give(void* p) {
  for (size_t i = 0; i < busy.size(); ++i) {
    if (busy[i].p == p) {
      idle.push_back(busy[i]);
      busy.erase(busy.begin() + (std::ptrdiff_t)i);
      return true;
    }
  }
  return false;
}
void ScratchCache::release() {
  for (auto& b : idle) b.al.free(b.p, b.bytes, b.s);
  for (auto& b : busy) b.al.free(b.p, b.bytes, b.s);
  idle.clear();
  busy.clear();
}
ScratchCache*& thread_scratch() {
  static thread_local ScratchCache* t = nullptr;
  return t;
}
ScratchCache*& thread_mean_scratch() {
  static thread_local ScratchCache* t = nullptr;
  return t;
}
void* scratch_alloc(const Allocator& al, size_t bytes, cudaStream_t s) {
  ScratchCache* c = thread_scratch();
  return c ? c->take(al, bytes, s) : al.alloc(bytes, s);
}
void scratch_free(const Allocator& al, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  ScratchCache* c = thread_scratch();
  if (c && c->give(p)) return;
  al.free(p, bytes, s);
}

GridDev GridHost::dev() const {
  GridDev d{};
  d.dim = dim;
  d.m = (int)m;
  for (int e = 0; e < LOVE_MAX_DIM; ++e) {
    d.g[e] = (int)g[e];
    d.stride[e] = (int)stride[e];
    d.lo_d[e] = lo[e];
    d.h_d[e] = h[e];
    d.inv_h_d[e] = 1.0 / h[e];
    d.lo_f[e] = (float)lo[e];
    d.inv_h_f[e] = (float)(1.0 / h[e]);
    d.off[e] = (int)off[e];
  }
  d.additive = additive ? 1 : 0;
  return d;
}

namespace {

inline cudaStream_t cs(love_stream_t s) { return (cudaStream_t)s; }

size_t dtype_size(love_dtype d) { return d == LOVE_F64 ? 8 : (d == LOVE_BF16 ? 2 : 4); }

love_status grid_from_desc(const love_ski_desc* d, GridHost& g) {
  if (!d || d->dim < 1 || d->dim > LOVE_MAX_DIM) return LOVE_ERR_ARG;
  if (!(d->outputscale > 0) || !(d->noise > 0)) return LOVE_ERR_ARG;
  g.dim = d->dim;
  int64_t m = 1;
  for (int e = 0; e < LOVE_MAX_DIM; ++e) {
    if (e < d->dim) {
      if (d->grid_size[e] < 4 || !(d->grid_hi[e] > d->grid_lo[e]) || !(d->lengthscale[e] > 0)) return LOVE_ERR_ARG;
      g.g[e] = d->grid_size[e];
      g.lo[e] = d->grid_lo[e];
      g.h[e] = (d->grid_hi[e] - d->grid_lo[e]) / (double)(d->grid_size[e] - 1);
      g.ls[e] = d->lengthscale[e];
    } else {
      g.g[e] = 1;
      g.lo[e] = 0;
      g.h[e] = 1;
      g.ls[e] = 1;
    }
    m *= g.g[e];
  }
  g.additive = d->additive != 0;
  if (g.additive) {
    // blocks of 1-D grids, one after the other
    m = 0;
    for (int e = 0; e < d->dim; ++e) {
      g.off[e] = m;
      m += g.g[e];
    }
  }
  if (m > (int64_t(1) << 30)) return LOVE_ERR_UNSUPPORTED;
  g.m = m;
  int64_t st = 1;
  for (int e = d->dim - 1; e >= 0; --e) {
    g.stride[e] = g.additive ? 1 : st;
    st *= g.g[e];
  }
  for (int e = d->dim; e < LOVE_MAX_DIM; ++e) g.stride[e] = 1;
  g.sf = d->outputscale;
  g.noise = d->noise;
  for (int e = 0; e < d->dim; ++e)
    for (int q = 0; q < 4; ++q) {
      double r = q * g.h[e];
      double ls = g.ls[e];
      double v = std::exp(-(r * r) / (2 * ls * ls));
      g.cloc[e][q] = v;
      g.cloc_dl[e][q] = v * r * r / (ls * ls * ls);
    }
  return LOVE_OK;
}

Allocator make_alloc(const love_allocator* a) {
  Allocator al;
  if (a && a->alloc && a->free) {
    al.a = *a;
    al.user = true;
  }
  return al;
}

int round_up(int v, int q) { return (v + q - 1) / q * q; }

// CUDA events around the pre-compute phases (reported by love_cache_info)
// Auxiliary streams for work that overlaps a call's main stream (kept for the
// process's lifetime, handed out round-robin).
cudaStream_t aux_stream() {
  static std::mutex mu;
  static std::vector<cudaStream_t> pool;
  static unsigned next = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (pool.empty()) {
    for (int i = 0; i < 16; ++i) {
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) pool.push_back(st);
    }
    if (pool.empty()) return nullptr;
  }
  return pool[next++ % pool.size()];
}

// High-priority streams (one per device, kept for the process's lifetime) for
// the Lanczos run while the mean solve runs beside it on an auxiliary stream:
// the block scheduler then fills freed SMs with the Lanczos kernels' CTAs first.
cudaStream_t priority_stream() {
  static std::mutex mu;
  static std::vector<cudaStream_t> per_dev;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1, nullptr);
  if (!per_dev[dev]) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest) == cudaSuccess) per_dev[dev] = st;
    else cudaGetLastError();
  }
  return per_dev[dev];
}

struct PhaseEvents {
  cudaEvent_t e[5] = {};
  bool ok = true;
  PhaseEvents() {
    for (auto& x : e) ok &= cudaEventCreate(&x) == cudaSuccess;
  }
  ~PhaseEvents() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  void record(int i, cudaStream_t s) {
    if (ok) cudaEventRecord(e[i], s);
  }
  void elapsed(float* out) {
    for (int i = 0; i < 4; ++i) {
      out[i] = 0.f;
      if (ok) cudaEventElapsedTime(&out[i], e[i], e[i + 1]);
    }
  }
};

void destroy_cache_buffers(love_cache* c, cudaStream_t s) {
  const Allocator& al = c->alloc;
  const int64_t m = c->grid.m;
  al.free(c->Rc, (size_t)m * c->ld * dtype_size(c->cache_dtype), s);
  al.free(c->S, (size_t)m * c->ld_s * dtype_size(c->dtype), s);
  al.free(c->P, (size_t)m * c->k_eff * dtype_size(c->dtype), s);
  al.free(c->KdP, (size_t)c->grid.dim * m * c->ld_g * dtype_size(c->dtype), s);
  al.free(c->B, (size_t)c->grid.dim * c->k_eff * c->k_eff * dtype_size(c->dtype), s);
  al.free(c->Minv, (size_t)c->k_eff * c->k_eff * dtype_size(c->dtype), s);
  al.free(c->status, sizeof(DevStatus), s);
  al.free(c->sws, c->sws_bytes, s);
  c->sws = nullptr;
  c->sws_bytes = 0;
  delete[] c->alpha;
  delete[] c->beta;
  c->Rc = c->S = c->P = c->KdP = c->B = c->Minv = nullptr;
  c->status = nullptr;
}

love_cache* new_cache(const GridHost& g, love_dtype dt, love_dtype cdt, unsigned flags, int k, const Allocator& al,
                      cudaStream_t s) {
  love_cache* c = new (std::nothrow) love_cache();
  if (!c) return nullptr;
  c->grid = g;
  c->dtype = dt;
  c->cache_dtype = cdt;
  c->flags = flags;
  c->k_eff = k;
  c->alloc = al;
  int vec = (int)(16 / dtype_size(cdt));
  c->ld = round_up(k + 1, vec);
  c->alpha = new double[k + 1]();
  c->beta = new double[k + 1]();
  c->status = (DevStatus*)al.alloc(sizeof(DevStatus), s);
  c->Rc = al.alloc((size_t)g.m * c->ld * dtype_size(cdt), s);
  if (!c->status || !c->Rc) {
    destroy_cache_buffers(c, s);
    delete c;
    return nullptr;
  }
  cudaMemsetAsync(c->status, 0, sizeof(DevStatus), s);
  return c;
}

__global__ void k_import_pack(const double* __restrict__ Rt, int k, const double* __restrict__ a, int64_t m,
                              int ld, int cdt, void* out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * ld) return;
  int64_t r = idx / ld;
  int c = (int)(idx - r * ld);
  double v = 0.0;
  if (c < k) v = Rt[r * k + c];
  else if (c == k && a) v = a[r];
  if (cdt == LOVE_BF16) ((__nv_bfloat16*)out)[idx] = __double2bfloat16(v);
  else if (cdt == LOVE_F64) ((double*)out)[idx] = v;
  else ((float*)out)[idx] = (float)v;
}
// row-major m x k doubles -> column-major m x k of dtype (or row-major with ld)
__global__ void k_import_colmajor(const double* __restrict__ src, int k, int64_t m, int dbl, void* out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * k) return;
  int64_t r = idx / k;
  int c = (int)(idx - r * k);
  if (dbl) ((double*)out)[(int64_t)c * m + r] = src[idx];
  else ((float*)out)[(int64_t)c * m + r] = (float)src[idx];
}
__global__ void k_import_rows(const double* __restrict__ src, int k, int64_t m, int ld, int dbl, void* out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * ld) return;
  int64_t r = idx / ld;
  int c = (int)(idx - r * ld);
  double v = c < k ? src[r * k + c] : 0.0;
  if (dbl) ((double*)out)[idx] = v;
  else ((float*)out)[idx] = (float)v;
}

// columns [0, k) of the predict cache (m x ld rows of the cache dtype) as a
// column-major m x k array of the data dtype T: the sampler's Rt operand
template <typename T>
__global__ void k_rc_to_cols(const void* __restrict__ Rc, int cdt, int64_t m, int ld, int k, T* __restrict__ out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * k) return;
  const int c = (int)(idx / m);
  const int64_t r = idx - (int64_t)c * m;
  const int64_t src = r * ld + c;
  double v;
  if (cdt == LOVE_BF16) v = (double)__bfloat162float(((const __nv_bfloat16*)Rc)[src]);
  else if (cdt == LOVE_F64) v = ((const double*)Rc)[src];
  else v = (double)((const float*)Rc)[src];
  out[idx] = (T)v;
}

template <typename T>
love_status sampler_for_cache(love_cache* c, int ks, uint64_t seed, cudaStream_t s) {
  const GridHost& g = c->grid;
  const Allocator& al = c->alloc;
  const int64_t m = g.m;
  const int k = c->k_eff;
  ks = std::min<int64_t>(ks, m);
  FftPlan plans[LOVE_MAX_DIM];
  love_status rc = LOVE_OK;
  for (int e = 0; e < g.dim && rc == LOVE_OK; ++e)
    rc = fft_plan_create(plans[e], g, e, al, s, c->dtype == LOVE_F32);
  const size_t rb = sizeof(T) * (size_t)m * k;
  T* rt = rc == LOVE_OK ? (T*)al.alloc(rb, s) : nullptr;
  if (rc == LOVE_OK && !rt) rc = LOVE_ERR_OOM;
  PhaseEvents ev;
  ev.record(3, s);
  if (rc == LOVE_OK) {
    LOVE_COUNT_LAUNCH(); k_rc_to_cols<T><<<ceil_div(m * k, 256), 256, 0, s>>>(c->Rc, (int)c->cache_dtype, m, c->ld, k, rt);
    rc = cuda_check(cudaGetLastError());
  }
  // the same breakdown tolerance as the sampler run of love_precompute (FP64 vectors)
  if (rc == LOVE_OK) rc = sampler_build<T>(g, plans, al, c, rt, ks, seed, 1e-12, s);
  ev.record(4, s);
  if (rt) al.free(rt, rb, s);
  for (int e = 0; e < g.dim; ++e) fft_plan_destroy(plans[e], al, s);
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc == LOVE_OK) {
    c->flags |= LOVE_WANT_SAMPLER;
    float ms = 0.f;
    if (ev.ok && cudaEventElapsedTime(&ms, ev.e[3], ev.e[4]) == cudaSuccess) c->phase_ms[3] = ms;
  }
  return rc;
}

double bf16_to_double(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

}  // namespace

extern "C" {

const char* love_status_string(love_status s) {
  switch (s) {
    case LOVE_OK: return "ok";
    case LOVE_ERR_ARG: return "invalid argument";
    case LOVE_ERR_DOMAIN: return "point outside the interpolable grid (or NaN)";
    case LOVE_ERR_NOT_PD: return "tridiagonal matrix not positive definite";
    case LOVE_ERR_NAN: return "NaN or Inf in a reduction";
    case LOVE_ERR_OOM: return "out of device memory";
    case LOVE_ERR_CUDA: return "CUDA runtime error";
    case LOVE_ERR_TIMEOUT: return "bounded device wait expired";
    case LOVE_ERR_STATE: return "handle lacks what the call needs";
    case LOVE_ERR_UNSUPPORTED: return "configuration not supported by this library";
  }
  return "unknown status";
}

int love_last_cuda_error(void) { return g_last_cuda_error; }
uint64_t love_launch_count(void) { return g_launches.load(); }
const char* love_version(void) { return "love-gb300 1.0 (sm_103a)"; }

love_status ski_destroy(love_ski_t ski) try {
  if (!ski) return LOVE_ERR_ARG;
  cudaStream_t s = 0;
  const Allocator& al = ski->alloc;
  size_t es = dtype_size(ski->dtype);
  al.free(ski->xs, (size_t)ski->n_pad * ski->grid.dim * es, s);
  al.free(ski->ys, (size_t)ski->n_pad * es, s);
  al.free(ski->perm, (size_t)ski->n * 4, s);
  al.free(ski->cell_start, (size_t)(ski->grid.m + 1) * 4, s);
  al.free(ski->status, sizeof(DevStatus), s);
  for (int e = 0; e < ski->grid.dim; ++e) {
    fft_plan_destroy(ski->fft[e], al, s);
    al.free(ski->xs1[e], (size_t)ski->n_pad * es, s);
    if (e > 0) al.free(ski->cs1[e], (size_t)(ski->grid.g[e] + 1) * 4, s);
    al.free(ski->map1[e], (size_t)ski->n * 4, s);
  }
  cudaStreamSynchronize(s);
  delete ski;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status ski_build(const love_ski_desc* desc, const void* x_train, const void* y_train, love_stream_t stream,
                      love_ski_t* out) try {
  if (!desc || !x_train || !out) return LOVE_ERR_ARG;
  *out = nullptr;
  if (desc->n < 1 || desc->n > (int64_t(1) << 31) - 1024) return LOVE_ERR_ARG;
  if (desc->dtype != LOVE_F32 && desc->dtype != LOVE_F64) return LOVE_ERR_ARG;
  GridHost g;
  LOVE_TRY(grid_from_desc(desc, g));
  cudaStream_t s = cs(stream);
  love_ski* ski = new (std::nothrow) love_ski();
  if (!ski) return LOVE_ERR_OOM;
  ski->grid = g;
  ski->dtype = desc->dtype;
  ski->n = desc->n;
  ski->n_pad = (desc->n + 255) / 256 * 256;
  ski->alloc = make_alloc(desc->allocator);
  cudaGetDevice(&ski->device);
  const Allocator& al = ski->alloc;
  size_t es = dtype_size(ski->dtype);
  ski->xs = al.alloc((size_t)ski->n_pad * g.dim * es, s);
  ski->ys = y_train ? al.alloc((size_t)ski->n_pad * es, s) : nullptr;
  ski->perm = (int32_t*)al.alloc((size_t)ski->n * 4, s);
  ski->cell_start = (int32_t*)al.alloc((size_t)(g.m + 1) * 4, s);
  ski->status = (DevStatus*)al.alloc(sizeof(DevStatus), s);
  if (!ski->xs || (y_train && !ski->ys) || !ski->perm || !ski->cell_start || !ski->status) {
    ski_destroy(ski);
    return LOVE_ERR_OOM;
  }
  love_status rc = cuda_check(cudaMemsetAsync(ski->status, 0, sizeof(DevStatus), s));
  for (int e = 0; e < g.dim && rc == LOVE_OK; ++e)
    rc = fft_plan_create(ski->fft[e], g, e, al, s, ski->dtype == LOVE_F32);
  if (rc == LOVE_OK) rc = sort_training_points(ski, x_train, y_train, s);
  if (rc == LOVE_OK && g.additive) rc = sort_additive_dims(ski, s);
  DevStatus st{};
  if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(&st, ski->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc == LOVE_OK && st.domain_errors) rc = LOVE_ERR_DOMAIN;
  if (rc != LOVE_OK) {
    ski_destroy(ski);
    return rc;
  }
  *out = ski;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status ski_mvm(love_ski_t ski, const void* v, void* out, love_stream_t stream) try {
  if (!ski || !v || !out || v == out) return LOVE_ERR_ARG;
  cudaStream_t s = cs(stream);
  const Allocator& al = ski->alloc;
  size_t es = dtype_size(ski->dtype);
  const GridHost& g = ski->grid;
  size_t fwb = fft_work_bytes(g, ski->fft, 1, ski->dtype == LOVE_F64);
  size_t wb = es * (size_t)g.m * 2 + fwb + 256;
  size_t vb = es * (size_t)ski->n_pad;
  void* work = al.alloc(wb, s);
  void* vs = al.alloc(vb, s);
  void* ys = al.alloc(vb, s);
  love_status rc = (work && vs && ys) ? LOVE_OK : LOVE_ERR_OOM;
  if (rc == LOVE_OK) {
    if (ski->dtype == LOVE_F64) {
      rc = permute_in<double>((const double*)v, ski->perm, ski->n, ski->n_pad, (double*)vs, s);
      if (rc == LOVE_OK) rc = ski_mvm_sorted<double>(ski, (const double*)vs, (double*)ys, work, s);
      if (rc == LOVE_OK) rc = permute_out<double>((const double*)ys, ski->perm, ski->n, (double*)out, s);
    } else {
      rc = permute_in<float>((const float*)v, ski->perm, ski->n, ski->n_pad, (float*)vs, s);
      if (rc == LOVE_OK) rc = ski_mvm_sorted<float>(ski, (const float*)vs, (float*)ys, work, s);
      if (rc == LOVE_OK) rc = permute_out<float>((const float*)ys, ski->perm, ski->n, (float*)out, s);
    }
  }
  al.free(work, wb, s);
  al.free(vs, vb, s);
  al.free(ys, vb, s);
  return rc;
}
LOVE_ENTRY_CATCH

love_status ski_mvm_kuu(love_ski_t ski, const void* v, void* out, love_stream_t stream) try {
  if (!ski || !v || !out) return LOVE_ERR_ARG;
  cudaStream_t s = cs(stream);
  const GridHost& g = ski->grid;
  size_t fwb = fft_work_bytes(g, ski->fft, 1, ski->dtype == LOVE_F64);
  void* fw = fwb ? ski->alloc.alloc(fwb, s) : nullptr;
  if (fwb && !fw) return LOVE_ERR_OOM;
  love_status rc;
  if (ski->dtype == LOVE_F64)
    rc = kuu_apply<double>(g, ski->fft, (const double*)v, (double*)out, 1, g.m, fw, -1, s);
  else
    rc = kuu_apply<float>(g, ski->fft, (const float*)v, (float*)out, 1, g.m, fw, -1, s);
  if (fw) ski->alloc.free(fw, fwb, s);
  return rc;
}
LOVE_ENTRY_CATCH

love_status love_cache_destroy(love_cache_t c) try {
  if (!c) return LOVE_ERR_ARG;
  destroy_cache_buffers(c, 0);
  cudaStreamSynchronize(0);
  delete c;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

}  // extern "C"

// The grid-space mean CG needs only the training data, not the Lanczos
// basis, so it runs on an auxiliary stream, driven by its own host thread,
// while the Lanczos, cache and sampler kernels run on the caller's stream;
// its mean weights are written into the cache after both finish.
struct MeanJob {
  std::thread th;
  love_status rc = LOVE_OK;
  int iters = 0;
  float ms = 0.f;
  ~MeanJob() {
    if (th.joinable()) th.join();
  }
};

// pre_Q / pre: the Lanczos run already made (by the batched run): Q (k columns,
// from ski's allocator; owned from here on) and its scalars
template <typename T>
static love_status precompute_impl(love_ski* ski, const love_precompute_opts* o, cudaStream_t s, love_cache** out,
                                   int* k_eff_out, T* pre_Q = nullptr, const BatchedLanczos::Gp* pre = nullptr,
                                   int pre_rows = 0) {
  const GridHost& g = ski->grid;
  const Allocator& al = ski->alloc;
  int k = std::min<int64_t>(o->k, std::min<int64_t>(ski->n, g.m));
  double tau = o->breakdown_tol > 0 ? o->breakdown_tol : (sizeof(T) == 8 ? 1e-12 : 1e-8);
  if (o->reorth != LOVE_REORTH_ALWAYS && o->reorth != LOVE_REORTH_DETECT && o->reorth != LOVE_REORTH_LOWSYNC)
    return LOVE_ERR_ARG;
  // DETECT / LOWSYNC: skip the second pass while |Q_j^T y'| <= eta |y'|, eta =
  // 4 units of rounding of the Q storage type unless given
  const bool lowsync = o->reorth == LOVE_REORTH_LOWSYNC;
  const double eta = o->reorth == LOVE_REORTH_ALWAYS
                         ? 0.0
                         : (o->reorth_eta > 0 ? o->reorth_eta : (sizeof(T) == 8 ? 0x1p-51 : 0x1p-22));
  unsigned flags = o->flags;
  if (!ski->ys) flags &= ~LOVE_WANT_MEAN;
  const bool want_mean = (flags & LOVE_WANT_MEAN) != 0;
  const bool grid_cg = want_mean && mean_grid_cg_supported(ski);
  const double cg_tol = o->cg_tol > 0 ? o->cg_tol : (sizeof(T) == 8 ? 1e-12 : 1e-6);
  const int cg_maxit = o->cg_max_iter > 0 ? o->cg_max_iter : 4000;
  const int64_t ldq = ski->n_pad;
  size_t qb = sizeof(T) * (size_t)ldq * k;
  const size_t amb = sizeof(double) * (size_t)g.m;
  double* am = nullptr;  // mean weights from the grid CG
  if (grid_cg) {
    am = (double*)al.alloc(amb, s);
    if (!am) return LOVE_ERR_OOM;
  }
  T* Q = pre_Q ? pre_Q : (T*)al.alloc(qb, s);
  if (!Q) {
    al.free(am, amb, s);
    return LOVE_ERR_OOM;
  }
  MeanJob mj;
  if (grid_cg) {
    cudaStream_t s2 = aux_stream();
    cudaEvent_t go = nullptr;
    love_status erc = cuda_check(cudaEventCreateWithFlags(&go, cudaEventDisableTiming));
    if (erc == LOVE_OK) erc = cuda_check(cudaEventRecord(go, s));
    if (erc == LOVE_OK) erc = cuda_check(cudaStreamWaitEvent(s2, go, 0));
    if (go) cudaEventDestroy(go);
    if (erc != LOVE_OK) {
      al.free(Q, qb, s);
      al.free(am, amb, s);
      return erc;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    const bool precond = o->cg_plain == 0;
    try {
      ScratchCache* mean_cache = thread_mean_scratch();
      mj.th = std::thread([ski, cg_tol, cg_maxit, am, s2, dev, precond, &mj, mean_cache] {
        cudaSetDevice(dev);
        thread_scratch() = mean_cache;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s2);
        try {
          mj.rc = mean_grid_cg<T>(ski, cg_tol, cg_maxit, am, &mj.iters, s2, precond);
        } catch (...) {   // host memory ran out: an exception must not leave the thread
          mj.rc = LOVE_ERR_OOM;
        }
        cudaEventRecord(e1, s2);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&mj.ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
      });
    } catch (...) {   // no host thread to be had
      al.free(Q, qb, s);
      al.free(am, amb, s);
      return LOVE_ERR_OOM;
    }
  }
  auto join_mean = [&]() {
    if (mj.th.joinable()) mj.th.join();
  };
  std::vector<double> alpha(k + 1), beta(k + 1);
  int keff = 0, skipped = 0;
  PhaseEvents ev;
  ev.record(0, s);
  float reorth_ms = 0.f;
  love_status rc = LOVE_OK;
  if (pre) {
    std::copy(pre->alpha.begin(), pre->alpha.begin() + std::min<size_t>(pre->alpha.size(), k), alpha.begin());
    std::copy(pre->beta.begin(), pre->beta.begin() + std::min<size_t>(pre->beta.size(), k), beta.begin());
    keff = pre->k_eff;
    skipped = pre->skipped;
  } else {
    // beside a mean solve, the Lanczos run goes to a high-priority stream,
    // ordered after the caller's stream and joined back to it
    cudaStream_t ls = grid_cg ? priority_stream() : nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (ls && (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(ls, fork, 0) != cudaSuccess)) {
      cudaGetLastError();
      ls = nullptr;
    }
    rc = lanczos_run<T>(ski, k, tau, eta, Q, ldq, alpha.data(), beta.data(), &keff, &skipped, ls ? ls : s,
                        (flags & LOVE_TIME_REORTH) ? &reorth_ms : nullptr, lowsync);
    if (ls) {
      love_status jrc = cuda_check(cudaEventRecord(join, ls));
      if (jrc == LOVE_OK) jrc = cuda_check(cudaStreamWaitEvent(s, join, 0));
      if (jrc != LOVE_OK) jrc = cuda_check(cudaStreamSynchronize(ls));   // ordered by the host instead
      if (rc == LOVE_OK) rc = jrc;
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
  ev.record(1, s);
  if (rc != LOVE_OK) {
    join_mean();
    al.free(Q, qb, s);
    al.free(am, amb, s);
    return rc;
  }
  // status from the Lanczos kernels (NaN, timeout)
  DevStatus dst{};
  cudaMemcpyAsync(&dst, ski->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (dst.bits & (1u << LOVE_ERR_TIMEOUT)) rc = LOVE_ERR_TIMEOUT;
  else if (dst.bits & (1u << LOVE_ERR_NAN)) rc = LOVE_ERR_NAN;
  if (rc == LOVE_OK && keff < 1) rc = LOVE_ERR_NAN;
  if (rc != LOVE_OK) {
    join_mean();
    cudaMemsetAsync(ski->status, 0, sizeof(DevStatus), s);
    al.free(Q, qb, s);
    al.free(am, amb, s);
    return rc;
  }
  love_cache* c = new_cache(g, ski->dtype, o->cache_dtype, flags, keff, al, s);
  if (!c) {
    join_mean();
    al.free(Q, qb, s);
    al.free(am, amb, s);
    return LOVE_ERR_OOM;
  }
  c->reorth_skipped = skipped;
  c->reorth_ms = reorth_ms;
  c->batched_rows = pre_rows;
  std::copy(alpha.begin(), alpha.begin() + keff, c->alpha);
  std::copy(beta.begin(), beta.begin() + std::max(keff - 1, 0), c->beta);
  // n-space mean CG (3-D grids), on this stream
  double* z = nullptr;
  const size_t zb = sizeof(double) * (size_t)ldq;
  if (want_mean && !grid_cg) {
    z = (double*)al.alloc(zb, s);
    if (!z) rc = LOVE_ERR_OOM;
    if (rc == LOVE_OK) rc = cg_solve<T>(ski, (const T*)ski->ys, z, cg_tol, cg_maxit, &c->cg_iters, s);
  }
  ev.record(2, s);
  if (rc == LOVE_OK && (flags & LOVE_WANT_GRAD)) {
    c->P = al.alloc(sizeof(T) * (size_t)g.m * keff, s);
    if (!c->P) rc = LOVE_ERR_OOM;
  }
  T* rt_keep = nullptr;
  size_t rtb = sizeof(T) * (size_t)g.m * keff;
  if (rc == LOVE_OK && (flags & LOVE_WANT_SAMPLER)) {
    rt_keep = (T*)al.alloc(rtb, s);
    if (!rt_keep) rc = LOVE_ERR_OOM;
  }
  if (rc == LOVE_OK) rc = build_cache<T>(ski, c, Q, ldq, z, s, rt_keep, nullptr);
  if (rc == LOVE_OK && (flags & LOVE_WANT_GRAD)) rc = backward_tables(c, ski->fft, c->P, keff, s);
  ev.record(3, s);
  if (z) al.free(z, zb, s);
  al.free(Q, qb, s);
  if (rc == LOVE_OK && (flags & LOVE_WANT_SAMPLER)) {
    int ks = o->sampler_k > 0 ? o->sampler_k : o->k;
    ks = std::min<int64_t>(ks, g.m);
    // breakdown tolerance of the sampler's Lanczos run: its vectors are FP64
    rc = sampler_build<T>(ski->grid, ski->fft, ski->alloc, c, rt_keep, ks, o->sampler_seed, 1e-12, s);
  }
  if (rt_keep) al.free(rt_keep, rtb, s);
  ev.record(4, s);
  // the grid CG's mean weights into the cache's mean column
  join_mean();
  if (grid_cg) {
    if (rc == LOVE_OK) rc = mj.rc;
    c->cg_iters = mj.iters;
    if (rc == LOVE_OK) rc = cache_set_mean(c, am, s);
  }
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  al.free(am, amb, s);
  if (rc == LOVE_OK) {
    ev.elapsed(c->phase_ms);
    if (grid_cg) c->phase_ms[1] = mj.ms;
  }
  if (rc != LOVE_OK) {
    love_cache_destroy(c);
    return rc;
  }
  *out = c;
  if (k_eff_out) *k_eff_out = keff;
  return LOVE_OK;
}

namespace love {

love_status precompute_opts_check(const love_ski* ski, const love_precompute_opts* opts) {
  if (opts->k < 1 || opts->k > LOVE_MAX_K) return LOVE_ERR_ARG;
  if (ski->dtype == LOVE_F64 && opts->cache_dtype != LOVE_F64) return LOVE_ERR_ARG;
  if (ski->dtype == LOVE_F32 && opts->cache_dtype == LOVE_F64) return LOVE_ERR_ARG;
  if (opts->sampler_k > LOVE_MAX_K) return LOVE_ERR_ARG;
  if (ski->grid.additive && (opts->flags & LOVE_WANT_GRAD)) return LOVE_ERR_UNSUPPORTED;
  return LOVE_OK;
}

int precompute_k(const love_ski* ski, const love_precompute_opts* o) {
  return (int)std::min<int64_t>(o->k, std::min<int64_t>(ski->n, ski->grid.m));
}

void precompute_lanczos_params(const love_ski* ski, const love_precompute_opts* o, double* tau, double* eta) {
  const bool f64 = ski->dtype == LOVE_F64;
  *tau = o->breakdown_tol > 0 ? o->breakdown_tol : (f64 ? 1e-12 : 1e-8);
  *eta = o->reorth == LOVE_REORTH_ALWAYS ? 0.0 : (o->reorth_eta > 0 ? o->reorth_eta : (f64 ? 0x1p-51 : 0x1p-22));
}

love_status precompute_from_lanczos(love_ski* ski, const love_precompute_opts* opts, cudaStream_t s, float* Q,
                                    const BatchedLanczos::Gp& r, int rows, float lanczos_ms, love_cache** out,
                                    int* k_eff) {
  *out = nullptr;
  const love_status rc = precompute_opts_check(ski, opts);
  if (rc != LOVE_OK || ski->dtype != LOVE_F32) {
    ski->alloc.free(Q, sizeof(float) * (size_t)ski->n_pad * precompute_k(ski, opts), s);
    return rc != LOVE_OK ? rc : LOVE_ERR_ARG;
  }
  const love_status prc = precompute_impl<float>(ski, opts, s, out, k_eff, Q, &r, rows);
  if (prc == LOVE_OK) (*out)->phase_ms[0] = lanczos_ms;   // the whole batch's run
  return prc;
}

}  // namespace love

extern "C" {

love_status love_precompute(love_ski_t ski, const love_precompute_opts* opts, love_stream_t stream,
                            love_cache_t* out, int* k_eff) try {
  if (!ski || !opts || !out) return LOVE_ERR_ARG;
  *out = nullptr;
  LOVE_TRY(precompute_opts_check(ski, opts));
  cudaStream_t s = cs(stream);
  if (ski->dtype == LOVE_F64) return precompute_impl<double>(ski, opts, s, out, k_eff);
  return precompute_impl<float>(ski, opts, s, out, k_eff);
}
LOVE_ENTRY_CATCH

love_status love_predict_mean_var(love_cache_t c, int64_t t, const void* x_test, void* mean, void* var,
                                  love_stream_t stream) try {
  if (!c || t < 0) return LOVE_ERR_ARG;
  if (t == 0) return LOVE_OK;
  if (!x_test || !var) return LOVE_ERR_ARG;
  if (mean && !(c->flags & LOVE_WANT_MEAN)) return LOVE_ERR_STATE;
  return predict_launch(c, t, x_test, mean, var, cs(stream));
}
LOVE_ENTRY_CATCH

// device address of a page-locked host buffer, or nullptr (pageable memory)
static void* host_mapped(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

love_status love_predict_mean_var_host(love_cache_t c, int64_t t, const void* x_test, void* mean, void* var,
                                       love_stream_t stream) try {
  if (!c || t < 0) return LOVE_ERR_ARG;
  if (t == 0) return LOVE_OK;
  if (!x_test || !var) return LOVE_ERR_ARG;
  if (mean && !(c->flags & LOVE_WANT_MEAN)) return LOVE_ERR_STATE;
  cudaStream_t s = cs(stream);
  void* dx = host_mapped(x_test);
  void* dv = host_mapped(var);
  void* dm = mean ? host_mapped(mean) : nullptr;
  if (dx && dv && (!mean || dm)) {
    // page-locked: the kernel reads x and writes the results over the link
    LOVE_TRY(predict_launch(c, t, dx, dm, dv, s));
    return cuda_check(cudaStreamSynchronize(s));
  }
  const size_t es = dtype_size(c->dtype);
  const int dim = c->grid.dim;
  const int64_t chunk = std::min<int64_t>(t, int64_t(1) << 20);
  const size_t xb = es * (size_t)chunk * dim, ob = es * (size_t)chunk;
  void* bx = c->alloc.alloc(xb, s);
  void* bv = c->alloc.alloc(ob, s);
  void* bm = mean ? c->alloc.alloc(ob, s) : nullptr;
  love_status rc = (bx && bv && (!mean || bm)) ? LOVE_OK : LOVE_ERR_OOM;
  for (int64_t o = 0; o < t && rc == LOVE_OK; o += chunk) {
    const int64_t n = std::min(chunk, t - o);
    rc = cuda_check(cudaMemcpyAsync(bx, (const char*)x_test + es * (size_t)o * dim, es * (size_t)n * dim,
                                    cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK) rc = predict_launch(c, n, bx, bm, bv, s);
    if (rc == LOVE_OK)
      rc = cuda_check(cudaMemcpyAsync((char*)var + es * (size_t)o, bv, es * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (rc == LOVE_OK && mean)
      rc = cuda_check(cudaMemcpyAsync((char*)mean + es * (size_t)o, bm, es * (size_t)n, cudaMemcpyDeviceToHost, s));
  }
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  c->alloc.free(bx, xb, s);
  c->alloc.free(bv, ob, s);
  if (bm) c->alloc.free(bm, ob, s);
  return rc;
}
LOVE_ENTRY_CATCH

love_status love_predict_covariance(love_cache_t c, int64_t t1, const void* x1, int64_t t2, const void* x2,
                                    void* cov, love_stream_t stream) try {
  if (!c || t1 < 0 || t2 < 0) return LOVE_ERR_ARG;
  if (c->grid.additive) return LOVE_ERR_UNSUPPORTED;
  if (t1 == 0 || t2 == 0) return LOVE_OK;
  if (!x1 || !x2 || !cov) return LOVE_ERR_ARG;
  return cov_launch(c, t1, x1, t2, x2, cov, cs(stream));
}
LOVE_ENTRY_CATCH

love_status love_predict_var_root(love_cache_t c, int64_t t, const void* x_test, void* var, love_stream_t stream) try {
  if (!c || t < 0) return LOVE_ERR_ARG;
  if (!c->S) return LOVE_ERR_STATE;
  if (t == 0) return LOVE_OK;
  if (!x_test || !var) return LOVE_ERR_ARG;
  return predict_root_launch(c, t, x_test, var, cs(stream));
}
LOVE_ENTRY_CATCH

love_status love_sample(love_cache_t c, int64_t t, const void* x_test, int s_count, const void* z, uint64_t seed,
                        void* out, love_stream_t stream) try {
  if (!c || t < 0 || s_count < 0) return LOVE_ERR_ARG;
  if (!c->S) return LOVE_ERR_STATE;
  if (t == 0 || s_count == 0) return LOVE_OK;
  if (!x_test || !out) return LOVE_ERR_ARG;
  // work space kept on the cache: no allocator call once it is large enough
  const size_t need = sample_ws_bytes(c, t, s_count);
  if (need > c->sws_bytes) {
    c->alloc.free(c->sws, c->sws_bytes, cs(stream));
    c->sws = c->alloc.alloc(need, cs(stream));
    c->sws_bytes = c->sws ? need : 0;
    if (!c->sws) return LOVE_ERR_OOM;
  }
  return sample_launch_z_ws(c, t, x_test, s_count, z, seed, out, c->sws, cs(stream));
}
LOVE_ENTRY_CATCH

love_status love_sampler_precompute(love_cache_t c, int ks, uint64_t seed, love_stream_t stream) try {
  if (!c || ks < 0 || ks > LOVE_MAX_K) return LOVE_ERR_ARG;
  if (ks == 0) ks = c->k_eff;
  if (c->dtype == LOVE_F64) return sampler_for_cache<double>(c, ks, seed, cs(stream));
  return sampler_for_cache<float>(c, ks, seed, cs(stream));
}
LOVE_ENTRY_CATCH

love_status love_var_backward(love_cache_t c, int64_t t, const void* x_test, const void* grad_var, void* grad_x,
                              double* grad_lengthscale, double* grad_noise, love_stream_t stream) try {
  if (!c || t < 0) return LOVE_ERR_ARG;
  if (c->grid.additive) return LOVE_ERR_UNSUPPORTED;
  if (!(c->flags & LOVE_WANT_GRAD) || !c->KdP) return LOVE_ERR_STATE;
  if (t > 0 && (!x_test || !grad_var)) return LOVE_ERR_ARG;
  return backward_launch(c, t, x_test, grad_var, grad_x, grad_lengthscale, grad_noise, cs(stream));
}
LOVE_ENTRY_CATCH

love_status love_cache_info(love_cache_t c, love_cache_info_t* info) try {
  if (!c || !info) return LOVE_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  info->dim = c->grid.dim;
  for (int e = 0; e < 3; ++e) info->grid_size[e] = c->grid.g[e];
  info->m = c->grid.m;
  info->k_eff = c->k_eff;
  info->ld = c->ld;
  info->sampler_k = c->ks;
  info->cg_iters = c->cg_iters;
  info->sampler_fallback = c->sampler_fallback;
  info->dtype = c->dtype;
  info->cache_dtype = c->cache_dtype;
  info->flags = c->flags;
  for (int i = 0; i < 4; ++i) info->phase_ms[i] = c->phase_ms[i];
  info->reorth_skipped = c->reorth_skipped;
  info->batched_rows = c->batched_rows;
  info->reorth_ms = c->reorth_ms;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status love_cache_import(const love_ski_desc* desc, int k, love_dtype cache_dtype, unsigned flags,
                              const double* Rt, const double* a, int ks, const double* S, const double* alpha,
                              const double* beta, const double* P, love_stream_t stream, love_cache_t* out) try {
  if (!desc || !Rt || !out || k < 1 || k > LOVE_MAX_K || ks < 0 || ks > LOVE_MAX_K) return LOVE_ERR_ARG;
  if (desc->dtype != LOVE_F32 && desc->dtype != LOVE_F64) return LOVE_ERR_ARG;
  if (desc->dtype == LOVE_F64 && cache_dtype != LOVE_F64) return LOVE_ERR_ARG;
  if (desc->dtype == LOVE_F32 && cache_dtype == LOVE_F64) return LOVE_ERR_ARG;
  if ((flags & LOVE_WANT_GRAD) && (!P || !alpha || !beta)) return LOVE_ERR_ARG;
  if ((flags & LOVE_WANT_SAMPLER) && (!S || ks < 1)) return LOVE_ERR_ARG;
  *out = nullptr;
  GridHost g;
  LOVE_TRY(grid_from_desc(desc, g));
  cudaStream_t s = cs(stream);
  Allocator al = make_alloc(desc->allocator);
  if (!a) flags &= ~LOVE_WANT_MEAN;
  love_cache* c = new_cache(g, desc->dtype, cache_dtype, flags, k, al, s);
  if (!c) return LOVE_ERR_OOM;
  if (alpha) std::copy(alpha, alpha + k, c->alpha);
  if (beta && k > 1) std::copy(beta, beta + k - 1, c->beta);
  const int64_t m = g.m;
  const bool dbl = desc->dtype == LOVE_F64;
  love_status rc = LOVE_OK;
  size_t hb = sizeof(double) * (size_t)m * (size_t)std::max(k, ks) + sizeof(double) * m;
  double* h = (double*)al.alloc(hb, s);
  if (!h) rc = LOVE_ERR_OOM;
  if (rc == LOVE_OK) {
    rc = cuda_check(cudaMemcpyAsync(h, Rt, sizeof(double) * m * k, cudaMemcpyHostToDevice, s));
    double* ad = nullptr;
    if (rc == LOVE_OK && a) {
      ad = h + (size_t)m * std::max(k, ks);
      rc = cuda_check(cudaMemcpyAsync(ad, a, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    }
    if (rc == LOVE_OK) {
      LOVE_COUNT_LAUNCH(); k_import_pack<<<ceil_div(m * c->ld, 256), 256, 0, s>>>(h, k, ad, m, c->ld, (int)cache_dtype, c->Rc);
      rc = cuda_check(cudaGetLastError());
    }
  }
  if (rc == LOVE_OK && (flags & LOVE_WANT_SAMPLER)) {
    c->ks = ks;
    c->ld_s = round_up(ks, dbl ? 2 : 4);
    c->S = al.alloc(dtype_size(desc->dtype) * (size_t)m * c->ld_s, s);
    if (!c->S) rc = LOVE_ERR_OOM;
    if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(h, S, sizeof(double) * m * ks, cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK) {
      LOVE_COUNT_LAUNCH(); k_import_rows<<<ceil_div(m * c->ld_s, 256), 256, 0, s>>>(h, ks, m, c->ld_s, dbl, c->S);
      rc = cuda_check(cudaGetLastError());
    }
  }
  if (rc == LOVE_OK && (flags & LOVE_WANT_GRAD)) {
    c->P = al.alloc(dtype_size(desc->dtype) * (size_t)m * k, s);
    if (!c->P) rc = LOVE_ERR_OOM;
    if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(h, P, sizeof(double) * m * k, cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK) {
      LOVE_COUNT_LAUNCH(); k_import_colmajor<<<ceil_div(m * k, 256), 256, 0, s>>>(h, k, m, dbl, c->P);
      rc = cuda_check(cudaGetLastError());
    }
    if (rc == LOVE_OK) {
      FftPlan plans[LOVE_MAX_DIM];
      for (int e = 0; e < g.dim && rc == LOVE_OK; ++e)
        rc = fft_plan_create(plans[e], g, e, al, s, desc->dtype == LOVE_F32);
      if (rc == LOVE_OK) rc = backward_tables(c, plans, c->P, k, s);
      for (int e = 0; e < g.dim; ++e) fft_plan_destroy(plans[e], al, s);
    }
  }
  if (h) al.free(h, hb, s);
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc != LOVE_OK) {
    love_cache_destroy(c);
    return rc;
  }
  *out = c;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status love_cache_export(love_cache_t c, double* Rt, double* a, double* S, double* P, double* alpha,
                              double* beta, love_stream_t stream) try {
  if (!c) return LOVE_ERR_ARG;
  cudaStream_t s = cs(stream);
  const int64_t m = c->grid.m;
  const int k = c->k_eff;
  if (Rt || a) {
    size_t es = dtype_size(c->cache_dtype);
    std::vector<unsigned char> buf((size_t)m * c->ld * es);
    LOVE_CUDA(cudaMemcpyAsync(buf.data(), c->Rc, buf.size(), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    for (int64_t r = 0; r < m; ++r)
      for (int q = 0; q <= k; ++q) {
        size_t idx = (size_t)r * c->ld + q;
        double v;
        if (c->cache_dtype == LOVE_F64) v = ((const double*)buf.data())[idx];
        else if (c->cache_dtype == LOVE_BF16) v = bf16_to_double(((const uint16_t*)buf.data())[idx]);
        else v = ((const float*)buf.data())[idx];
        if (q < k && Rt) Rt[r * k + q] = v;
        if (q == k && a) a[r] = (c->flags & LOVE_WANT_MEAN) ? v : 0.0;
      }
  }
  const bool dbl = c->dtype == LOVE_F64;
  if (S && c->S) {
    std::vector<unsigned char> buf((size_t)m * c->ld_s * (dbl ? 8 : 4));
    LOVE_CUDA(cudaMemcpyAsync(buf.data(), c->S, buf.size(), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    for (int64_t r = 0; r < m; ++r)
      for (int q = 0; q < c->ks; ++q) {
        size_t idx = (size_t)r * c->ld_s + q;
        S[r * c->ks + q] = dbl ? ((const double*)buf.data())[idx] : ((const float*)buf.data())[idx];
      }
  }
  if (P && c->P) {
    std::vector<unsigned char> buf((size_t)m * k * (dbl ? 8 : 4));
    LOVE_CUDA(cudaMemcpyAsync(buf.data(), c->P, buf.size(), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    for (int64_t r = 0; r < m; ++r)
      for (int q = 0; q < k; ++q) {
        size_t idx = (size_t)q * m + r;
        P[r * k + q] = dbl ? ((const double*)buf.data())[idx] : ((const float*)buf.data())[idx];
      }
  }
  if (alpha) std::copy(c->alpha, c->alpha + k, alpha);
  if (beta && k > 1) std::copy(c->beta, c->beta + k - 1, beta);
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status love_get_device_status(love_cache_t c, int reset, love_device_status_t* st, love_stream_t stream) try {
  if (!c || !st) return LOVE_ERR_ARG;
  cudaStream_t s = cs(stream);
  DevStatus d{};
  LOVE_CUDA(cudaMemcpyAsync(&d, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  if (reset) LOVE_CUDA(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  st->bits = d.bits;
  st->domain_errors = (int64_t)d.domain_errors;
  st->clamped = (int64_t)d.clamped;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

// ---- checkpoint ---------------------------------------------------------------
static const char kMagic[8] = {'L', 'O', 'V', 'E', 'C', 'A', 'C', 'H'};
static const uint32_t kVersion = 2;

struct CacheHeader {
  char magic[8];
  uint32_t version;
  int32_t dim;
  int64_t g[3];
  double lo[3], h[3], ls[3];
  double sf, noise;
  int32_t dtype, cache_dtype;
  uint32_t flags;
  int32_t k_eff, ld, ks, ld_s, ld_g, cg_iters, sampler_fallback;
  uint64_t bytes_rc, bytes_s, bytes_p, bytes_kdp, bytes_b, bytes_minv;
  int32_t additive, pad;     // version 2
};

// A cache file is accepted only if its header describes exactly the buffers
// the library writes for such a cache (sizes from the grid, k_eff and the
// dtypes; the gradient tables all present or all absent) and the file holds
// exactly those bytes: any other file could make a kernel read past a buffer.
static bool header_ok(const CacheHeader& hd, uint64_t file_bytes) {
  if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kVersion) return false;
  if (hd.dim < 1 || hd.dim > LOVE_MAX_DIM || hd.k_eff < 1 || hd.k_eff > LOVE_MAX_K) return false;
  if (hd.additive != 0 && hd.additive != 1) return false;
  if (hd.dtype != LOVE_F32 && hd.dtype != LOVE_F64) return false;
  if (hd.dtype == LOVE_F64 ? hd.cache_dtype != LOVE_F64
                           : (hd.cache_dtype != LOVE_F32 && hd.cache_dtype != LOVE_BF16))
    return false;
  if (!(hd.sf > 0) || !(hd.noise > 0) || !std::isfinite(hd.sf) || !std::isfinite(hd.noise)) return false;
  uint64_t m = hd.additive ? 0 : 1;
  for (int e = 0; e < LOVE_MAX_DIM; ++e) {
    if (e >= hd.dim) {
      if (hd.g[e] != 1) return false;
      continue;
    }
    if (hd.g[e] < 4 || hd.g[e] > (int64_t(1) << 30) || !std::isfinite(hd.lo[e]) || !(hd.h[e] > 0) ||
        !std::isfinite(hd.h[e]) || !(hd.ls[e] > 0) || !std::isfinite(hd.ls[e]))
      return false;
    m = hd.additive ? m + (uint64_t)hd.g[e] : m * (uint64_t)hd.g[e];
    if (m > (uint64_t(1) << 34)) return false;
  }
  const uint64_t k = (uint64_t)hd.k_eff;
  const uint64_t cb = dtype_size((love_dtype)hd.cache_dtype), eb = dtype_size((love_dtype)hd.dtype);
  if (hd.ld != round_up(hd.k_eff + 1, (int)(16 / cb)) || hd.bytes_rc != m * (uint64_t)hd.ld * cb) return false;
  if (hd.bytes_s == 0 ? hd.ks != 0
                      : (hd.ks < 1 || hd.ks > LOVE_MAX_K || hd.ld_s != round_up(hd.ks, (int)(16 / eb)) ||
                         hd.bytes_s != m * (uint64_t)hd.ld_s * eb))
    return false;
  const bool grad = hd.bytes_p != 0;
  if (grad) {
    if (hd.ld_g != round_up(hd.k_eff, (int)(16 / eb)) || hd.bytes_p != m * k * eb ||
        hd.bytes_kdp != (uint64_t)hd.dim * m * (uint64_t)hd.ld_g * eb || hd.bytes_b != (uint64_t)hd.dim * k * k * eb ||
        hd.bytes_minv != k * k * eb)
      return false;
  } else if (hd.bytes_kdp != 0 || hd.bytes_b != 0 || hd.bytes_minv != 0) {
    return false;
  }
  const uint64_t total = sizeof(CacheHeader) + 2 * sizeof(double) * k + hd.bytes_rc + hd.bytes_s + hd.bytes_p +
                         hd.bytes_kdp + hd.bytes_b + hd.bytes_minv;
  return total == file_bytes;
}

static love_status write_dev(FILE* f, const void* dptr, size_t bytes, cudaStream_t s) {
  if (!bytes) return LOVE_OK;
  std::vector<unsigned char> buf(bytes);
  LOVE_CUDA(cudaMemcpyAsync(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  return fwrite(buf.data(), 1, bytes, f) == bytes ? LOVE_OK : LOVE_ERR_ARG;
}
static love_status read_dev(FILE* f, void** dptr, size_t bytes, const Allocator& al, cudaStream_t s) {
  if (!bytes) return LOVE_OK;
  std::vector<unsigned char> buf(bytes);
  if (fread(buf.data(), 1, bytes, f) != bytes) return LOVE_ERR_ARG;
  *dptr = al.alloc(bytes, s);
  if (!*dptr) return LOVE_ERR_OOM;
  LOVE_CUDA(cudaMemcpyAsync(*dptr, buf.data(), bytes, cudaMemcpyHostToDevice, s));
  return cuda_check(cudaStreamSynchronize(s));
}

love_status love_cache_save(love_cache_t c, const char* path, love_stream_t stream) try {
  if (!c || !path) return LOVE_ERR_ARG;
  cudaStream_t s = cs(stream);
  CacheHeader hd{};
  std::memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.additive = c->grid.additive ? 1 : 0;
  hd.dim = c->grid.dim;
  for (int e = 0; e < 3; ++e) {
    hd.g[e] = c->grid.g[e];
    hd.lo[e] = c->grid.lo[e];
    hd.h[e] = c->grid.h[e];
    hd.ls[e] = c->grid.ls[e];
  }
  hd.sf = c->grid.sf;
  hd.noise = c->grid.noise;
  hd.dtype = c->dtype;
  hd.cache_dtype = c->cache_dtype;
  hd.flags = c->flags;
  hd.k_eff = c->k_eff;
  hd.ld = c->ld;
  hd.ks = c->ks;
  hd.ld_s = c->ld_s;
  hd.ld_g = c->ld_g;
  hd.cg_iters = c->cg_iters;
  hd.sampler_fallback = c->sampler_fallback;
  const int64_t m = c->grid.m;
  size_t es = dtype_size(c->dtype);
  hd.bytes_rc = (uint64_t)m * c->ld * dtype_size(c->cache_dtype);
  hd.bytes_s = c->S ? (uint64_t)m * c->ld_s * es : 0;
  hd.bytes_p = c->P ? (uint64_t)m * c->k_eff * es : 0;
  hd.bytes_kdp = c->KdP ? (uint64_t)c->grid.dim * m * c->ld_g * es : 0;
  hd.bytes_b = c->B ? (uint64_t)c->grid.dim * c->k_eff * c->k_eff * es : 0;
  hd.bytes_minv = c->Minv ? (uint64_t)c->k_eff * c->k_eff * es : 0;
  FILE* f = std::fopen(path, "wb");
  if (!f) return LOVE_ERR_ARG;
  love_status rc = fwrite(&hd, sizeof(hd), 1, f) == 1 ? LOVE_OK : LOVE_ERR_ARG;
  if (rc == LOVE_OK && fwrite(c->alpha, sizeof(double), c->k_eff, f) != (size_t)c->k_eff) rc = LOVE_ERR_ARG;
  if (rc == LOVE_OK && fwrite(c->beta, sizeof(double), c->k_eff, f) != (size_t)c->k_eff) rc = LOVE_ERR_ARG;
  if (rc == LOVE_OK) rc = write_dev(f, c->Rc, hd.bytes_rc, s);
  if (rc == LOVE_OK) rc = write_dev(f, c->S, hd.bytes_s, s);
  if (rc == LOVE_OK) rc = write_dev(f, c->P, hd.bytes_p, s);
  if (rc == LOVE_OK) rc = write_dev(f, c->KdP, hd.bytes_kdp, s);
  if (rc == LOVE_OK) rc = write_dev(f, c->B, hd.bytes_b, s);
  if (rc == LOVE_OK) rc = write_dev(f, c->Minv, hd.bytes_minv, s);
  std::fclose(f);
  return rc;
}
LOVE_ENTRY_CATCH

love_status love_cache_load(const char* path, const love_allocator* allocator, love_stream_t stream,
                            love_cache_t* out) try {
  if (!path || !out) return LOVE_ERR_ARG;
  *out = nullptr;
  cudaStream_t s = cs(stream);
  FILE* f = std::fopen(path, "rb");
  if (!f) return LOVE_ERR_ARG;
  CacheHeader hd{};
  bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && std::fseek(f, 0, SEEK_END) == 0;
  const long fb = ok ? std::ftell(f) : -1;
  ok = ok && fb >= 0 && header_ok(hd, (uint64_t)fb) && std::fseek(f, (long)sizeof(hd), SEEK_SET) == 0;
  if (!ok) {
    std::fclose(f);
    return LOVE_ERR_ARG;
  }
  love_cache* c = new (std::nothrow) love_cache();
  if (!c) {
    std::fclose(f);
    return LOVE_ERR_OOM;
  }
  try {   // a host allocation that throws below must not leak the file or the cache
    GridHost& g = c->grid;
    g.dim = hd.dim;
    g.additive = hd.additive != 0;
    g.m = 1;
    for (int e = 0; e < 3; ++e) {
      g.g[e] = hd.g[e];
      g.lo[e] = hd.lo[e];
      g.h[e] = hd.h[e];
      g.ls[e] = hd.ls[e];
      g.m *= g.g[e];
    }
    if (g.additive) {
      g.m = 0;
      for (int e = 0; e < g.dim; ++e) {
        g.off[e] = g.m;
        g.m += g.g[e];
      }
    }
    int64_t st = 1;
    for (int e = g.dim - 1; e >= 0; --e) {
      g.stride[e] = g.additive ? 1 : st;
      st *= g.g[e];
    }
    g.sf = hd.sf;
    g.noise = hd.noise;
    for (int e = 0; e < g.dim; ++e)
      for (int q = 0; q < 4; ++q) {
        double r = q * g.h[e], ls = g.ls[e];
        double v = std::exp(-(r * r) / (2 * ls * ls));
        g.cloc[e][q] = v;
        g.cloc_dl[e][q] = v * r * r / (ls * ls * ls);
      }
    c->dtype = (love_dtype)hd.dtype;
    c->cache_dtype = (love_dtype)hd.cache_dtype;
    c->flags = hd.flags;
    c->k_eff = hd.k_eff;
    c->ld = hd.ld;
    c->ks = hd.ks;
    c->ld_s = hd.ld_s;
    c->ld_g = hd.ld_g;
    c->cg_iters = hd.cg_iters;
    c->sampler_fallback = hd.sampler_fallback;
    c->alloc = make_alloc(allocator);
    c->alpha = new double[c->k_eff + 1]();
    c->beta = new double[c->k_eff + 1]();
    love_status rc = LOVE_OK;
    if (fread(c->alpha, sizeof(double), c->k_eff, f) != (size_t)c->k_eff) rc = LOVE_ERR_ARG;
    if (rc == LOVE_OK && fread(c->beta, sizeof(double), c->k_eff, f) != (size_t)c->k_eff) rc = LOVE_ERR_ARG;
    if (rc == LOVE_OK) rc = read_dev(f, &c->Rc, hd.bytes_rc, c->alloc, s);
    if (rc == LOVE_OK) rc = read_dev(f, &c->S, hd.bytes_s, c->alloc, s);
    if (rc == LOVE_OK) rc = read_dev(f, &c->P, hd.bytes_p, c->alloc, s);
    if (rc == LOVE_OK) rc = read_dev(f, &c->KdP, hd.bytes_kdp, c->alloc, s);
    if (rc == LOVE_OK) rc = read_dev(f, &c->B, hd.bytes_b, c->alloc, s);
    if (rc == LOVE_OK) rc = read_dev(f, &c->Minv, hd.bytes_minv, c->alloc, s);
    std::fclose(f);
    f = nullptr;
    if (rc == LOVE_OK) {
      c->status = (DevStatus*)c->alloc.alloc(sizeof(DevStatus), s);
      if (!c->status) rc = LOVE_ERR_OOM;
      else rc = cuda_check(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), s));
    }
    if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc != LOVE_OK) {
      love_cache_destroy(c);
      return rc;
    }
    *out = c;
    return LOVE_OK;
  } catch (...) {
    if (f) std::fclose(f);
    love_cache_destroy(c);
    return LOVE_ERR_OOM;
  }
}
LOVE_ENTRY_CATCH

}  // extern "C"
