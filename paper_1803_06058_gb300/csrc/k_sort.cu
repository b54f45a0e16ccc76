// k_sort.cu -- training-point ordering for deterministic SKI scatters.
//
// Not in the paper (an implementation choice): each training point is keyed by
// the linear index of its interpolation cell (the base node of its cubic
// stencil in every dimension, Sec. 2.3), the points are stably sorted by that
// key with an LSD radix sort, and cell_start[c] gives the first sorted point
// of cell c.  W v (n -> m) then becomes a per-node gather over contiguous
// point ranges, with a fixed summation order and no floating-point atomics.
#include "love_internal.cuh"

namespace love {
namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // 2048 keys per block
constexpr int RADIX = 256;

template <typename T>
__global__ void k_cell_keys(const T* __restrict__ x, int64_t n, GridDev g, uint32_t* __restrict__ keys,
                            int32_t* __restrict__ vals, DevStatus* st) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t key = 0;
  bool ok = true;
  for (int e = 0; e < g.dim; ++e) {
    T s = grid_coord(x[i * g.dim + e], g, e);
    int b;
    T w[4];
    ok &= keys_weights(s, g.g[e], b, w);
    // additive composition: the primary order is by the cell of dimension 0
    if (!g.additive) key += (uint32_t)b * (uint32_t)g.stride[e];
    else if (e == 0) key = (uint32_t)b;
  }
  if (!ok) {
    key = 0;
    atomicAdd(&st->domain_errors, 1ull);
    dev_flag(st, LOVE_ERR_DOMAIN);
  }
  keys[i] = key;
  vals[i] = (int32_t)i;
}

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                             uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t h[RADIX];
  for (int d = threadIdx.x; d < RADIX; d += blockDim.x) h[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * SORT_TILE;
  for (int it = 0; it < SORT_ITEMS; ++it) {
    int64_t i = base + it * SORT_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// exclusive scan of `len` counters by one block (len = RADIX * nblocks)
__global__ void k_exclusive_scan(uint32_t* __restrict__ a, int64_t len) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < len; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < len ? a[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int nw = blockDim.x >> 5;
      uint32_t ws = lane < nw ? warp_sums[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      if (lane < nw) warp_sums[lane] = ws;
    }
    __syncthreads();
    uint32_t excl = carry + x - v + (warp > 0 ? warp_sums[warp - 1] : 0u);
    if (i < len) a[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                                uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n,
                                int shift, const uint32_t* __restrict__ offs, int nblocks) {
  constexpr int NW = SORT_THREADS / 32;
  __shared__ uint32_t cnt[NW][RADIX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < RADIX; d += 32) cnt[warp][d] = 0;
  __syncwarp();
  int64_t base = (int64_t)blockIdx.x * SORT_TILE + (int64_t)warp * (SORT_ITEMS * 32);
  uint32_t key[SORT_ITEMS], rank[SORT_ITEMS];
  int32_t val[SORT_ITEMS];
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < SORT_ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    bool valid = i < n;
    key[r] = valid ? keys_in[i] : 0xffffffffu;
    val[r] = valid ? vals_in[i] : 0;
    uint32_t d = (key[r] >> shift) & (RADIX - 1);
    unsigned act = __ballot_sync(0xffffffffu, valid);
    unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu) & act;
    uint32_t before = valid ? cnt[warp][d] : 0u;
    rank[r] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, per digit
  for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < NW; ++w) {
      uint32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < SORT_ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i >= n) continue;
    uint32_t d = (key[r] >> shift) & (RADIX - 1);
    uint32_t pos = offs[(int64_t)d * nblocks + blockIdx.x] + cnt[warp][d] + rank[r];
    keys_out[pos] = key[r];
    vals_out[pos] = val[r];
  }
}

// cell_start[c] = first sorted position with key >= c, for c in [0, m]
__global__ void k_cell_start(const uint32_t* __restrict__ keys, int64_t n, int64_t m,
                             int32_t* __restrict__ cell_start) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p > n) return;
  int64_t prev = p > 0 ? (int64_t)keys[p - 1] : -1;
  int64_t cur = p < n ? (int64_t)keys[p] : m;
  for (int64_t c = prev + 1; c <= cur; ++c) cell_start[c] = (int32_t)p;
}

template <typename T>
__global__ void k_permute(const T* __restrict__ x, const T* __restrict__ y, const int32_t* __restrict__ vals,
                          int64_t n, int64_t n_pad, int dim, GridDev g, T* __restrict__ xs, T* __restrict__ ys,
                          int32_t* __restrict__ perm) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pad) return;
  if (p < n) {
    int32_t src = vals[p];
    for (int e = 0; e < dim; ++e) xs[p * dim + e] = x[(int64_t)src * dim + e];
    if (ys) ys[p] = y[src];
    perm[p] = src;
  } else {
    // padding rows: an interior coordinate; their Lanczos entries stay zero
    for (int e = 0; e < dim; ++e) xs[p * dim + e] = (T)(g.lo_d[e] + 2.0 * g.h_d[e]);
    if (ys) ys[p] = T(0);
  }
}

template <typename T>
love_status sort_impl(love_ski* ski, const void* x_in, const void* y_in, cudaStream_t s) {
  const int64_t n = ski->n, m = ski->grid.additive ? ski->grid.g[0] : ski->grid.m;   // cells keyed
  const GridDev gd = ski->grid.dev();
  const Allocator& al = ski->alloc;
  size_t kb = (size_t)n * 4;
  uint32_t* k0 = (uint32_t*)al.alloc(kb, s);
  uint32_t* k1 = (uint32_t*)al.alloc(kb, s);
  int32_t* v0 = (int32_t*)al.alloc(kb, s);
  int32_t* v1 = (int32_t*)al.alloc(kb, s);
  int nblocks = ceil_div(n, SORT_TILE);
  size_t hb = (size_t)RADIX * nblocks * 4;
  uint32_t* hist = (uint32_t*)al.alloc(hb, s);
  love_status rc = LOVE_OK;
  if (!k0 || !k1 || !v0 || !v1 || !hist) rc = LOVE_ERR_OOM;
  if (rc == LOVE_OK) {
    LOVE_COUNT_LAUNCH(); k_cell_keys<T><<<ceil_div(n, 256), 256, 0, s>>>((const T*)x_in, n, gd, k0, v0, ski->status);
    int nbits = 1;
    while ((int64_t(1) << nbits) < m) ++nbits;
    for (int shift = 0; shift < nbits; shift += 8) {
      LOVE_COUNT_LAUNCH(); k_radix_hist<<<nblocks, SORT_THREADS, 0, s>>>(k0, n, shift, hist, nblocks);
      LOVE_COUNT_LAUNCH(); k_exclusive_scan<<<1, 1024, 0, s>>>(hist, (int64_t)RADIX * nblocks);
      LOVE_COUNT_LAUNCH(); k_radix_scatter<<<nblocks, SORT_THREADS, 0, s>>>(k0, v0, k1, v1, n, shift, hist, nblocks);
      std::swap(k0, k1);
      std::swap(v0, v1);
    }
    LOVE_COUNT_LAUNCH(); k_cell_start<<<ceil_div(n + 1, 256), 256, 0, s>>>(k0, n, m, ski->cell_start);
    LOVE_COUNT_LAUNCH(); k_permute<T><<<ceil_div(ski->n_pad, 256), 256, 0, s>>>((const T*)x_in, (const T*)y_in, v0, n, ski->n_pad,
                                                          gd.dim, gd, (T*)ski->xs, (T*)ski->ys, ski->perm);
    rc = cuda_check(cudaGetLastError());
  }
  al.free(k0, kb, s);
  al.free(k1, kb, s);
  al.free(v0, kb, s);
  al.free(v1, kb, s);
  al.free(hist, hb, s);
  return rc;
}

// key of a primary-ordered point: its cell in dimension e
template <typename T>
__global__ void k_cell_keys_dim(const T* __restrict__ xs, int64_t n, GridDev g, int e, uint32_t* __restrict__ keys,
                                int32_t* __restrict__ vals) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b;
  T w[4];
  keys_weights(grid_coord(xs[i * g.dim + e], g, e), g.g[e], b, w);  // in range: checked by the primary sort
  keys[i] = (uint32_t)b;
  vals[i] = (int32_t)i;
}
// 1-D coordinates of dimension e in the order `map` (identity if null); padding rows interior
template <typename T>
__global__ void k_gather_dim(const T* __restrict__ xs, const int32_t* __restrict__ map, int64_t n, int64_t n_pad,
                             GridDev g, int e, T* __restrict__ out) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pad) return;
  out[p] = p < n ? xs[(int64_t)(map ? map[p] : p) * g.dim + e] : (T)(g.lo_d[e] + 2.0 * g.h_d[e]);
}

template <typename T>
love_status sort_dims_impl(love_ski* ski, cudaStream_t s) {
  const int64_t n = ski->n, np = ski->n_pad;
  const GridDev gd = ski->grid.dev();
  const Allocator& al = ski->alloc;
  const T* xs = (const T*)ski->xs;
  for (int e = 0; e < gd.dim; ++e) {
    ski->xs1[e] = al.alloc(sizeof(T) * (size_t)np, s);
    if (!ski->xs1[e]) return LOVE_ERR_OOM;
  }
  ski->cs1[0] = ski->cell_start;
  LOVE_COUNT_LAUNCH(); k_gather_dim<T><<<ceil_div(np, 256), 256, 0, s>>>(xs, nullptr, n, np, gd, 0, (T*)ski->xs1[0]);
  size_t kb = (size_t)n * 4;
  int nblocks = ceil_div(n, SORT_TILE);
  size_t hb = (size_t)RADIX * nblocks * 4;
  uint32_t* k0 = (uint32_t*)al.alloc(kb, s);
  uint32_t* k1 = (uint32_t*)al.alloc(kb, s);
  int32_t* v0 = (int32_t*)al.alloc(kb, s);
  int32_t* v1 = (int32_t*)al.alloc(kb, s);
  uint32_t* hist = (uint32_t*)al.alloc(hb, s);
  love_status rc = (k0 && k1 && v0 && v1 && hist) ? LOVE_OK : LOVE_ERR_OOM;
  for (int e = 1; e < gd.dim && rc == LOVE_OK; ++e) {
    const int64_t cells = gd.g[e];
    ski->cs1[e] = (int32_t*)al.alloc(sizeof(int32_t) * (size_t)(cells + 1), s);
    ski->map1[e] = (int32_t*)al.alloc(kb, s);
    if (!ski->cs1[e] || !ski->map1[e]) {
      rc = LOVE_ERR_OOM;
      break;
    }
    LOVE_COUNT_LAUNCH(); k_cell_keys_dim<T><<<ceil_div(n, 256), 256, 0, s>>>(xs, n, gd, e, k0, v0);
    int nbits = 1;
    while ((int64_t(1) << nbits) < cells) ++nbits;
    uint32_t *ka = k0, *kb2 = k1;
    int32_t *va = v0, *vb = v1;
    for (int shift = 0; shift < nbits; shift += 8) {
      LOVE_COUNT_LAUNCH(); k_radix_hist<<<nblocks, SORT_THREADS, 0, s>>>(ka, n, shift, hist, nblocks);
      LOVE_COUNT_LAUNCH(); k_exclusive_scan<<<1, 1024, 0, s>>>(hist, (int64_t)RADIX * nblocks);
      LOVE_COUNT_LAUNCH(); k_radix_scatter<<<nblocks, SORT_THREADS, 0, s>>>(ka, va, kb2, vb, n, shift, hist, nblocks);
      std::swap(ka, kb2);
      std::swap(va, vb);
    }
    LOVE_COUNT_LAUNCH(); k_cell_start<<<ceil_div(n + 1, 256), 256, 0, s>>>(ka, n, cells, ski->cs1[e]);
    rc = cuda_check(cudaMemcpyAsync(ski->map1[e], va, kb, cudaMemcpyDeviceToDevice, s));
    if (rc != LOVE_OK) break;
    LOVE_COUNT_LAUNCH(); k_gather_dim<T><<<ceil_div(np, 256), 256, 0, s>>>(xs, ski->map1[e], n, np, gd, e, (T*)ski->xs1[e]);
    rc = cuda_check(cudaGetLastError());
  }
  al.free(k0, kb, s);
  al.free(k1, kb, s);
  al.free(v0, kb, s);
  al.free(v1, kb, s);
  al.free(hist, hb, s);
  return rc;
}

}  // namespace

love_status sort_additive_dims(love_ski* ski, cudaStream_t s) {
  if (ski->dtype == LOVE_F64) return sort_dims_impl<double>(ski, s);
  return sort_dims_impl<float>(ski, s);
}

love_status sort_training_points(love_ski* ski, const void* x_in, const void* y_in, cudaStream_t s) {
  if (ski->dtype == LOVE_F64) return sort_impl<double>(ski, x_in, y_in, s);
  return sort_impl<float>(ski, x_in, y_in, s);
}

}  // namespace love
