// k_predict.cu -- the LOVE test phase: O(k) predictive mean and variance.
//
// Algorithm 1 (lines u = sparse_mm(R, w_i), v = sparse_mm(R', w_j), return
// k(x_i, x_j) - u^T v) with i = j and the symmetric cache Rt (Rt Rt^T = R^T R'):
//   v = Rt^T w*          (4^d cache rows, weights from cubic interpolation)
//   var = p(x*) - |v|^2  (p = w*^T K_UU w*, or s_f with the exact prior)
//   mean = w*^T a        (eq. pred_mean_ski; a is column k of the cache)
//
// Layout: the cache is m rows of ld elements, row r = [Rt[r, 0..k) | a[r] | 0 pad],
// rows padded to 16 bytes.  A group of G lanes serves one test point: lane l
// owns the 16-byte column vectors l, l + G, ... and, for each, reads that
// vector from the 4^d stencil rows (coalesced 16-byte loads across the group).
// In 1-D the 4 rows are one contiguous span.
//
// Precision (FP32 path): v in FP32, |v|^2 per lane in FP32, then the group
// sum of (prior terms - squares) in double-float, so the cancellation
// p - |v|^2 (var/p ~ 1e-7 on the 1-D, n = 1e6 workload) is taken without
// losing the variance's leading digits.  The 16 prior products of the 1-D
// stencil are spread over the group's lanes and folded into the same sum.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "love_internal.cuh"

namespace love {
namespace {

struct PredArgs {
  GridDev g;
  int64_t t;
  const void* x;
  void* mean;
  void* var;
  const void* Rc;
  int ld;          // elements per cache row
  int k;           // variance columns
  int has_mean;
  int exact_prior;
  int root;        // variance from the posterior root: +|S^T w|^2, no prior term
  double sf;
  df cl[LOVE_MAX_DIM][4];      // Toeplitz entries T_e[0..3] (s_f folded into e = 0), double-float
  double cld[LOVE_MAX_DIM][4];
  DevStatus* status;
};

template <typename CT> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecOf<__nv_bfloat16> { using type = uint4; static constexpr int n = 8; };
template <> struct VecOf<double> { using type = double2; static constexpr int n = 2; };

template <typename R>
__device__ __forceinline__ void vec_fma(R* acc, float4 v, R w) {
  acc[0] = fma(w, (R)v.x, acc[0]);
  acc[1] = fma(w, (R)v.y, acc[1]);
  acc[2] = fma(w, (R)v.z, acc[2]);
  acc[3] = fma(w, (R)v.w, acc[3]);
}
template <typename R>
__device__ __forceinline__ void vec_fma(R* acc, double2 v, R w) {
  acc[0] = fma(w, (R)v.x, acc[0]);
  acc[1] = fma(w, (R)v.y, acc[1]);
}
template <typename R>
__device__ __forceinline__ void vec_fma(R* acc, uint4 v, R w) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 f = __bfloat1622float2(h[q]);
    acc[2 * q] = fma(w, (R)f.x, acc[2 * q]);
    acc[2 * q + 1] = fma(w, (R)f.y, acc[2 * q + 1]);
  }
}

template <typename V>
__device__ __forceinline__ V ldg_vec(const V* p) { return __ldg(p); }

// w^T T^loc w for one dimension in double-float:
// c0 sum w_r^2 + 2 c1 (w0w1 + w1w2 + w2w3) + 2 c2 (w0w2 + w1w3) + 2 c3 w0w3
__device__ __forceinline__ df local_quad_df(const float* w, const df* c) {
  df s0 = two_prod(w[0], w[0]);
  s0 = df_add(s0, two_prod(w[1], w[1]));
  s0 = df_add(s0, two_prod(w[2], w[2]));
  s0 = df_add(s0, two_prod(w[3], w[3]));
  df s1 = df_add(df_add(two_prod(w[0], w[1]), two_prod(w[1], w[2])), two_prod(w[2], w[3]));
  df s2 = df_add(two_prod(w[0], w[2]), two_prod(w[1], w[3]));
  df s3 = two_prod(w[0], w[3]);
  df r = df_mul(c[0], s0);
  df two = {2.f, 0.f};
  r = df_add(r, df_mul(df_mul(two, c[1]), s1));
  r = df_add(r, df_mul(df_mul(two, c[2]), s2));
  r = df_add(r, df_mul(df_mul(two, c[3]), s3));
  return r;
}
__device__ __forceinline__ double local_quad_d(const double* w, const double* c) {
  double r = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) r += w[a] * w[b] * c[a > b ? a - b : b - a];
  return r;
}

// acc[0..VC) = sum over the 4^D stencil rows r of w_r * (column group cg of row r);
// with RS > 1 (3-D only) just the rows of first-dimension offsets
// part (4 / RS) .. (part + 1)(4 / RS) - 1
template <typename CT, typename R, int D, int RS = 1>
__device__ __forceinline__ void gather_rows(const PredArgs& a, const typename VecOf<CT>::type* __restrict__ base_ptr,
                                            int NG, const int (&base)[D], const R (&w)[D][4], bool ok, int cg,
                                            R (&acc)[VecOf<CT>::n], int part = 0) {
  using V = typename VecOf<CT>::type;
  constexpr int VC = VecOf<CT>::n;
#pragma unroll
  for (int c = 0; c < VC; ++c) acc[c] = R(0);
  if (!ok) return;
  if (D > 1 && a.g.additive) {
    // stacked interpolation vector: 4 rows per 1-D block
#pragma unroll
    for (int e = 0; e < D; ++e) {
      const V* p = base_ptr + (int64_t)(a.g.off[e] + base[e] - 1) * NG + cg;
#pragma unroll
      for (int r = 0; r < 4; ++r) vec_fma(acc, ldg_vec(p + r * NG), w[e][r]);
    }
    return;
  }
  if (D == 1) {
    // small outer Keys weights first, so the two large terms are added last
    const V* p = base_ptr + (int64_t)(base[0] - 1) * NG + cg;
    const V r0 = ldg_vec(p), r1 = ldg_vec(p + NG), r2 = ldg_vec(p + 2 * NG), r3 = ldg_vec(p + 3 * NG);
    vec_fma(acc, r3, w[0][3]);
    vec_fma(acc, r0, w[0][0]);
    vec_fma(acc, r2, w[0][2]);
    vec_fma(acc, r1, w[0][1]);
  } else if (D == 2) {
#pragma unroll
    for (int r0 = 0; r0 < 4; ++r0) {
      const int64_t row0 = (int64_t)(base[0] - 1 + r0) * a.g.stride[0] + (base[D - 1] - 1);
#pragma unroll
      for (int r1 = 0; r1 < 4; ++r1)
        vec_fma(acc, ldg_vec(base_ptr + (row0 + r1) * NG + cg), w[0][r0] * w[D - 1][r1]);
    }
  } else {
#pragma unroll
    for (int rr = 0; rr < 4 / RS; ++rr)
#pragma unroll
      for (int r1 = 0; r1 < 4; ++r1) {
        // (selects between static indices: w stays in registers)
        const int r0 = RS == 2 ? 2 * part + rr : rr;
        const R w0 = RS == 2 ? (part ? w[0][(rr + 2) & 3] : w[0][rr]) : w[0][rr];
        const int64_t row0 = (int64_t)(base[0] - 1 + r0) * a.g.stride[0] +
                             (int64_t)(base[1] - 1 + r1) * a.g.stride[1] + (base[D - 1] - 1);
        const R w01 = w0 * w[1][r1];
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2)
          vec_fma(acc, ldg_vec(base_ptr + (row0 + r2) * NG + cg), w01 * w[D - 1][r2]);
      }
  }
}

// G lanes per point.  R = arithmetic type (float for F32/BF16 caches, double for F64).
// Serves points [.., a.t): the calling warp's first point is warp_first + lane / G
// and every group advances by gstride, so all groups of a warp iterate the same
// number of times (uniform shuffles).
// RS > 1 (3-D): the group's lanes form RS sets of G / RS lanes, set p gathering
// the stencil rows of first-dimension offsets in its share (gather_rows); the
// sets' partial sums are added by shuffles before the squares.  For a BF16
// cache, whose rows hold half as many 16-byte vectors as FP32 ones, this keeps
// every lane of the group loading.
template <typename CT, typename R, int D, int G, int RS = 1>
__device__ __forceinline__ void predict_groups(const PredArgs& a, int64_t warp_first, int64_t gstride) {
  using V = typename VecOf<CT>::type;
  constexpr int VC = VecOf<CT>::n;
  constexpr int NROW = D == 1 ? 4 : (D == 2 ? 16 : 64);
  const int lane = threadIdx.x & 31;
  const int li = lane & (G - 1);
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int NG = a.ld / VC;
  const V* __restrict__ base_ptr = reinterpret_cast<const V*>(a.Rc);
  const R* __restrict__ xs = reinterpret_cast<const R*>(a.x);
  // the coordinates of the group's next point are loaded one iteration ahead
  // (they may live in host memory, read over the CPU-GPU link)
  R xnext[D];
  {
    const int64_t pt = warp_first + lane / G;
#pragma unroll
    for (int e = 0; e < D; ++e) xnext[e] = pt < a.t ? xs[pt * D + e] : R(0);
  }
  for (int64_t pt0 = warp_first; pt0 < a.t; pt0 += gstride) {
    const int64_t pt = pt0 + lane / G;
    const bool live = pt < a.t;
    R xcur[D];
#pragma unroll
    for (int e = 0; e < D; ++e) xcur[e] = xnext[e];
    {
      const int64_t pn = pt + gstride;
#pragma unroll
      for (int e = 0; e < D; ++e) xnext[e] = pn < a.t ? xs[pn * D + e] : R(0);
    }
    R w[D][4];
    int base[D];
    bool ok = live;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      R s = grid_coord(live ? xcur[e] : R(0), a.g, e);
      ok &= keys_weights(s, a.g.g[e], base[e], w[e]);
    }
    // row index of stencil row q (0 <= q < 4^D), weight
    R sq = R(0);     // sum of squares of this lane's columns
    R mu = R(0);
    bool has_mu = false;
    constexpr int CGW = G / RS;   // lanes per row set
    const int part = li / CGW;
    const int iters = (NG + CGW - 1) / CGW;
    for (int it = 0; it < iters; ++it) {
      const int cg = li % CGW + it * CGW;
      const bool act = cg < NG;
      R acc[VC];
      gather_rows<CT, R, D, RS>(a, base_ptr, NG, base, w, ok && act, cg, acc, part);
      if (RS > 1) {
#pragma unroll
        for (int o = CGW; o < G; o <<= 1)
#pragma unroll
          for (int c = 0; c < VC; ++c) acc[c] += __shfl_xor_sync(gmask, acc[c], o, G);
        if (part != 0) continue;
      }
      if (!act) continue;
      if ((cg + 1) * VC <= a.k) {
        // a group of variance columns only (all but the last one or two)
#pragma unroll
        for (int c = 0; c < VC; ++c) sq = fma(acc[c], acc[c], sq);
      } else {
#pragma unroll
        for (int c = 0; c < VC; ++c) {
          const int col = cg * VC + c;
          if (col < a.k) sq = fma(acc[c], acc[c], sq);
          else if (col == a.k) { mu = acc[c]; has_mu = true; }
        }
      }
    }
    (void)NROW;
    // group sum of (prior terms - squares)
    if constexpr (std::is_same<R, float>::value) {
      df tot = {a.root ? sq : -sq, 0.f};
      if (ok && !a.root) {
        if (a.exact_prior) {
          if (li == 0) tot = df_add(tot, df_from_double(a.sf));
        } else if (D == 1) {
          // 16 products w_r w_s T[|r-s|] spread over the G lanes
          for (int pi = li; pi < 16; pi += G) {
            int r = pi >> 2, s2 = pi & 3;
            int dd = r > s2 ? r - s2 : s2 - r;
            tot = df_add(tot, df_mul(two_prod(w[0][r], w[0][s2]), a.cl[0][dd]));
          }
        } else if (li == 0) {
          df p = local_quad_df(w[0], a.cl[0]);
#pragma unroll
          for (int e = 1; e < D; ++e) {
            const df q = local_quad_df(w[e], a.cl[e]);
            p = a.g.additive ? df_add(p, q) : df_mul(p, q);   // sum of blocks / Kronecker product
          }
          tot = df_add(tot, p);
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        df other;
        other.hi = __shfl_xor_sync(gmask, tot.hi, o, G);
        other.lo = __shfl_xor_sync(gmask, tot.lo, o, G);
        tot = df_add(tot, other);
      }
      if (live && li == 0) {
        float* var = reinterpret_cast<float*>(a.var);
        float v = tot.hi + tot.lo;
        if (!ok) {
          v = __int_as_float(0x7fc00000);
          atomicAdd(&a.status->domain_errors, 1ull);
          dev_flag(a.status, LOVE_ERR_DOMAIN);
        } else if (v < 0.f) {
          v = 0.f;
          atomicAdd(&a.status->clamped, 1ull);
        }
        var[pt] = v;
        if (a.has_mean && !ok) reinterpret_cast<float*>(a.mean)[pt] = __int_as_float(0x7fc00000);
      }
      if (live && ok && has_mu && a.has_mean) reinterpret_cast<float*>(a.mean)[pt] = (float)mu;
    } else {
      double tot = a.root ? (double)sq : -(double)sq;
      if (ok && li == 0 && !a.root) {
        if (a.exact_prior) {
          tot += a.sf;
        } else {
          double p = a.g.additive ? 0.0 : 1.0;
#pragma unroll
          for (int e = 0; e < D; ++e) {
            double wd[4] = {(double)w[e][0], (double)w[e][1], (double)w[e][2], (double)w[e][3]};
            const double q = local_quad_d(wd, a.cld[e]);
            p = a.g.additive ? p + q : p * q;
          }
          tot += p;
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) tot += __shfl_xor_sync(gmask, tot, o, G);
      if (live && li == 0) {
        double* var = reinterpret_cast<double*>(a.var);
        double v = tot;
        if (!ok) {
          v = __longlong_as_double(0x7ff8000000000000ll);
          atomicAdd(&a.status->domain_errors, 1ull);
          dev_flag(a.status, LOVE_ERR_DOMAIN);
        } else if (v < 0.0) {
          v = 0.0;
          atomicAdd(&a.status->clamped, 1ull);
        }
        var[pt] = v;
        if (a.has_mean && !ok) reinterpret_cast<double*>(a.mean)[pt] = __longlong_as_double(0x7ff8000000000000ll);
      }
      if (live && ok && has_mu && a.has_mean) reinterpret_cast<double*>(a.mean)[pt] = (double)mu;
    }
  }
}

// rows split between lane sets: 3-D BF16 caches with a full warp per point
template <typename CT, int D, int G> struct RowSplit {
  static constexpr int v = (D == 3 && G == 32 && std::is_same<CT, __nv_bfloat16>::value) ? 2 : 1;
};

template <typename CT, typename R, int D, int G>
__global__ void __launch_bounds__(256, D == 3 ? 2 : 4) k_predict(PredArgs a) {
  const int64_t groups_per_block = blockDim.x / G;
  const int64_t gid0 = (int64_t)blockIdx.x * groups_per_block + threadIdx.x / G;
  predict_groups<CT, R, D, G, RowSplit<CT, D, G>::v>(a, gid0 - ((threadIdx.x & 31) / G),
                                                     (int64_t)gridDim.x * groups_per_block);
}

// Batched form: a persistent grid walks a list of row chunks, each inside one
// GP; the CTA copies that GP's descriptor to shared memory, points it at the
// GP's rows of the concatenated x / mean / var, and serves the chunk.
template <typename CT, typename R, int D, int G>
__global__ void __launch_bounds__(256, D == 3 ? 2 : 4) k_predict_batched(const PredArgs* __restrict__ descs,
                                                         const int64_t* __restrict__ t_off,
                                                         const PredChunk* __restrict__ chunks, int nchunks,
                                                         const void* x, void* mean, void* var) {
  __shared__ PredArgs sa;
  __shared__ int64_t begin;
  const int64_t groups_per_block = blockDim.x / G;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const PredChunk ch = chunks[c];
      sa = descs[ch.gp];
      const int64_t off = t_off[ch.gp];
      sa.x = reinterpret_cast<const R*>(x) + off * D;
      sa.var = reinterpret_cast<R*>(var) + off;
      sa.mean = mean ? reinterpret_cast<R*>(mean) + off : nullptr;
      sa.has_mean = mean != nullptr;
      sa.t = ch.end;
      begin = ch.begin;
    }
    __syncthreads();
    predict_groups<CT, R, D, G, RowSplit<CT, D, G>::v>(sa, begin + (threadIdx.x / 32) * (32 / G), groups_per_block);
  }
}

template <typename CT, typename R, int D, int G>
love_status launch_predict(const PredArgs& a, cudaStream_t s) {
  const int threads = 256;
  const int64_t groups = (a.t + 0);
  int64_t blocks = (groups + (threads / G) - 1) / (threads / G);
  int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  LOVE_COUNT_LAUNCH(); k_predict<CT, R, D, G><<<(unsigned)blocks, threads, 0, s>>>(a);
  return cuda_check(cudaGetLastError());
}

// lanes per point: 4 in 1-D (timed fastest of 4 / 8 / 16 on the 1-D n = 1e6
// workload by the batch autotuner), 16 in 2-D, 32 in 3-D
template <typename CT, typename R>
love_status predict_dim(const PredArgs& a, cudaStream_t s) {
  switch (a.g.dim) {
    case 1: return launch_predict<CT, R, 1, 4>(a, s);
    case 2: return launch_predict<CT, R, 2, 16>(a, s);
    default: return launch_predict<CT, R, 3, 32>(a, s);
  }
}

}  // namespace

namespace {
PredArgs make_pred_args(const love_cache* c) {
  PredArgs a{};
  a.g = c->grid.dev();
  a.Rc = c->Rc;
  a.ld = c->ld;
  a.k = c->k_eff;
  a.exact_prior = (c->flags & LOVE_PRIOR_EXACT) ? 1 : 0;
  // exact prior k(x, x): s_f, or d s_f for an additive composition of d kernels
  a.sf = c->grid.sf * (c->grid.additive ? c->grid.dim : 1);
  for (int e = 0; e < LOVE_MAX_DIM; ++e)
    for (int q = 0; q < 4; ++q) {
      // outputscale folded into dimension 0: p = prod_e w_e^T T_e w_e (into every
      // block of an additive grid: p = sum_e s_f w_e^T T_e w_e)
      double v = c->grid.cloc[e][q] * ((e == 0 || c->grid.additive) ? c->grid.sf : 1.0);
      float hi = (float)v;
      a.cl[e][q] = {hi, (float)(v - (double)hi)};
      a.cld[e][q] = v;
    }
  a.status = c->status;
  return a;
}

template <typename CT, typename R, int D, int G>
love_status launch_batched(const void* descs, const int64_t* toff, const PredChunk* chunks, int nchunks,
                           int ctas_per_sm, const void* x, void* mean, void* var, cudaStream_t s) {
  const int blocks = std::max(1, std::min(nchunks, ctas_per_sm * num_sms()));
  LOVE_COUNT_LAUNCH();
  k_predict_batched<CT, R, D, G><<<blocks, 256, 0, s>>>((const PredArgs*)descs, toff, chunks, nchunks, x, mean, var);
  return cuda_check(cudaGetLastError());
}
template <typename CT, typename R>
love_status batched_dim(int dim, int lanes, const void* descs, const int64_t* toff, const PredChunk* chunks,
                        int nchunks, int ctas, const void* x, void* mean, void* var, cudaStream_t s) {
#define LOVE_PB(D, G) \
  if (dim == D && lanes == G) return launch_batched<CT, R, D, G>(descs, toff, chunks, nchunks, ctas, x, mean, var, s);
  LOVE_PB(1, 4) LOVE_PB(1, 8) LOVE_PB(1, 16)
  LOVE_PB(2, 8) LOVE_PB(2, 16) LOVE_PB(2, 32)
  LOVE_PB(3, 8) LOVE_PB(3, 16) LOVE_PB(3, 32)
#undef LOVE_PB
  return LOVE_ERR_ARG;
}
}  // namespace

love_status predict_launch(love_cache* c, int64_t t, const void* x, void* mean, void* var, cudaStream_t s) {
  if (t == 0) return LOVE_OK;
  PredArgs a = make_pred_args(c);
  a.t = t;
  a.x = x;
  a.mean = mean;
  a.var = var;
  a.has_mean = mean != nullptr;
  if (c->dtype == LOVE_F64) return predict_dim<double, double>(a, s);
  if (c->cache_dtype == LOVE_BF16) return predict_dim<__nv_bfloat16, float>(a, s);
  return predict_dim<float, float>(a, s);
}

// var = |S^T w*|^2 from the sampler root S (m x ld_s rows in the data dtype)
love_status predict_root_launch(love_cache* c, int64_t t, const void* x, void* var, cudaStream_t s) {
  if (t == 0) return LOVE_OK;
  PredArgs a = make_pred_args(c);
  a.Rc = c->S;
  a.ld = c->ld_s;
  a.k = c->ks;
  a.has_mean = 0;
  a.root = 1;
  a.t = t;
  a.x = x;
  a.mean = nullptr;
  a.var = var;
  if (c->dtype == LOVE_F64) return predict_dim<double, double>(a, s);
  return predict_dim<float, float>(a, s);
}

size_t predict_desc_bytes() { return sizeof(PredArgs); }
void predict_fill_desc(const love_cache* c, void* dst) {
  PredArgs a = make_pred_args(c);
  std::memcpy(dst, &a, sizeof(PredArgs));
}
int predict_lane_candidates(int dim, int* out) {
  static const int c1[] = {4, 8, 16}, c2[] = {8, 16, 32}, c3[] = {8, 16, 32};
  const int* c = dim == 1 ? c1 : (dim == 2 ? c2 : c3);
  const int n = 3;
  for (int i = 0; i < n; ++i) out[i] = c[i];
  return n;
}
love_status predict_batched_launch(const void* descs, const int64_t* toff, const PredChunk* chunks, int nchunks,
                                   int dim, love_dtype dtype, love_dtype cache_dtype, int lanes, int ctas_per_sm,
                                   const void* x, void* mean, void* var, cudaStream_t s) {
  if (nchunks == 0) return LOVE_OK;
  if (dtype == LOVE_F64)
    return batched_dim<double, double>(dim, lanes, descs, toff, chunks, nchunks, ctas_per_sm, x, mean, var, s);
  if (cache_dtype == LOVE_BF16)
    return batched_dim<__nv_bfloat16, float>(dim, lanes, descs, toff, chunks, nchunks, ctas_per_sm, x, mean, var, s);
  return batched_dim<float, float>(dim, lanes, descs, toff, chunks, nchunks, ctas_per_sm, x, mean, var, s);
}

}  // namespace love
