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

// G lanes per point.  R = arithmetic type (float for F32/BF16 caches, double for F64).
template <typename CT, typename R, int D, int G>
__global__ void __launch_bounds__(256) k_predict(PredArgs a) {
  using V = typename VecOf<CT>::type;
  constexpr int VC = VecOf<CT>::n;
  constexpr int NROW = D == 1 ? 4 : (D == 2 ? 16 : 64);
  const int lane = threadIdx.x & 31;
  const int li = lane & (G - 1);
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int NG = a.ld / VC;
  const V* __restrict__ base_ptr = reinterpret_cast<const V*>(a.Rc);
  const R* __restrict__ xs = reinterpret_cast<const R*>(a.x);
  const int64_t groups_per_block = blockDim.x / G;
  const int64_t gid0 = (int64_t)blockIdx.x * groups_per_block + threadIdx.x / G;
  const int64_t gstride = (int64_t)gridDim.x * groups_per_block;
  // all groups of a warp iterate the same number of times (uniform shuffles)
  const int64_t warp_first = gid0 - (lane / G);
  for (int64_t pt0 = warp_first; pt0 < a.t; pt0 += gstride) {
    const int64_t pt = pt0 + lane / G;
    const bool live = pt < a.t;
    R w[D][4];
    int base[D];
    bool ok = live;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      R xv = live ? xs[pt * D + e] : R(0);
      R s = grid_coord(xv, a.g, e);
      ok &= keys_weights(s, a.g.g[e], base[e], w[e]);
    }
    // row index of stencil row q (0 <= q < 4^D), weight
    R sq = R(0);     // sum of squares of this lane's columns
    R mu = R(0);
    bool has_mu = false;
    for (int cg = li; cg < NG; cg += G) {
      R acc[VC];
#pragma unroll
      for (int c = 0; c < VC; ++c) acc[c] = R(0);
      if (ok) {
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
            const int64_t row0 = (int64_t)(base[0] - 1 + r0) * a.g.stride[0] + (base[1] - 1);
#pragma unroll
            for (int r1 = 0; r1 < 4; ++r1)
              vec_fma(acc, ldg_vec(base_ptr + (row0 + r1) * NG + cg), w[0][r0] * w[1][r1]);
          }
        } else {
#pragma unroll
          for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
            for (int r1 = 0; r1 < 4; ++r1) {
              const int64_t row0 = (int64_t)(base[0] - 1 + r0) * a.g.stride[0] +
                                   (int64_t)(base[1] - 1 + r1) * a.g.stride[1] + (base[2] - 1);
              const R w01 = w[0][r0] * w[1][r1];
#pragma unroll
              for (int r2 = 0; r2 < 4; ++r2) vec_fma(acc, ldg_vec(base_ptr + (row0 + r2) * NG + cg), w01 * w[2][r2]);
            }
        }
      }
#pragma unroll
      for (int c = 0; c < VC; ++c) {
        const int col = cg * VC + c;
        if (col < a.k) sq = fma(acc[c], acc[c], sq);
        else if (col == a.k) { mu = acc[c]; has_mu = true; }
      }
    }
    (void)NROW;
    // group sum of (prior terms - squares)
    if constexpr (std::is_same<R, float>::value) {
      df tot = {-sq, 0.f};
      if (ok) {
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
          for (int e = 1; e < D; ++e) p = df_mul(p, local_quad_df(w[e], a.cl[e]));
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
      double tot = -(double)sq;
      if (ok && li == 0) {
        if (a.exact_prior) {
          tot += a.sf;
        } else {
          double p = 1.0;
#pragma unroll
          for (int e = 0; e < D; ++e) {
            double wd[4] = {(double)w[e][0], (double)w[e][1], (double)w[e][2], (double)w[e][3]};
            p *= local_quad_d(wd, a.cld[e]);
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

template <typename CT, typename R>
love_status predict_dim(const PredArgs& a, cudaStream_t s) {
  switch (a.g.dim) {
    case 1: return launch_predict<CT, R, 1, 8>(a, s);
    case 2: return launch_predict<CT, R, 2, 16>(a, s);
    default: return launch_predict<CT, R, 3, 32>(a, s);
  }
}

}  // namespace

love_status predict_launch(love_cache* c, int64_t t, const void* x, void* mean, void* var, cudaStream_t s) {
  if (t == 0) return LOVE_OK;
  PredArgs a{};
  a.g = c->grid.dev();
  a.t = t;
  a.x = x;
  a.mean = mean;
  a.var = var;
  a.Rc = c->Rc;
  a.ld = c->ld;
  a.k = c->k_eff;
  a.has_mean = mean != nullptr;
  a.exact_prior = (c->flags & LOVE_PRIOR_EXACT) ? 1 : 0;
  a.sf = c->grid.sf;
  for (int e = 0; e < LOVE_MAX_DIM; ++e)
    for (int q = 0; q < 4; ++q) {
      // outputscale folded into dimension 0: p = prod_e w_e^T T_e w_e
      double v = c->grid.cloc[e][q] * (e == 0 ? c->grid.sf : 1.0);
      float hi = (float)v;
      a.cl[e][q] = {hi, (float)(v - (double)hi)};
      a.cld[e][q] = v;
    }
  a.status = c->status;
  if (c->dtype == LOVE_F64) return predict_dim<double, double>(a, s);
  if (c->cache_dtype == LOVE_BF16) return predict_dim<__nv_bfloat16, float>(a, s);
  return predict_dim<float, float>(a, s);
}

}  // namespace love
