// k_backward.cu -- vector-Jacobian product of the LOVE variances.
//
// Not in the paper: derived from eq. pred_covar_ski_cache by matrix calculus,
// with every K^^{-1} replaced by the Lanczos approximation M M^T,
// M = Q L^{-T}, Q held fixed.  With v_i = Rt^T w_i and P = W M:
//   d var_i / d x*_e = 2 (dw_i/dx_e)^T K w_i - 2 (Rt^T dw_i/dx_e) . v_i
//   d var_i / d l_e  = (w_i - P v_i)^T K'_e (w_i - P v_i),  K'_e = dK_UU/dl_e
//                    = w_i^T K'_e w_i - 2 w_i^T (K'_e P) v_i + v_i^T (P^T K'_e P) v_i
//   d var_i / d s^2  = |L^{-T} v_i|^2 = v_i^T (L^{-1} L^{-T}) v_i
// (with the exact prior p = s_f the w^T K w and w^T K'_e w terms drop out).
//
// Tables built once per cache (backward_tables): KdP_e = K'_e P (m x k, rows
// padded like the predict cache, FFT with the derivative spectrum in mode e),
// B_e = P^T KdP_e (k x k), Minv = L^{-1} L^{-T} (k x k).  The per-point kernel
// then only gathers the 4^d stencil rows of [Rt | a] and of KdP_e -- no
// scatter, no atomics -- and reduces the hyperparameter terms over points in a
// fixed order.
#include <algorithm>
#include <cmath>

#include "love_internal.cuh"

namespace love {
namespace {

template <typename T> struct AccT;
template <> struct AccT<float> { using type = DotAccF; };
template <> struct AccT<double> { using type = DotAccD; };
__device__ __forceinline__ void merge_into(DotAccF& a, const DotAccF& b) { a.merge(b.s, b.c); }
__device__ __forceinline__ void merge_into(DotAccD& a, const DotAccD& b) { a.s += b.s; }

// row-major copy with padding: dst[r * ld + c] = src[c * m + r]
template <typename T>
__global__ void k_colmajor_to_rows(const T* __restrict__ src, int64_t m, int k, T* __restrict__ dst, int ld) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * ld) return;
  int64_t r = idx / ld;
  int c = (int)(idx - r * ld);
  dst[idx] = c < k ? src[(int64_t)c * m + r] : T(0);
}

// B[a, b] = sum_r P[r, a] Y[r, b]  (P, Y column-major m x k), one block per (a, b)
template <typename T>
__global__ void k_gram(const T* __restrict__ P, const T* __restrict__ Y, int64_t m, int k, T* __restrict__ B) {
  using Acc = typename AccT<T>::type;
  __shared__ Acc red[32];
  const int a = blockIdx.x / k, b = blockIdx.x % k;
  Acc acc;
  acc.zero();
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) acc.add_prod(P[(int64_t)a * m + r], Y[(int64_t)b * m + r]);
  warp_merge(acc);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    Acc t = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) merge_into(t, red[i]);
    B[(int64_t)a * k + b] = (T)t.value();
  }
}

// Minv = L^{-1} L^{-T} with T = L L^T (lower bidiagonal L: diag d, sub e), one
// block: thread 0 factors T (l_11 = sqrt(alpha_1), e_j = beta_j / l_jj,
// l_{j+1,j+1} = sqrt(alpha_{j+1} - e_j^2)); X = L^{-1} by forward substitution
// column by column; Minv = X X^T.  work: 2 (k + 1) + k^2 doubles.
__global__ void k_minv(const double* __restrict__ alpha, const double* __restrict__ beta, int k,
                       double* __restrict__ work, void* out, int dbl, DevStatus* status) {
  double* d = work;
  double* e = work + (k + 1);
  double* X = work + 2 * (k + 1);
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    double piv = alpha[0];
    for (int j = 0; j < k; ++j) {
      if (j > 0) {
        e[j - 1] = beta[j - 1] / d[j - 1];
        piv = alpha[j] - e[j - 1] * e[j - 1];
      }
      if (!(piv > 0.0)) {
        ok = 0;
        dev_flag(status, LOVE_ERR_NOT_PD);
        break;
      }
      d[j] = sqrt(piv);
    }
  }
  __syncthreads();
  if (!ok) return;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    // column c of L^{-1}: x_r = 0 (r < c), x_c = 1/d_c, x_r = -e_{r-1} x_{r-1} / d_r
    double prev = 0.0;
    for (int r = 0; r < k; ++r) {
      double v = 0.0;
      if (r == c) v = 1.0 / d[r];
      else if (r > c) v = -e[r - 1] * prev / d[r];
      X[(int64_t)r * k + c] = v;
      prev = v;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    int a = idx / k, b = idx % k;
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += X[(int64_t)a * k + j] * X[(int64_t)b * k + j];
    if (dbl) ((double*)out)[idx] = acc;
    else ((float*)out)[idx] = (float)acc;
  }
}

struct BwdArgs {
  GridDev g;
  int64_t t;
  const void* x;
  const void* gv;
  void* gx;
  const void* Rc;      // [Rt | a] rows, ld, cache dtype (F32 / BF16 / F64)
  int ld;
  int cdt;
  const void* KdP;     // dim x m x ld_g rows (ski dtype)
  int ld_g;
  const void* B;       // dim x k x k
  const void* Minv;    // k x k
  int k;
  int exact_prior;
  double cl[LOVE_MAX_DIM][4];     // T_e[0..3], s_f folded into e = 0
  double cld[LOVE_MAX_DIM][4];    // dT_e/dl_e [0..3] (s_f folded into e = 0 when e = 0)
  double2* partial;    // [gridDim][LOVE_MAX_DIM + 1]
  double* result;      // LOVE_MAX_DIM + 1
  unsigned* counter;
  DevStatus* status;
};

template <typename T>
__device__ __forceinline__ T ldc(const void* Rc, int64_t idx, int cdt) {
  if (cdt == LOVE_BF16) return (T)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Rc)[idx]);
  if (cdt == LOVE_F64) return (T)reinterpret_cast<const double*>(Rc)[idx];
  return (T)reinterpret_cast<const float*>(Rc)[idx];
}

// (w_l)^T T^loc (w_r) for one dimension, FP64
__device__ __forceinline__ double quad_loc(const double* wl, const double* wr, const double* c) {
  double q = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) q += wl[a] * wr[b] * c[a > b ? a - b : b - a];
  return q;
}

constexpr int BWD_WARPS = 8;
constexpr int BWD_MAXK = 256;
constexpr int NCOL = BWD_MAXK / 32;

// one warp per test point
template <typename T, int D>
__global__ void __launch_bounds__(BWD_WARPS * 32) k_var_backward(BwdArgs a) {
  using Acc = typename AccT<T>::type;
  __shared__ T vsh[BWD_WARPS][BWD_MAXK];
  __shared__ double red[BWD_WARPS][LOVE_MAX_DIM + 1];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const T* x = reinterpret_cast<const T*>(a.x);
  const T* gv = reinterpret_cast<const T*>(a.gv);
  const T* KdP = reinterpret_cast<const T*>(a.KdP);
  const T* Bm = reinterpret_cast<const T*>(a.B);
  const T* Mi = reinterpret_cast<const T*>(a.Minv);
  constexpr int NR = D == 1 ? 4 : (D == 2 ? 16 : 64);
  double hyp[LOVE_MAX_DIM + 1] = {0, 0, 0, 0};   // this lane-0's sums (points handled by the warp)
  const int64_t w0 = (int64_t)blockIdx.x * BWD_WARPS + wp;
  const int64_t nw = (int64_t)gridDim.x * BWD_WARPS;
  for (int64_t pt = w0; pt < a.t; pt += nw) {
    int base[D];
    T w[D][4], dw[D][4];
    bool ok = true;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      T s = grid_coord(x[pt * D + e], a.g, e);
      ok &= keys_weights(s, a.g.g[e], base[e], w[e]);
      keys_dweights(s, base[e], (T)a.g.inv_h_d[e], dw[e]);
    }
    const T g = gv[pt];
    if (!ok) {
      if (lane == 0) {
        if (a.gx)
          for (int e = 0; e < D; ++e) reinterpret_cast<T*>(a.gx)[pt * D + e] = (T)NAN;
        atomicAdd(&a.status->domain_errors, 1ull);
        dev_flag(a.status, LOVE_ERR_DOMAIN);
      }
      continue;
    }
    // v = Rt^T w, dv_e = Rt^T dw_e, u_e = KdP_e^T w  (lanes own columns lane + 32 j)
    T v[NCOL], dv[D][NCOL], u[D][NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      v[j] = T(0);
#pragma unroll
      for (int e = 0; e < D; ++e) dv[e][j] = u[e][j] = T(0);
    }
#pragma unroll 1
    for (int q = 0; q < NR; ++q) {
      int r0 = q & 3, r1 = (q >> 2) & 3, r2 = (q >> 4) & 3;
      int64_t row;
      T wq, dq[D];
      if (D == 1) {
        row = base[0] - 1 + r0;
        wq = w[0][r0];
        dq[0] = dw[0][r0];
      } else if (D == 2) {
        row = (int64_t)(base[0] - 1 + r1) * a.g.stride[0] + (base[1] - 1 + r0);
        wq = w[0][r1] * w[1][r0];
        dq[0] = dw[0][r1] * w[1][r0];
        dq[D - 1] = w[0][r1] * dw[1][r0];
      } else {
        row = (int64_t)(base[0] - 1 + r2) * a.g.stride[0] + (int64_t)(base[1] - 1 + r1) * a.g.stride[1] +
              (base[2] - 1 + r0);
        wq = w[0][r2] * w[1][r1] * w[2][r0];
        dq[0] = dw[0][r2] * w[1][r1] * w[2][r0];
        dq[1 % D] = w[0][r2] * dw[1][r1] * w[2][r0];
        dq[D - 1] = w[0][r2] * w[1][r1] * dw[2][r0];
      }
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        int c = lane + 32 * j;
        if (c < a.k) {
          T rv = ldc<T>(a.Rc, row * a.ld + c, a.cdt);
          v[j] += wq * rv;
#pragma unroll
          for (int e = 0; e < D; ++e) {
            dv[e][j] += dq[e] * rv;
            u[e][j] += wq * KdP[((int64_t)e * a.g.m + row) * a.ld_g + c];
          }
        }
      }
    }
    // warp sums: v.dv_e, u_e.v, v^T B_e v, v^T Minv v (double-float accumulation)
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      int c = lane + 32 * j;
      if (c < a.k) vsh[wp][c] = v[j];
    }
    __syncwarp();
    Acc s_vdv[D], s_uv[D], s_b[D], s_m;
    s_m.zero();
#pragma unroll
    for (int e = 0; e < D; ++e) {
      s_vdv[e].zero();
      s_uv[e].zero();
      s_b[e].zero();
    }
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      int c = lane + 32 * j;
      if (c >= a.k) continue;
#pragma unroll
      for (int e = 0; e < D; ++e) {
        s_vdv[e].add_prod(v[j], dv[e][j]);
        s_uv[e].add_prod(u[e][j], v[j]);
      }
      // row c of B_e and Minv against v.  Both matrices are symmetric, so row c
      // is read as column c (lanes read consecutive addresses); four
      // independent accumulators per product keep the chains short.
      Acc bm[D][4], mm[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        mm[u].zero();
#pragma unroll
        for (int e = 0; e < D; ++e) bm[e][u].zero();
      }
      int b = 0;
      for (; b + 3 < a.k; b += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T vb = vsh[wp][b + u];
          mm[u].add_prod(Mi[(int64_t)(b + u) * a.k + c], vb);
#pragma unroll
          for (int e = 0; e < D; ++e) bm[e][u].add_prod(Bm[((int64_t)e * a.k + b + u) * a.k + c], vb);
        }
      }
      for (; b < a.k; ++b) {
        const T vb = vsh[wp][b];
        mm[0].add_prod(Mi[(int64_t)b * a.k + c], vb);
#pragma unroll
        for (int e = 0; e < D; ++e) bm[e][0].add_prod(Bm[((int64_t)e * a.k + b) * a.k + c], vb);
      }
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        mm[0].merge(mm[u].s, mm[u].c);
#pragma unroll
        for (int e = 0; e < D; ++e) bm[e][0].merge(bm[e][u].s, bm[e][u].c);
      }
      s_m.add_prod((T)mm[0].value(), v[j]);
#pragma unroll
      for (int e = 0; e < D; ++e) s_b[e].add_prod((T)bm[e][0].value(), v[j]);
    }
    __syncwarp();
    warp_merge(s_m);
#pragma unroll
    for (int e = 0; e < D; ++e) {
      warp_merge(s_vdv[e]);
      warp_merge(s_uv[e]);
      warp_merge(s_b[e]);
    }
    if (lane == 0) {
      double wd[D][4], dwd[D][4];
#pragma unroll
      for (int e = 0; e < D; ++e)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          wd[e][r] = (double)w[e][r];
          dwd[e][r] = (double)dw[e][r];
        }
      const double gd = (double)g;
#pragma unroll
      for (int e = 0; e < D; ++e) {
        // (dw/dx_e)^T K w and w^T K'_e w on the 4^d stencil (product kernel factorises)
        double dp = 1.0, pl = 1.0;
#pragma unroll
        for (int f = 0; f < D; ++f) {
          dp *= (f == e) ? quad_loc(dwd[f], wd[f], a.cl[f]) : quad_loc(wd[f], wd[f], a.cl[f]);
          pl *= (f == e) ? quad_loc(wd[f], wd[f], a.cld[f]) : quad_loc(wd[f], wd[f], a.cl[f]);
        }
        if (a.exact_prior) {
          dp = 0.0;
          pl = 0.0;
        }
        if (a.gx) reinterpret_cast<T*>(a.gx)[pt * D + e] = (T)(gd * 2.0 * (dp - s_vdv[e].value()));
        hyp[e] += gd * (pl - 2.0 * s_uv[e].value() + s_b[e].value());
      }
      hyp[LOVE_MAX_DIM] += gd * s_m.value();
    }
  }
  // block and grid reduction of the hyperparameter sums (fixed order)
  if (lane == 0)
    for (int q = 0; q <= LOVE_MAX_DIM; ++q) red[wp][q] = hyp[q];
  __syncthreads();
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    double tot[LOVE_MAX_DIM + 1] = {0, 0, 0, 0};
    for (int w_ = 0; w_ < BWD_WARPS; ++w_)
      for (int q = 0; q <= LOVE_MAX_DIM; ++q) tot[q] += red[w_][q];
    for (int q = 0; q <= LOVE_MAX_DIM; ++q) a.partial[(int64_t)blockIdx.x * (LOVE_MAX_DIM + 1) + q] = make_double2(tot[q], 0.0);
    __threadfence();
    is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    for (int q = 0; q <= LOVE_MAX_DIM; ++q) {
      double s = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&a.partial[(int64_t)b * (LOVE_MAX_DIM + 1) + q]).x;
      a.result[q] = s;
    }
    *a.counter = 0u;
  }
}

template <typename T>
love_status tables_impl(love_cache* c, const FftPlan* plans, const T* P, int k, cudaStream_t s) {
  const GridHost& gh = c->grid;
  const Allocator& al = c->alloc;
  const int64_t m = gh.m;
  const int dim = gh.dim;
  const int vec = 16 / (int)sizeof(T);
  c->ld_g = (k + vec - 1) / vec * vec;
  c->KdP = al.alloc(sizeof(T) * (size_t)dim * m * c->ld_g, s);
  c->B = al.alloc(sizeof(T) * (size_t)dim * k * k, s);
  c->Minv = al.alloc(sizeof(T) * (size_t)k * k, s);
  if (!c->KdP || !c->B || !c->Minv) return LOVE_ERR_OOM;
  size_t yb = sizeof(T) * (size_t)m * k;
  size_t fwb = fft_work_bytes(gh, plans, k, true);
  T* Y = (T*)al.alloc(yb, s);
  void* fw = al.alloc(std::max<size_t>(fwb, 16), s);
  const size_t ddb = sizeof(double) * (4 * (k + 1) + (size_t)k * k);
  double* dd = (double*)al.alloc(ddb, s);
  love_status rc = (Y && fw && dd) ? LOVE_OK : LOVE_ERR_OOM;
  for (int e = 0; e < dim && rc == LOVE_OK; ++e) {
    rc = kuu_apply<T>(gh, plans, P, Y, k, m, fw, e, s);
    if (rc != LOVE_OK) break;
    LOVE_COUNT_LAUNCH(); k_colmajor_to_rows<T><<<ceil_div(m * c->ld_g, 256), 256, 0, s>>>(Y, m, k, (T*)c->KdP + (size_t)e * m * c->ld_g, c->ld_g);
    LOVE_COUNT_LAUNCH(); k_gram<T><<<k * k, 256, 0, s>>>(P, Y, m, k, (T*)c->B + (size_t)e * k * k);
    rc = cuda_check(cudaGetLastError());
  }
  if (rc == LOVE_OK) {
    // alpha, beta of T to the device; k_minv factors T and forms L^{-1} L^{-T}
    rc = cuda_check(cudaMemcpyAsync(dd, c->alpha, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK && k > 1)
      rc = cuda_check(cudaMemcpyAsync(dd + (k + 1), c->beta, sizeof(double) * (k - 1), cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK) {
      LOVE_COUNT_LAUNCH(); k_minv<<<1, 256, 0, s>>>(dd, dd + (k + 1), k, dd + 2 * (k + 1), c->Minv, sizeof(T) == 8, c->status);
      rc = cuda_check(cudaGetLastError());
    }
  }
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  al.free(Y, yb, s);
  al.free(fw, std::max<size_t>(fwb, 16), s);
  al.free(dd, ddb, s);
  return rc;
}

template <typename T>
love_status bwd_impl(love_cache* c, int64_t t, const void* x, const void* gv, void* gx, double* gl, double* gn,
                     cudaStream_t s) {
  const Allocator& al = c->alloc;
  if (c->k_eff > BWD_MAXK) return LOVE_ERR_UNSUPPORTED;
  BwdArgs a{};
  a.g = c->grid.dev();
  a.t = t;
  a.x = x;
  a.gv = gv;
  a.gx = gx;
  a.Rc = c->Rc;
  a.ld = c->ld;
  a.cdt = c->cache_dtype;
  a.KdP = c->KdP;
  a.ld_g = c->ld_g;
  a.B = c->B;
  a.Minv = c->Minv;
  a.k = c->k_eff;
  a.exact_prior = (c->flags & LOVE_PRIOR_EXACT) ? 1 : 0;
  for (int e = 0; e < LOVE_MAX_DIM; ++e)
    for (int q = 0; q < 4; ++q) {
      double sc = e == 0 ? c->grid.sf : 1.0;
      a.cl[e][q] = c->grid.cloc[e][q] * sc;
      a.cld[e][q] = c->grid.cloc_dl[e][q] * sc;
    }
  a.status = c->status;
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((t + BWD_WARPS - 1) / BWD_WARPS, (int64_t)num_sms() * 8));
  size_t pb = sizeof(double2) * (size_t)blocks * (LOVE_MAX_DIM + 1);
  size_t rb = sizeof(double) * (LOVE_MAX_DIM + 1) + 64;
  double2* part = (double2*)al.alloc(pb, s);
  double* res = (double*)al.alloc(rb, s);
  if (!part || !res) return LOVE_ERR_OOM;
  a.partial = part;
  a.result = res;
  a.counter = (unsigned*)(res + LOVE_MAX_DIM + 1);
  love_status rc = cuda_check(cudaMemsetAsync(res, 0, rb, s));
  if (rc == LOVE_OK && t > 0) {
    switch (a.g.dim) {
      case 1: LOVE_COUNT_LAUNCH(); k_var_backward<T, 1><<<blocks, BWD_WARPS * 32, 0, s>>>(a); break;
      case 2: LOVE_COUNT_LAUNCH(); k_var_backward<T, 2><<<blocks, BWD_WARPS * 32, 0, s>>>(a); break;
      default: LOVE_COUNT_LAUNCH(); k_var_backward<T, 3><<<blocks, BWD_WARPS * 32, 0, s>>>(a);
    }
    rc = cuda_check(cudaGetLastError());
  }
  if (rc == LOVE_OK && (gl || gn)) {
    double h[LOVE_MAX_DIM + 1];
    rc = cuda_check(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc == LOVE_OK) {
      if (gl)
        for (int e = 0; e < c->grid.dim; ++e) gl[e] = h[e];
      if (gn) *gn = h[LOVE_MAX_DIM];
    }
  }
  al.free(part, pb, s);
  al.free(res, rb, s);
  return rc;
}

}  // namespace

love_status backward_tables(love_cache* c, const FftPlan* plans, const void* P, int k, cudaStream_t s) {
  if (c->dtype == LOVE_F64) return tables_impl<double>(c, plans, (const double*)P, k, s);
  return tables_impl<float>(c, plans, (const float*)P, k, s);
}

love_status backward_launch(love_cache* c, int64_t t, const void* x, const void* gv, void* gx, double* gl, double* gn,
                            cudaStream_t s) {
  if (c->dtype == LOVE_F64) return bwd_impl<double>(c, t, x, gv, gx, gl, gn, s);
  return bwd_impl<float>(c, t, x, gv, gx, gl, gn, s);
}

}  // namespace love
