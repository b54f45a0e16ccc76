// k_cg.cu -- the mean cache's solves (Sec. 3, predictive mean): CG on
// K^ z = y in the training points' space (FP64, or double-float for FP32
// data), and the grid-space solves of 1-D and 2-D grids (CG in the K inner
// product, right-preconditioned GMRES).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lanczos_common.cuh"

namespace love {

namespace {

constexpr int GM_R = 40;        // GMRES restart length (Arnoldi steps per cycle)
constexpr int GM_CYCLES = 4;    // GMRES cycles before the mean solve falls back to plain CG

// ---------------------------------------------------------------------------
// CG (Sec. 2.1) for the mean cache: K^ z = y on the cell-sorted vectors.  The
// vectors and all reductions are FP64 whatever the coordinate type T (the
// interpolation weights stay in T, as in the Lanczos MVMs): an FP32 CG stalls
// on this ill-conditioned system (cond(K^) ~ 1e7 on the n = 1e6 workload).
// p = r + beta p (the new direction, written back); Ap = W^T u + s^2 p; pAp = p . Ap
// (u = K_UU W p was scattered from r + beta p on the fly)
template <typename T, int D>
__global__ void k_cg_gather_dot(GridDev g, const T* __restrict__ xs, int64_t n, int64_t n_pad,
                                const double* __restrict__ u, double noise, const double* __restrict__ r,
                                double* __restrict__ pv, double* __restrict__ Ap, double2* partial, LanczosState* st) {
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double be = st->cg_beta;
  DotAccD a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    const double pn = r[p] + be * pv[p];
    pv[p] = pn;
    double q = 0.0;
    if (p < n) {
      Stencil<T, D> stc;
      stc.compute(xs + p * D, g);
      q = stc.apply(u, g) + noise * pn;
    }
    Ap[p] = q;
    a.add_prod(pn, q);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->pap, st->counter2);
  if (last && threadIdx.x == 0) st->cg_alpha = st->rr / st->pap;
}
// x += a p ; r -= a Ap ; rr' = r.r
__global__ void k_cg_update(int64_t n_pad, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ pv, const double* __restrict__ Ap, double2* partial,
                            LanczosState* st, int max_iter, DevStatus* status) {
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double al = st->cg_alpha;
  DotAccD a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    x[p] += al * pv[p];
    double rv = r[p] - al * Ap[p];
    r[p] = rv;
    a.add_prod(rv, rv);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    double rrn = st->norm2;
    st->cg_beta = rrn / st->rr;
    st->rr = rrn;
    st->cg_iters += 1;
    if (!isfinite(rrn)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (rrn <= st->tol2 || st->cg_iters >= max_iter) {
      st->cg_done = 1;
    }
  }
}
template <typename T>
__global__ void k_cg_init(int64_t n_pad, const T* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
                          double* __restrict__ pv, double2* partial, LanczosState* st, double tol) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)b[p];
    x[p] = 0.0;
    r[p] = v;
    pv[p] = 0.0;  // first direction r + 0 p = r
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr = st->norm2;
    st->rr0 = st->norm2;
    st->tol2 = tol * tol * st->norm2;
    st->cg_iters = 0;
    st->cg_beta = 0.0;
    st->cg_done = st->norm2 == 0.0 ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// The same CG for the FP32 path in double-float: x, r, p, Ap are (hi, lo) float
// pairs (~48-bit), every operation runs on the FP32 pipes (GB300's FP64 rate
// is a small fraction of FP32), and K_UU still goes through the FP64 FFT on
// the m-sized grid vectors.
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ void acc_add_dfprod(DotAccF& acc, df a, df b) {
  acc.add_prod(a.hi, b.hi);
  acc.c += fmaf(a.hi, b.lo, a.lo * b.hi);
}

// u[node] = sum over sorted points of w_p(node) (r_p + beta p_p), FP64 result
template <int D>
__global__ void k_scatter_df(GridDev g, const float* __restrict__ xs, const int* __restrict__ cell_start,
                             const df* __restrict__ r, const df* __restrict__ pv, const LanczosState* st,
                             double* __restrict__ u) {
  if (st->cg_done) return;
  const df be = df_from_double(st->cg_beta);
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t node = wg; node < g.m; node += nw) {
    int nd[D];
    node_index<D>(node, g, nd);
    NodeRanges<D> rg;
    rg.build(g, nd, cell_start, lane);
    DotAccF acc;
    acc.zero();
    for (int f = lane; f < rg.total; f += 32) {
      int p = rg.point(f);
      df val = df_add(r[p], df_mul(be, pv[p]));
      float w = node_weight<float, D>(xs + (int64_t)p * D, g, nd);
      acc.add_prod(w, val.hi);
      acc.c += w * val.lo;
    }
    warp_merge(acc);
    if (lane == 0) u[node] = acc.value();
  }
}
__global__ void k_double_to_df(int64_t m, const double* __restrict__ a, df* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = df_from_double(a[i]);
}
// p = r + beta p (written back); Ap = W^T u + s^2 p; pAp = p . Ap
template <int D>
__global__ void k_cgdf_gather_dot(GridDev g, const float* __restrict__ xs, int64_t n, int64_t n_pad,
                                  const df* __restrict__ u, double noise, const df* __restrict__ r,
                                  df* __restrict__ pv, df* __restrict__ Ap, double2* partial, LanczosState* st) {
  __shared__ DotAccF red[32];
  if (st->cg_done) return;
  const df be = df_from_double(st->cg_beta);
  const df nz = df_from_double(noise);
  DotAccF a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    const df pn = df_add(r[p], df_mul(be, pv[p]));
    pv[p] = pn;
    df q = {0.f, 0.f};
    if (p < n) {
      Stencil<float, D> stc;
      stc.compute(xs + p * D, g);
      // sum over the 4^D stencil nodes of w * u (df)
      if (D == 1) {
#pragma unroll
        for (int r0 = 0; r0 < 4; ++r0) q = df_add(q, df_mul_f(u[stc.base[0] - 1 + r0], stc.w[0][r0]));
      } else if (D == 2) {
#pragma unroll
        for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
          for (int r1 = 0; r1 < 4; ++r1) {
            int64_t node = (int64_t)(stc.base[0] - 1 + r0) * g.stride[0] + (stc.base[1] - 1 + r1);
            q = df_add(q, df_mul_f(u[node], stc.w[0][r0] * stc.w[1][r1]));
          }
      } else {
#pragma unroll
        for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
          for (int r1 = 0; r1 < 4; ++r1)
#pragma unroll
            for (int r2 = 0; r2 < 4; ++r2) {
              int64_t node = (int64_t)(stc.base[0] - 1 + r0) * g.stride[0] +
                             (int64_t)(stc.base[1] - 1 + r1) * g.stride[1] + (stc.base[2] - 1 + r2);
              q = df_add(q, df_mul_f(u[node], stc.w[0][r0] * stc.w[1][r1] * stc.w[2][r2]));
            }
      }
      q = df_add(q, df_mul(nz, pn));
    }
    Ap[p] = q;
    acc_add_dfprod(a, pn, q);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccF>(partial, 1, 1, &st->pap, st->counter2);
  if (last && threadIdx.x == 0) st->cg_alpha = st->rr / st->pap;
}
// x += a p ; r -= a Ap ; rr' = r.r
__global__ void k_cgdf_update(int64_t n_pad, df* __restrict__ x, df* __restrict__ r, const df* __restrict__ pv,
                              const df* __restrict__ Ap, double2* partial, LanczosState* st, int max_iter,
                              DevStatus* status) {
  __shared__ DotAccF red[32];
  if (st->cg_done) return;
  const df al = df_from_double(st->cg_alpha);
  const df mal = df_neg(al);
  DotAccF a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    x[p] = df_add(x[p], df_mul(al, pv[p]));
    df rv = df_add(r[p], df_mul(mal, Ap[p]));
    r[p] = rv;
    acc_add_dfprod(a, rv, rv);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccF>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    double rrn = st->norm2;
    st->cg_beta = rrn / st->rr;
    st->rr = rrn;
    st->cg_iters += 1;
    if (!isfinite(rrn)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (rrn <= st->tol2 || st->cg_iters >= max_iter) {
      st->cg_done = 1;
    }
  }
}
__global__ void k_cgdf_init(int64_t n_pad, const float* __restrict__ b, df* __restrict__ x, df* __restrict__ r,
                            df* __restrict__ pv, double2* partial, LanczosState* st, double tol) {
  __shared__ DotAccF red[32];
  DotAccF a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    float v = b[p];
    x[p] = {0.f, 0.f};
    r[p] = {v, 0.f};
    pv[p] = {0.f, 0.f};
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccF>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr = st->norm2;
    st->rr0 = st->norm2;
    st->tol2 = tol * tol * st->norm2;
    st->cg_iters = 0;
    st->cg_beta = 0.0;
    st->cg_done = st->norm2 == 0.0 ? 1 : 0;
  }
}
__global__ void k_df_to_double(int64_t n, const df* __restrict__ a, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = df_to_double(a[i]);
}

}  // namespace

// FP32 ski: double-float CG; the solution is returned as FP64 in x
love_status cg_solve_df(love_ski* ski, const float* b, double* x, double tol, int max_iter, int* iters,
                        cudaStream_t s) {
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int64_t np = ski->n_pad;
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), xb(ski->alloc, s), r(ski->alloc, s), pv(ski->alloc, s),
      Ap(ski->alloc, s), u(ski->alloc, s), udf(ski->alloc, s), fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * 1024) || !xb.get(sizeof(df) * np) ||
      !r.get(sizeof(df) * np) || !pv.get(sizeof(df) * np) || !Ap.get(sizeof(df) * np) ||
      !u.get(sizeof(double) * gh.m * 2) || !udf.get(sizeof(df) * gh.m) || !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  double* u1 = u.as<double>();
  double* u2 = u1 + gh.m;
  const int blocks = std::min(1024, ceil_div(np, 256));
  const int sblocks = (int)std::min<int64_t>((g.m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, 1, 0.0);
  LOVE_COUNT_LAUNCH(); k_cgdf_init<<<blocks, 256, 0, s>>>(np, b, xb.as<df>(), r.as<df>(), pv.as<df>(), part.as<double2>(), st, tol);
  LOVE_LAUNCH_CHECK();
  int it = 0;
  const int chunk = 32;
  while (it < max_iter) {
    for (int c = 0; c < chunk && it < max_iter; ++c, ++it) {
      switch (g.dim) {
        case 1: LOVE_COUNT_LAUNCH(); k_scatter_df<1><<<sblocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->cell_start, r.as<df>(), pv.as<df>(), st, u1); break;
        case 2: LOVE_COUNT_LAUNCH(); k_scatter_df<2><<<sblocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->cell_start, r.as<df>(), pv.as<df>(), st, u1); break;
        default: LOVE_COUNT_LAUNCH(); k_scatter_df<3><<<sblocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->cell_start, r.as<df>(), pv.as<df>(), st, u1);
      }
      LOVE_TRY(kuu_apply<double>(gh, ski->fft, u1, u2, 1, gh.m, fw.p, -1, s));
      LOVE_COUNT_LAUNCH(); k_double_to_df<<<ceil_div(gh.m, 256), 256, 0, s>>>(gh.m, u2, udf.as<df>());
      switch (g.dim) {
        case 1: LOVE_COUNT_LAUNCH(); k_cgdf_gather_dot<1><<<blocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->n, np, udf.as<df>(), gh.noise, r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st); break;
        case 2: LOVE_COUNT_LAUNCH(); k_cgdf_gather_dot<2><<<blocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->n, np, udf.as<df>(), gh.noise, r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st); break;
        default: LOVE_COUNT_LAUNCH(); k_cgdf_gather_dot<3><<<blocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->n, np, udf.as<df>(), gh.noise, r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st);
      }
      LOVE_COUNT_LAUNCH(); k_cgdf_update<<<blocks, 256, 0, s>>>(np, xb.as<df>(), r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st, max_iter, ski->status);
      LOVE_LAUNCH_CHECK();
    }
    int done = 0;
    LOVE_CUDA(cudaMemcpyAsync(&done, &st->cg_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (done) break;
  }
  LOVE_COUNT_LAUNCH(); k_df_to_double<<<ceil_div(np, 256), 256, 0, s>>>(np, xb.as<df>(), x);
  LOVE_LAUNCH_CHECK();
  int n_it = 0;
  LOVE_CUDA(cudaMemcpyAsync(&n_it, &st->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = n_it;
  return LOVE_OK;
}

template <typename T>
love_status cg_solve(love_ski* ski, const T* b, double* x, double tol, int max_iter, int* iters, cudaStream_t s) {
  // the double-float form scatters over the product grid only; an additive
  // grid takes the FP64-vector form below
  if (sizeof(T) == 4 && !ski->grid.additive) return cg_solve_df(ski, (const float*)b, x, tol, max_iter, iters, s);
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int64_t np = ski->n_pad;
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), r(ski->alloc, s), pv(ski->alloc, s), Ap(ski->alloc, s),
      u(ski->alloc, s), fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * 1024) || !r.get(sizeof(double) * np) ||
      !pv.get(sizeof(double) * np) || !Ap.get(sizeof(double) * np) || !u.get(sizeof(double) * gh.m * 2) ||
      !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  double* u1 = u.as<double>();
  double* u2 = u1 + gh.m;
  int blocks = std::min(1024, ceil_div(np, 256));
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, 1, 0.0);
  LOVE_COUNT_LAUNCH(); k_cg_init<T><<<blocks, 256, 0, s>>>(np, b, x, r.as<double>(), pv.as<double>(), part.as<double2>(), st, tol);
  LOVE_LAUNCH_CHECK();
  int it = 0;
  const int chunk = 32;
  while (it < max_iter) {
    for (int c = 0; c < chunk && it < max_iter; ++c, ++it) {
      LOVE_TRY(scatter_any<T, double>(ski, r.as<double>(), nullptr, 1.0, u1, s, pv.as<double>(), &st->cg_beta,
                                      &st->cg_done));
      LOVE_TRY(kuu_apply<double>(gh, ski->fft, u1, u2, 1, gh.m, fw.p, -1, s));
      switch (g.dim) {
        case 1: LOVE_COUNT_LAUNCH(); k_cg_gather_dot<T, 1><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, np, u2, gh.noise, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st); break;
        case 2: LOVE_COUNT_LAUNCH(); k_cg_gather_dot<T, 2><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, np, u2, gh.noise, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st); break;
        default: LOVE_COUNT_LAUNCH(); k_cg_gather_dot<T, 3><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, np, u2, gh.noise, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st);
      }
      LOVE_COUNT_LAUNCH(); k_cg_update<<<blocks, 256, 0, s>>>(np, x, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st, max_iter,
                                           ski->status);
      LOVE_LAUNCH_CHECK();
    }
    int done = 0;
    LOVE_CUDA(cudaMemcpyAsync(&done, &st->cg_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (done) break;
  }
  int n_it = 0;
  LOVE_CUDA(cudaMemcpyAsync(&n_it, &st->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = n_it;
  return LOVE_OK;
}

// ---------------------------------------------------------------------------
// Mean cache on the grid (d <= 2).  W is m x n here (u = W v scatters points
// to nodes) and G = W W^T is the m x m Gram matrix of the interpolation
// weights, banded with 7^d diagonals.  The push-through identity
//   W (W^T K W + s^2 I)^-1 = (G K + s^2 I)^-1 W
// turns the mean weights a = K_UU W K^^-1 y (Sec. 3, predictive mean) into
//   a = K z,   A z = W y,   A = G K + s^2 I,
// an m-sized system.  A is self-adjoint and positive definite in the inner
// product <u, v>_K = u^T K v (K A = K G K + s^2 K), with eigenvalues >= s^2,
// so CG runs in that inner product: s = K r and q = K p are carried by
// recurrence, leaving one K product (FFT) per iteration and no n-sized work.
// Stopping rule: CG minimises E = <e, A e>_K over the Krylov space (e the
// error of z), and |W^T (a_i - a)|^2 = e^T K G K e <= E <= <r, r>_K / s^2, so
//   rho = r^T K r <= tol^2 s^2 |y|^2
// bounds the error of the fitted values at the training points by tol |y|,
// the same guarantee the rule |y - K^ x| <= tol |y| gives CG on K^ x = y
// (there W^T (a_i - a) = (K^ - s^2 I) K^^-1 r, a contraction of r).
namespace {

template <int D> struct Band { static constexpr int B = D == 1 ? 7 : 49; };

// G[o][node] = sum_p w_p(node) w_p(node + off(o)), offsets -3..3 per dimension;
// warp per node over the cell-sorted points, FP64 accumulation
template <typename T, int D>
__global__ void k_gram_band(GridDev g, const T* __restrict__ xs, const int* __restrict__ cell_start,
                            double* __restrict__ G) {
  constexpr int B = Band<D>::B;
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t node = wg; node < g.m; node += nw) {
    int nd[D];
    node_index<D>(node, g, nd);
    NodeRanges<D> rg;
    rg.build(g, nd, cell_start, lane);
    double acc[B];
#pragma unroll
    for (int o = 0; o < B; ++o) acc[o] = 0.0;
    for (int f = lane; f < rg.total; f += 32) {
      const int p = rg.point(f);
      T wd[D][7];
#pragma unroll
      for (int e = 0; e < D; ++e) {
        T sc = grid_coord(xs[(int64_t)p * D + e], g, e);
        int i = (int)floor(sc);
        if (i > g.g[e] - 3) i = g.g[e] - 3;
        T fr = sc - T(i);
#pragma unroll
        for (int o = 0; o < 7; ++o) wd[e][o] = keys_u(fr + T(1) - T(nd[e] + o - 3 - (i - 1)));
      }
      if constexpr (D == 1) {
#pragma unroll
        for (int o = 0; o < 7; ++o) acc[o] = fma((double)wd[0][3], (double)wd[0][o], acc[o]);
      } else {
        const T wu = wd[0][3] * wd[D - 1][3];
#pragma unroll
        for (int o0 = 0; o0 < 7; ++o0)
#pragma unroll
          for (int o1 = 0; o1 < 7; ++o1)
            acc[o0 * 7 + o1] = fma((double)wu, (double)(wd[0][o0] * wd[D - 1][o1]), acc[o0 * 7 + o1]);
      }
    }
#pragma unroll
    for (int o = 0; o < B; ++o) {
      double v = acc[o];
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
      if (lane == 0) G[(int64_t)o * g.m + node] = v;
    }
  }
}

// The new direction p = r + beta p', q = s + beta q' (q = K p) is formed on
// the fly (at the node and at its band neighbours, the same fma everywhere)
// and written to the other buffer of a pair; then t = G q + s^2 p (= A p) and
// pi = q . t (= <p, A p>_K).
template <int D>
__global__ void k_mcg_band(GridDev g, const double* __restrict__ G, const double* __restrict__ r,
                           const double* __restrict__ sv, const double* __restrict__ p_old,
                           const double* __restrict__ q_old, double* __restrict__ p_new, double* __restrict__ q_new,
                           double noise, double* __restrict__ t, double2* partial, LanczosState* st, int max_iter,
                           DevStatus* status) {
  constexpr int B = Band<D>::B;
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double be = st->cg_beta;
  DotAccD api;
  api.zero();
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.m;
       node += (int64_t)gridDim.x * blockDim.x) {
    int nd[D];
    node_index<D>(node, g, nd);
    double gq = 0.0;
#pragma unroll
    for (int o = 0; o < B; ++o) {
      const int o0 = D == 1 ? o : o / 7, o1 = o % 7;
      const int a0 = nd[0] + o0 - 3;
      const int a1 = D == 1 ? 0 : nd[D - 1] + o1 - 3;
      bool in = a0 >= 0 && a0 < g.g[0];
      if (D == 2) in = in && a1 >= 0 && a1 < g.g[1];
      if (in) {
        const int64_t nb = D == 1 ? a0 : (int64_t)a0 * g.stride[0] + a1;
        gq = fma(G[(int64_t)o * g.m + node], fma(be, q_old[nb], sv[nb]), gq);
      }
    }
    const double pn = fma(be, p_old[node], r[node]);
    const double qn = fma(be, q_old[node], sv[node]);
    p_new[node] = pn;
    q_new[node] = qn;
    const double tv = gq + noise * pn;
    t[node] = tv;
    api.add_prod(qn, tv);
  }
  block_merge(api, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, api);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->pap, st->counter2);
  if (last && threadIdx.x == 0) {
    const double pi = st->pap;
    if (!isfinite(pi)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (pi <= 0.0 || st->cg_iters >= max_iter) {
      st->cg_done = 1;
    } else {
      st->cg_alpha = st->rr / pi;
    }
  }
}

// w += a q;  r -= a t;  s -= a K t;  rho' = r . s
__global__ void k_mcg_update(int64_t m, double* __restrict__ w, double* __restrict__ r, double* __restrict__ sv,
                             const double* __restrict__ q, const double* __restrict__ t,
                             const double* __restrict__ Kt, double2* partial, LanczosState* st, DevStatus* status) {
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double al = st->cg_alpha;
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    w[i] = fma(al, q[i], w[i]);
    const double rv = fma(-al, t[i], r[i]);
    const double sn = fma(-al, Kt[i], sv[i]);
    r[i] = rv;
    sv[i] = sn;
    a.add_prod(rv, sn);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    const double rho = st->norm2;
    st->cg_beta = rho / st->rr;
    st->rr = rho;
    st->cg_iters += 1;
    if (!isfinite(rho)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (rho <= st->tol2) {
      st->cg_done = 1;
    }
  }
}

// |y|^2 -> the stopping threshold tol^2 s^2 |y|^2
template <typename T>
__global__ void k_mcg_ynorm(int64_t n, const T* __restrict__ y, double* __restrict__ yd, double tol, double noise,
                            double2* partial, LanczosState* st) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)y[i];
    if (yd) yd[i] = v;
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr0 = st->norm2;
    st->tol2 = tol * tol * st->norm2 * noise;
    st->cg_iters = 0;
    st->cg_beta = 0.0;
    st->cg_done = st->norm2 == 0.0 ? 1 : 0;
  }
}

// r = b, s = K b, w = 0, p' = q' = 0 (so the first direction is p = r, q = s);
// rho = r . s
__global__ void k_mcg_start(int64_t m, const double* __restrict__ b, const double* __restrict__ Kb,
                            double* __restrict__ r, double* __restrict__ pv, double* __restrict__ sv,
                            double* __restrict__ q, double* __restrict__ w, double2* partial, LanczosState* st) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = b[i];
    pv[i] = 0.0;
    sv[i] = Kb[i];
    q[i] = 0.0;
    w[i] = 0.0;
    a.add_prod(b[i], Kb[i]);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr = st->norm2;
    if (!(st->norm2 > st->tol2)) st->cg_done = 1;
  }
}

// ---- preconditioned grid-space solve (1-D grids) ------------------------------
// M = B K + s^2 I, B the symmetric Toeplitz stencil of G = W W^T averaged over
// the interior nodes (7 diagonals).  B and K are both Toeplitz, so on the
// circulant embedding of length N, P = M^{-1} is approximated by the spectral
// multiplier 1 / (lambda_B lambda_K + s^2) applied to the zero-padded vector
// and cropped back to the grid.  P does not commute with K exactly (the crop),
// so it is used as a right preconditioner of GMRES rather than inside CG.

// bhat[d] = average over interior nodes of (G[node, node+d] + G[node, node-d]) / 2;
// bhat[4] = fraction of interior nodes whose G_ii is below a fifth of the
// average (empty stretches of the grid, where the stencil does not fit)
__global__ void k_pcg_stencil(const double* __restrict__ G, int64_t m, double* __restrict__ bhat) {
  __shared__ double red[4][256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t lo = 6, hi = m - 6;   // nodes whose 7-wide band sees the whole data range
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    acc[0] += G[3 * m + i];
#pragma unroll
    for (int d = 1; d < 4; ++d) acc[d] += 0.5 * (G[(int64_t)(3 + d) * m + i] + G[(int64_t)(3 - d) * m + i]);
  }
#pragma unroll
  for (int d = 0; d < 4; ++d) red[d][threadIdx.x] = acc[d];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int d = 0; d < 4; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + w];
    __syncthreads();
  }
  const double b0 = hi > lo ? red[0][0] / (double)(hi - lo) : 0.0;
  if (threadIdx.x < 4) bhat[threadIdx.x] = hi > lo ? red[threadIdx.x][0] / (double)(hi - lo) : 0.0;
  __syncthreads();
  double cnt = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) cnt += G[3 * m + i] < 0.2 * b0 ? 1.0 : 0.0;
  red[0][threadIdx.x] = cnt;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[0][threadIdx.x] += red[0][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) bhat[4] = hi > lo ? red[0][0] / (double)(hi - lo) : 1.0;
}

// symbol of P on the embedding (stored / N like the K_UU spectrum) and the
// largest eigenvalue of K's circulant embedding (>= the largest of K)
__global__ void k_pcg_symbol(const double* __restrict__ lamK, int64_t N, const double* __restrict__ bhat, double noise,
                             double* __restrict__ sym, unsigned long long* __restrict__ lk_bits) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double lb = bhat[0];
#pragma unroll
  for (int d = 1; d < 4; ++d) lb += 2.0 * bhat[d] * cospi(2.0 * (double)(d * j % N) / (double)N);
  const double lk = fmax((double)N * lamK[j], 0.0);
  sym[j] = 1.0 / ((fmax(lb, 0.0) * lk + noise) * (double)N);
  atomicMax(lk_bits, (unsigned long long)__double_as_longlong(lk));   // lk >= 0: bit order = value order
}

}  // namespace

bool mean_grid_cg_supported(const love_ski* ski) { return ski->grid.dim <= 2 && !ski->grid.additive; }

template <typename T>
love_status mean_grid_gmres(love_ski* ski, double tol, int max_iter, double* a, int* iters, bool* converged,
                            cudaStream_t s);

template <typename T>
love_status mean_grid_cg(love_ski* ski, double tol, int max_iter, double* a, int* iters, cudaStream_t s,
                         bool precond) {
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int dim = gh.dim;
  if (dim > 2) return LOVE_ERR_UNSUPPORTED;
  int pre_iters = 0;
  if (precond && dim == 1 && gh.g[0] >= 16) {
    // the averaged stencil fits G where the training points are spread over
    // the grid; where they are not (clusters, gaps) the GMRES setup declines
    // (more than 10 % of the interior nearly empty) or, should it stall, the
    // plain CG below takes over from zero after GM_CYCLES restarts
    bool conv = false;
    LOVE_TRY(mean_grid_gmres<T>(ski, tol, std::min(max_iter, GM_CYCLES * GM_R), a, &pre_iters, &conv, s));
    if (conv || pre_iters >= max_iter) {
      if (iters) *iters = pre_iters;
      return LOVE_OK;
    }
    max_iter -= pre_iters;
  }
  const int64_t m = gh.m, n = ski->n;
  const int B = dim == 1 ? 7 : 49;
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), Gb(ski->alloc, s), vec(ski->alloc, s), yb(ski->alloc, s),
      fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  const bool conv = sizeof(T) != sizeof(double);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * 2048) || !Gb.get(sizeof(double) * B * m) ||
      !vec.get(sizeof(double) * 9 * m) || (conv && !yb.get(sizeof(double) * std::max<int64_t>(n, 1))) ||
      !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  double* v = vec.as<double>();
  double *b = v, *r = v + m, *sv = v + 2 * m, *t = v + 3 * m, *Kt = v + 4 * m;
  double* pbuf[2] = {v + 5 * m, v + 6 * m};  // directions p, q: double-buffered
  double* qbuf[2] = {v + 7 * m, v + 8 * m};
  double* w = a;  // a = K z accumulates in place
  double2* pp = part.as<double2>();
  const int sblocks = (int)std::min<int64_t>((m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  const int mblocks = (int)std::min<int64_t>(ceil_div(m, 256), 1024);
  const int nblocks = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), 1024);
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, 1, 0.0);
  // G = W W^T
  if (dim == 1) {
    LOVE_COUNT_LAUNCH(); k_gram_band<T, 1><<<sblocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Gb.as<double>());
  } else {
    LOVE_COUNT_LAUNCH(); k_gram_band<T, 2><<<sblocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Gb.as<double>());
  }
  // b = W y (FP64), |y|^2
  const double* yd = conv ? yb.as<double>() : (const double*)ski->ys;
  LOVE_COUNT_LAUNCH();
  k_mcg_ynorm<T><<<nblocks, 256, 0, s>>>(n, (const T*)ski->ys, conv ? yb.as<double>() : nullptr, tol, gh.noise, pp, st);
  LOVE_LAUNCH_CHECK();
  // K products in FP64 transforms: with FP32 transforms (error ~log2(N) 2^-24)
  // the K-inner product loses positivity on the high-frequency components and
  // the iteration stops early (mean errors ~6e-3 std(y) on the n = 1e6 workload)
  auto kmul = [&](const double* in, double* out) -> love_status {
    return kuu_apply<double>(gh, ski->fft, in, out, 1, m, fw.p, -1, s);
  };
  LOVE_TRY(scatter_any<T, double>(ski, yd, nullptr, 1.0, b, s));
  LOVE_TRY(kmul(b, Kt));
  LOVE_COUNT_LAUNCH(); k_mcg_start<<<mblocks, 256, 0, s>>>(m, b, Kt, r, pbuf[0], sv, qbuf[0], w, pp, st);
  LOVE_LAUNCH_CHECK();
  int it = 0;
  const int chunk = 64;
  while (it <= max_iter) {
    for (int c = 0; c < chunk && it <= max_iter; ++c, ++it) {
      const double *po = pbuf[it & 1], *qo = qbuf[it & 1];
      double *pn = pbuf[(it + 1) & 1], *qn = qbuf[(it + 1) & 1];
      if (dim == 1) {
        LOVE_COUNT_LAUNCH(); k_mcg_band<1><<<mblocks, 256, 0, s>>>(g, Gb.as<double>(), r, sv, po, qo, pn, qn, gh.noise, t, pp, st, max_iter, ski->status);
      } else {
        LOVE_COUNT_LAUNCH(); k_mcg_band<2><<<mblocks, 256, 0, s>>>(g, Gb.as<double>(), r, sv, po, qo, pn, qn, gh.noise, t, pp, st, max_iter, ski->status);
      }
      LOVE_TRY(kmul(t, Kt));
      LOVE_COUNT_LAUNCH(); k_mcg_update<<<mblocks, 256, 0, s>>>(m, w, r, sv, qn, t, Kt, pp, st, ski->status);
      LOVE_LAUNCH_CHECK();
    }
    int done = 0;
    LOVE_CUDA(cudaMemcpyAsync(&done, &st->cg_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (done) break;
  }
  int n_it = 0;
  LOVE_CUDA(cudaMemcpyAsync(&n_it, &st->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = pre_iters + n_it;
  return LOVE_OK;
}
template love_status mean_grid_cg<float>(love_ski*, double, int, double*, int*, cudaStream_t, bool);
template love_status mean_grid_cg<double>(love_ski*, double, int, double*, int*, cudaStream_t, bool);

// ---------------------------------------------------------------------------
// Right-preconditioned GMRES for the grid-space mean system (1-D grids):
// A z = W y with A = G K_UU + s^2 I (G = W W^T banded), a = K_UU z; solved as
// A P u = W y, z = P u, with P the spectral approximation of (B K_UU + s^2 I)^{-1}.
// The Arnoldi basis V (m_pad x (R + 1), FP64) is orthogonalised by the same
// CGS2 tile kernels as the Lanczos runs; the Hessenberg columns go through
// Givens rotations on the device, so |g_{j+1}| is the Euclidean residual of
// the current iterate.  The solve stops when |g_{j+1}|^2 <= tol^2 s^2 |y|^2 /
// (2 lambda_max(K)), which implies the CG stopping rule r^T K r <= tol^2 s^2 |y|^2
// for the recursively updated residual (as the plain CG applies it); a cycle
// that ends without meeting it restarts from the recomputed residual b - A z.
namespace {

struct GmresState {
  double H[(GM_R + 1) * GM_R];   // rotated Hessenberg columns (upper triangle), ld GM_R + 1
  double cs[GM_R], sn[GM_R];
  double g[GM_R + 1];
  double y[GM_R];
  int ncols;
  int converged;
  double target2;
  unsigned long long lk_bits;   // largest eigenvalue of K's circulant embedding
};

__global__ void k_gm_target(GmresState* gm, const LanczosState* cg) {
  const double lk = __longlong_as_double((long long)gm->lk_bits);
  gm->target2 = 0.5 * cg->tol2 / fmax(lk, 1e-300);
}

// V[:, 0] = r (zero past m); g = (|r|, 0, ...); scal_0 = 1 / |r|
__global__ void k_gm_start(int64_t m, int64_t m_pad, const double* __restrict__ r, double* __restrict__ v0,
                           double2* partial, LanczosState* st, GmresState* gm, DevStatus* status) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = i < m ? r[i] : 0.0;
    v0[i] = v;
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter);
  if (last && threadIdx.x == 0) {
    const double b2 = st->norm2, b = sqrt(b2);
    gm->g[0] = b;
    for (int i = 1; i <= GM_R; ++i) gm->g[i] = 0.0;
    gm->ncols = 0;
    st->scal[0] = b > 0.0 ? 1.0 / b : 0.0;
    if (!isfinite(b2)) dev_flag(status, LOVE_ERR_NAN);
    if (!(b2 > gm->target2)) {
      st->done = 1;
      st->k_eff = 0;
      gm->converged = 1;
    }
  }
}

// y = G (K P v) + s^2 (P v) over the padded rows (zero past m)
__global__ void k_gm_band(int64_t m, int64_t m_pad, const double* __restrict__ G, const double* __restrict__ kv,
                          const double* __restrict__ pv, double noise, double* __restrict__ y,
                          const LanczosState* st) {
  if (st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (i < m) {
#pragma unroll
      for (int o = 0; o < 7; ++o) {
        const int64_t nb = i + o - 3;
        if (nb >= 0 && nb < m) acc = fma(G[(int64_t)o * m + i], kv[nb], acc);
      }
      acc = fma(noise, pv[i], acc);
    }
    y[i] = acc;
  }
}

// Hessenberg column j: h_ij = c_i + c'_i (the two Gram-Schmidt passes), h_{j+1,j}
// = beta_j; earlier rotations, then the rotation that zeroes h_{j+1,j}
__global__ void k_gm_givens(LanczosState* st, GmresState* gm, int j, DevStatus* status) {
  if (j >= st->k_eff || gm->ncols != j) return;
  double h[GM_R + 1];
  for (int i = 0; i <= j; ++i) h[i] = st->coef[i] + st->coef2[i];
  h[j + 1] = st->beta[j];
  for (int i = 0; i < j; ++i) {
    const double t = gm->cs[i] * h[i] + gm->sn[i] * h[i + 1];
    h[i + 1] = -gm->sn[i] * h[i] + gm->cs[i] * h[i + 1];
    h[i] = t;
  }
  const double r = hypot(h[j], h[j + 1]);
  const double c = r > 0.0 ? h[j] / r : 1.0, sn = r > 0.0 ? h[j + 1] / r : 0.0;
  gm->cs[j] = c;
  gm->sn[j] = sn;
  h[j] = r;
  gm->g[j + 1] = -sn * gm->g[j];
  gm->g[j] = c * gm->g[j];
  for (int i = 0; i <= j; ++i) gm->H[(int64_t)j * (GM_R + 1) + i] = h[i];
  gm->ncols = j + 1;
  if (!isfinite(gm->g[j + 1])) {
    dev_flag(status, LOVE_ERR_NAN);
    gm->converged = 1;   // nothing more to gain; the status reports it
    st->done = 1;
    st->k_eff = j;
    gm->ncols = j;
  } else if (gm->g[j + 1] * gm->g[j + 1] <= gm->target2) {
    st->done = 1;
    st->k_eff = j + 1;
    gm->converged = 1;
  }
}

// R y = g by back substitution (ncols columns)
__global__ void k_gm_solve(GmresState* gm) {
  const int kc = gm->ncols;
  for (int i = kc - 1; i >= 0; --i) {
    double v = gm->g[i];
    for (int l = i + 1; l < kc; ++l) v -= gm->H[(int64_t)l * (GM_R + 1) + i] * gm->y[l];
    const double d = gm->H[(int64_t)i * (GM_R + 1) + i];
    gm->y[i] = d != 0.0 ? v / d : 0.0;
  }
}

// u = V y
__global__ void k_gm_combine(int64_t m, const double* __restrict__ V, int64_t ldv, const GmresState* gm,
                             double* __restrict__ u) {
  const int kc = gm->ncols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < kc; ++c) acc = fma(V[(int64_t)c * ldv + i], gm->y[c], acc);
    u[i] = acc;
  }
}

__global__ void k_gm_add(int64_t m, double* __restrict__ z, const double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += d[i];
}

// r = b - (G K z + s^2 z)
__global__ void k_gm_resid(int64_t m, const double* __restrict__ G, const double* __restrict__ kz,
                           const double* __restrict__ z, const double* __restrict__ b, double noise,
                           double* __restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
      const int64_t nb = i + o - 3;
      if (nb >= 0 && nb < m) acc = fma(G[(int64_t)o * m + i], kz[nb], acc);
    }
    r[i] = b[i] - fma(noise, z[i], acc);
  }
}

}  // namespace

template <typename T>
love_status mean_grid_gmres(love_ski* ski, double tol, int max_iter, double* a, int* iters, bool* converged,
                            cudaStream_t s) {
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int64_t m = gh.m, n = ski->n;
  const int64_t m_pad = (m + TILE_R - 1) / TILE_R * TILE_R;
  const FftPlan& kp = ski->fft[0];
  const int bc = box_cols(sizeof(double));
  const int max_grid = std::max(TILE_CTAS_PER_SM * num_sms(), 1024);
  DevBuf stb(ski->alloc, s), cgb(ski->alloc, s), gmb(ski->alloc, s), part(ski->alloc, s), Gb(ski->alloc, s),
      vec(ski->alloc, s), Vb(ski->alloc, s), yb(ski->alloc, s), fw(ski->alloc, s), symb(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  const bool conv = sizeof(T) != sizeof(double);
  if (!stb.get(sizeof(LanczosState)) || !cgb.get(sizeof(LanczosState)) || !gmb.get(sizeof(GmresState)) ||
      !part.get(sizeof(double2) * (size_t)max_grid * (GM_R + 2)) || !Gb.get(sizeof(double) * 7 * m) ||
      !vec.get(sizeof(double) * (6 * m + m_pad)) || !Vb.get(sizeof(double) * m_pad * (GM_R + 1)) ||
      (conv && !yb.get(sizeof(double) * std::max<int64_t>(n, 1))) || !fw.get(std::max<size_t>(fwb, 16)) ||
      !symb.get(sizeof(double) * (kp.N + 8)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();   // Arnoldi state (tile kernels)
  LanczosState* cg = cgb.as<LanczosState>();   // |y|^2 and the stopping threshold
  GmresState* gm = gmb.as<GmresState>();
  double* v = vec.as<double>();
  double *b = v, *r = v + m, *z = v + 2 * m, *pv = v + 3 * m, *kv = v + 4 * m, *u = v + 5 * m, *yv = v + 6 * m;
  double* V = Vb.as<double>();
  double* sym = symb.as<double>();
  double* bhat = sym + kp.N;
  double2* pp = part.as<double2>();
  const int sblocks = (int)std::min<int64_t>((m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  const int mblocks = (int)std::min<int64_t>(ceil_div(m_pad, 256), 1024);
  const int nblocks = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), 1024);
  FftPlan pplan = kp;   // the same transform with the spectrum of P (never the dense form)
  pplan.lam_d = sym;
  pplan.col2 = pplan.coldl2 = nullptr;
  auto kmul = [&](const double* in, double* out) -> love_status {
    return kuu_apply<double>(gh, ski->fft, in, out, 1, m, fw.p, -1, s);
  };
  auto pmul = [&](const double* in, double* out) -> love_status {
    return kuu_apply<double>(gh, &pplan, in, out, 1, m, fw.p, -1, s);
  };
  LOVE_CUDA(cudaMemsetAsync(gm, 0, sizeof(GmresState), s));
  LOVE_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * m, s));
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(cg, 1, 0.0);
  LOVE_COUNT_LAUNCH(); k_gram_band<T, 1><<<sblocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Gb.as<double>());
  LOVE_COUNT_LAUNCH(); k_pcg_stencil<<<1, 256, 0, s>>>(Gb.as<double>(), m, bhat);
  LOVE_LAUNCH_CHECK();
  {
    // more than 10 % of the interior nearly empty: leave the solve to the CG
    double empty = 1.0;
    LOVE_CUDA(cudaMemcpyAsync(&empty, bhat + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (!(empty <= 0.1)) {
      *iters = 0;
      return LOVE_OK;
    }
  }
  LOVE_COUNT_LAUNCH();
  k_pcg_symbol<<<ceil_div(kp.N, 256), 256, 0, s>>>((const double*)kp.lam_d, kp.N, bhat, gh.noise, sym, &gm->lk_bits);
  const double* yd = conv ? yb.as<double>() : (const double*)ski->ys;
  LOVE_COUNT_LAUNCH();
  k_mcg_ynorm<T><<<nblocks, 256, 0, s>>>(n, (const T*)ski->ys, conv ? yb.as<double>() : nullptr, tol, gh.noise, pp, cg);
  LOVE_COUNT_LAUNCH(); k_gm_target<<<1, 1, 0, s>>>(gm, cg);
  LOVE_LAUNCH_CHECK();
  LOVE_TRY(scatter_any<T, double>(ski, yd, nullptr, 1.0, b, s));
  LOVE_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  TileArgs<double> ta{};
  ta.n_pad = m_pad;
  ta.kcols = GM_R + 1;
  ta.bc = bc;
  ta.Q = V;
  ta.ldq = m_pad;
  ta.y = yv;
  ta.partial = pp;
  ta.st = st;
  ta.status = ski->status;
  const int nb = std::min(4 * num_sms(), ceil_div(m_pad, 256));
  int total = 0;
  for (int cycle = 0; total < max_iter; ++cycle) {
    LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, GM_R, 1e-14);
    LOVE_COUNT_LAUNCH(); k_gm_start<<<mblocks, 256, 0, s>>>(m, m_pad, r, V, pp, st, gm, ski->status);
    LOVE_LAUNCH_CHECK();
    const int steps = std::min(GM_R, max_iter - total);
    for (int j = 0; j < steps; ++j) {
      double* vj = V + (int64_t)j * m_pad;
      LOVE_COUNT_LAUNCH(); k_normalize_col<double><<<nb, 256, 0, s>>>(vj, m_pad, st->scal + j, st);
      LOVE_TRY(pmul(vj, pv));
      LOVE_TRY(kmul(pv, kv));
      LOVE_COUNT_LAUNCH(); k_gm_band<<<mblocks, 256, 0, s>>>(m, m_pad, Gb.as<double>(), kv, pv, gh.noise, yv, st);
      LOVE_LAUNCH_CHECK();
      ta.j = j;
      LOVE_TRY(reorth_sweep<double, MODE_DOT>(ta, s));
      LOVE_TRY(reorth_sweep<double, MODE_UPDATE_DOT>(ta, s));
      LOVE_TRY(reorth_sweep<double, MODE_UPDATE_NORM>(ta, s));
      LOVE_COUNT_LAUNCH(); k_gm_givens<<<1, 1, 0, s>>>(st, gm, j, ski->status);
      LOVE_LAUNCH_CHECK();
      if (j % 6 == 5) {   // stop launching once the cycle has converged
        int done = 0;
        LOVE_CUDA(cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        LOVE_CUDA(cudaStreamSynchronize(s));
        if (done) break;
      }
    }
    // z += P V y; a = K z
    LOVE_COUNT_LAUNCH(); k_gm_solve<<<1, 1, 0, s>>>(gm);
    LOVE_COUNT_LAUNCH(); k_gm_combine<<<mblocks, 256, 0, s>>>(m, V, m_pad, gm, u);
    LOVE_TRY(pmul(u, pv));
    LOVE_COUNT_LAUNCH(); k_gm_add<<<mblocks, 256, 0, s>>>(m, z, pv);
    LOVE_TRY(kmul(z, a));
    LOVE_LAUNCH_CHECK();
    int hs[2] = {0, 0};   // columns, converged
    LOVE_CUDA(cudaMemcpyAsync(&hs[0], &gm->ncols, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaMemcpyAsync(&hs[1], &gm->converged, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    total += hs[0];
    if (hs[1]) *converged = true;
    if (hs[1] || hs[0] == 0) break;   // converged, or no progress possible
    // restart from the recomputed residual r = b - A z
    LOVE_COUNT_LAUNCH(); k_gm_resid<<<mblocks, 256, 0, s>>>(m, Gb.as<double>(), a, z, b, gh.noise, r);
    LOVE_LAUNCH_CHECK();
  }
  if (iters) *iters = total;
  return LOVE_OK;
}

template love_status mean_grid_gmres<float>(love_ski*, double, int, double*, int*, bool*, cudaStream_t);
template love_status mean_grid_gmres<double>(love_ski*, double, int, double*, int*, bool*, cudaStream_t);
template love_status cg_solve<float>(love_ski*, const float*, double*, double, int, int*, cudaStream_t);
template love_status cg_solve<double>(love_ski*, const double*, double*, double, int, int*, cudaStream_t);

}  // namespace love
