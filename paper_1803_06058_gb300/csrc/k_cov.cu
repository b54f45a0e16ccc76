// k_cov.cu -- posterior cross-covariances between two sets of test points
// (Sec. 3, eq. pred_covar_ski_fast with i != j; Algorithm 1 with two sets):
//   cov[i, j] = p(x1_i, x2_j) - (Rt^T w1_i) . (Rt^T w2_j)
// p = w1^T K_UU w2 (the SKI prior; the kernel factorises over dimensions into
// 4 x 4 quadratic forms with the Toeplitz columns of K_UU) or, with
// LOVE_PRIOR_EXACT, outputscale * k(x1_i, x2_j).
//
//   k_cov_gather   warp per point: v = Rt^T w (lanes over columns, 4^d rows
//                  of the packed cache) and the point's stencil (base, weights)
//   k_cov_gemm_tc05  FP32 data: V2 V1^T on the 5th-generation tensor cores
//                  (tcgen05 kind::tf32, each operand split in two TF32 parts,
//                  as the sample GEMM; accumulator in tensor memory), the prior
//                  and the subtraction in FP64 in the epilogue
//   k_cov_gemm     FP64 data: the same product in FP64 on the SIMT pipes
#include <type_traits>
#include <utility>
#include <vector>

#include "love_internal.cuh"
#include "umma.cuh"

namespace love {
namespace {

template <typename CT, typename R>
__device__ __forceinline__ R cload(const void* Rc, int64_t idx) {
  if constexpr (std::is_same<CT, __nv_bfloat16>::value)
    return (R)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Rc)[idx]);
  else
    return (R)reinterpret_cast<const CT*>(Rc)[idx];
}

struct CovPts {
  const void* x;     // t x D (data dtype)
  int64_t t;
  void* V;           // t x ldv (data dtype)
  int* base;         // t x D (-1: the stencil leaves the grid)
  void* w;           // t x D x 4 (data dtype)
};

template <typename CT, typename R, int D>
__global__ void k_cov_gather(GridDev g, const void* __restrict__ Rc, int ld, int k, int ldv, CovPts P,
                             DevStatus* status) {
  const int lane = threadIdx.x & 31;
  const int64_t wp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const R* x = reinterpret_cast<const R*>(P.x);
  R* V = reinterpret_cast<R*>(P.V);
  R* W = reinterpret_cast<R*>(P.w);
  for (int64_t pt = wp; pt < P.t; pt += nw) {
    int base[D];
    R w[D][4];
    bool ok = true;
#pragma unroll
    for (int e = 0; e < D; ++e) ok &= keys_weights(grid_coord(x[pt * D + e], g, e), g.g[e], base[e], w[e]);
    if (lane == 0) {
#pragma unroll
      for (int e = 0; e < D; ++e) {
        P.base[pt * D + e] = ok ? base[e] : -1;
#pragma unroll
        for (int r = 0; r < 4; ++r) W[(pt * D + e) * 4 + r] = w[e][r];
      }
      if (!ok) {
        atomicAdd(&status->domain_errors, 1ull);
        dev_flag(status, LOVE_ERR_DOMAIN);
      }
    }
    for (int c = lane; c < ldv; c += 32) {
      R acc = R(0);
      if (ok && c < k) {
        for (int q = 0; q < (1 << (2 * D)); ++q) {
          const int r0 = q & 3, r1 = (q >> 2) & 3, r2 = (q >> 4) & 3;
          int64_t row;
          R wq;
          if (D == 1) {
            row = base[0] - 1 + r0;
            wq = w[0][r0];
          } else if (D == 2) {
            row = (int64_t)(base[0] - 1 + r1) * g.stride[0] + (base[D - 1] - 1 + r0);
            wq = w[0][r1] * w[D - 1][r0];
          } else {
            row = (int64_t)(base[0] - 1 + r2) * g.stride[0] + (int64_t)(base[1 % D] - 1 + r1) * g.stride[1] +
                  (base[D - 1] - 1 + r0);
            wq = w[0][r2] * w[1 % D][r1] * w[D - 1][r0];
          }
          acc = fma(wq, cload<CT, R>(Rc, row * ld + c), acc);
        }
      }
      V[pt * ldv + c] = acc;
    }
  }
}

// first Toeplitz columns of the factors, FP64, outputscale folded into dim 0
__global__ void k_cov_columns(double* col, int64_t total, GridDev g, double sf, double l0, double l1, double l2) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= total) return;
  int e = 0;
  int64_t r = j;
  while (e < g.dim - 1 && r >= g.g[e]) {
    r -= g.g[e];
    ++e;
  }
  const double ls = e == 0 ? l0 : (e == 1 ? l1 : l2);
  const double d = (double)r * g.h_d[e];
  col[j] = (e == 0 ? sf : 1.0) * exp(-(d * d) / (2.0 * ls * ls));
}

struct CovPrior {
  GridDev g;
  const double* col;     // concatenated Toeplitz columns (dim 0, then 1, 2)
  int64_t coff[3];       // offset of each dimension's column
  int exact;
  double sf;
  double inv2l2[3];      // 1 / (2 l_e^2)
};

// p(i, j): SKI prior from the two stencils, or the exact kernel at the points
template <typename R, int D>
__device__ __forceinline__ double cov_prior(const CovPrior& cp, const R* x1, const int* b1, const R* w1,
                                            const R* x2, const int* b2, const R* w2) {
  if (cp.exact) {
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      const double d = (double)x1[e] - (double)x2[e];
      s += d * d * cp.inv2l2[e];
    }
    return cp.sf * exp(-s);
  }
  double p = 1.0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const int d0 = b1[e] - b2[e];
    const double* col = cp.col + cp.coff[e];
    double q = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double a = 0.0;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        int o = d0 + r - s;
        o = o < 0 ? -o : o;
        a = fma((double)w2[e * 4 + s], col[o], a);
      }
      q = fma((double)w1[e * 4 + r], a, q);
    }
    p *= q;
  }
  return p;
}

template <typename R, int D>
__device__ __forceinline__ void cov_store(const CovPrior& cp, const CovPts& A, const CovPts& B, int64_t i, int64_t j,
                                          double dot, R* __restrict__ out) {
  const int* b1 = A.base + i * D;
  const int* b2 = B.base + j * D;
  R v;
  if (b1[0] < 0 || b2[0] < 0) {
    v = R(NAN);
  } else {
    const R* x1 = reinterpret_cast<const R*>(A.x) + i * D;
    const R* x2 = reinterpret_cast<const R*>(B.x) + j * D;
    const double p = cov_prior<R, D>(cp, x1, b1, reinterpret_cast<const R*>(A.w) + i * D * 4, x2, b2,
                                     reinterpret_cast<const R*>(B.w) + j * D * 4);
    v = (R)(p - dot);
  }
  out[i * B.t + j] = v;
}

// ---- FP32: V2 V1^T on the tensor cores (tcgen05), split TF32 ----
// A CTA computes 128 points of set 2 (tensor-memory lanes: A = V2 rows) by
// 128 points of set 1 (accumulator columns: B = V1 rows), K chunks through two
// shared-memory buffers with the next chunk's loads held in registers, one
// thread issuing the MMAs and committing them to the buffer's mbarrier.  In
// the epilogue lane j and column i give cov[i][j] (consecutive j per store).
template <int D>
__global__ void __launch_bounds__(256, 1) k_cov_gemm_tc05(CovPts A, CovPts B, int k, int ldv, CovPrior cp,
                                                           float* __restrict__ out, DevStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 8 * (size_t)U_TILE_BYTES);   // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  const float* V1 = reinterpret_cast<const float*>(A.V);
  const float* V2 = reinterpret_cast<const float*>(B.V);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * UM;   // set 2 (lanes)
  const int64_t i0 = (int64_t)blockIdx.y * UN;   // set 1 (columns)
  if (warp == 0) tmem_alloc_warp(tmem_slot, UN);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  uint32_t uses[2] = {0u, 0u};
  RowTileRegs ra, rb;
  ra.load(V2, ldv, j0, B.t, 0, k, tid);
  rb.load(V1, ldv, i0, A.t, 0, k, tid);
  int chunk = 0;
  for (int c0 = 0; c0 < k; c0 += UKC, ++chunk) {
    const int b = chunk & 1;
    unsigned char* Ahi = smem_raw + (size_t)b * 4 * U_TILE_BYTES;
    unsigned char* Alo = Ahi + U_TILE_BYTES;
    unsigned char* Bhi = Alo + U_TILE_BYTES;
    unsigned char* Blo = Bhi + U_TILE_BYTES;
    if (uses[b] > 0) {
      ok = ok && mbar_wait_bounded(&bar[b], (uses[b] - 1u) & 1u);
      if (__syncthreads_or(!ok)) break;
    }
    const int kc = min(UKC, (k - c0 + 7) & ~7);
    ra.store(Ahi, Alo, kc, tid);
    rb.store(Bhi, Blo, kc, tid);
    if (c0 + UKC < k) {
      ra.load(V2, ldv, j0, B.t, c0 + UKC, k, tid);
      rb.load(V1, ldv, i0, A.t, c0 + UKC, k, tid);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      umma_chunk(tmem, Ahi, Alo, Bhi, Blo, kc, c0 == 0);
      umma_commit(&bar[b]);
    }
    uses[b] += 1u;
  }
  if (ok && chunk > 0) {
    const int b = (chunk - 1) & 1;
    ok = mbar_wait_bounded(&bar[b], (uses[b] - 1u) & 1u);
    ok = !__syncthreads_or(!ok);
  }
  tc_fence_after();
  if (ok) {
    const int lb = 32 * (warp & 3), cb = 64 * (warp >> 2);
    const int64_t j = j0 + lb + lane;
#pragma unroll 1
    for (int c = 0; c < 64; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)(cb + c), v);
      if (j < B.t) {
        for (int q = 0; q < 16; ++q) {
          const int64_t i = i0 + cb + c + q;
          if (i < A.t) cov_store<float, D>(cp, A, B, i, j, (double)v[q], out);
        }
      }
    }
  } else if (tid == 0) {
    dev_flag(status, LOVE_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc_warp(tmem, UN);
  }
}

// ---- FP64: SIMT tiles of 64 x 64, 4 x 4 per thread ----
template <int D>
__global__ void __launch_bounds__(256) k_cov_gemm(CovPts A, CovPts B, int k, int ldv, CovPrior cp,
                                                  double* __restrict__ out) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const double* V1 = reinterpret_cast<const double*>(A.V);
  const double* V2 = reinterpret_cast<const double*>(B.V);
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  const int64_t j0 = (int64_t)blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int c0 = 0; c0 < k; c0 += 16) {
    for (int idx = threadIdx.x; idx < 64 * 16; idx += 256) {
      const int ii = idx >> 4, cc = idx & 15;
      const int64_t i = i0 + ii, j = j0 + ii;
      As[cc][ii] = (i < A.t && c0 + cc < k) ? V1[i * ldv + c0 + cc] : 0.0;
      Bs[cc][ii] = (j < B.t && c0 + cc < k) ? V2[j * ldv + c0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[cc][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[cc][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + tx + 16 * a;
    if (i >= A.t) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = j0 + ty + 16 * b;
      if (j < B.t) cov_store<double, D>(cp, A, B, i, j, acc[a][b], out);
    }
  }
}

template <typename CT, typename R>
love_status gather_any(const love_cache* c, int ldv, CovPts& P, cudaStream_t s) {
  const GridDev g = c->grid.dev();
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((P.t * 32 + 255) / 256, (int64_t)num_sms() * 16));
  switch (g.dim) {
    case 1: LOVE_COUNT_LAUNCH(); k_cov_gather<CT, R, 1><<<blocks, 256, 0, s>>>(g, c->Rc, c->ld, c->k_eff, ldv, P, c->status); break;
    case 2: LOVE_COUNT_LAUNCH(); k_cov_gather<CT, R, 2><<<blocks, 256, 0, s>>>(g, c->Rc, c->ld, c->k_eff, ldv, P, c->status); break;
    default: LOVE_COUNT_LAUNCH(); k_cov_gather<CT, R, 3><<<blocks, 256, 0, s>>>(g, c->Rc, c->ld, c->k_eff, ldv, P, c->status);
  }
  return cuda_check(cudaGetLastError());
}

struct Tmp {
  const Allocator& al;
  cudaStream_t s;
  std::vector<std::pair<void*, size_t>> bufs;
  Tmp(const Allocator& a, cudaStream_t st) : al(a), s(st) {}
  void* get(size_t b) {
    void* p = al.alloc(b, s);
    if (p) bufs.push_back({p, b});
    return p;
  }
  ~Tmp() {
    for (auto& b : bufs) al.free(b.first, b.second, s);
  }
};

}  // namespace

love_status cov_launch(love_cache* c, int64_t t1, const void* x1, int64_t t2, const void* x2, void* out,
                       cudaStream_t s) {
  if (t1 == 0 || t2 == 0) return LOVE_OK;
  const bool dbl = c->dtype == LOVE_F64;
  const size_t el = dbl ? 8 : 4;
  const int D = c->grid.dim;
  const int k = c->k_eff;
  const int ldv = (k + 3) / 4 * 4;
  Tmp tmp(c->alloc, s);
  CovPts A{x1, t1, tmp.get(el * (size_t)t1 * ldv), (int*)tmp.get(sizeof(int) * (size_t)t1 * D),
           tmp.get(el * (size_t)t1 * D * 4)};
  CovPts B{x2, t2, tmp.get(el * (size_t)t2 * ldv), (int*)tmp.get(sizeof(int) * (size_t)t2 * D),
           tmp.get(el * (size_t)t2 * D * 4)};
  CovPrior cp{};
  cp.g = c->grid.dev();
  int64_t tot = 0;
  for (int e = 0; e < D; ++e) {
    cp.coff[e] = tot;
    tot += c->grid.g[e];
  }
  double* col = (double*)tmp.get(sizeof(double) * (size_t)tot);
  if (!A.V || !A.base || !A.w || !B.V || !B.base || !B.w || !col) return LOVE_ERR_OOM;
  cp.col = col;
  cp.exact = (c->flags & LOVE_PRIOR_EXACT) ? 1 : 0;
  cp.sf = c->grid.sf;
  for (int e = 0; e < 3; ++e) cp.inv2l2[e] = e < D ? 1.0 / (2.0 * c->grid.ls[e] * c->grid.ls[e]) : 0.0;
  LOVE_COUNT_LAUNCH();
  k_cov_columns<<<ceil_div(tot, 256), 256, 0, s>>>(col, tot, cp.g, c->grid.sf, c->grid.ls[0], c->grid.ls[1],
                                                   c->grid.ls[2]);
  LOVE_TRY(cuda_check(cudaGetLastError()));
  if (dbl) {
    LOVE_TRY((gather_any<double, double>(c, ldv, A, s)));
    LOVE_TRY((gather_any<double, double>(c, ldv, B, s)));
    dim3 grid((unsigned)((t1 + 63) / 64), (unsigned)((t2 + 63) / 64));
    LOVE_COUNT_LAUNCH();
    if (D == 1) k_cov_gemm<1><<<grid, 256, 0, s>>>(A, B, k, ldv, cp, (double*)out);
    else if (D == 2) k_cov_gemm<2><<<grid, 256, 0, s>>>(A, B, k, ldv, cp, (double*)out);
    else k_cov_gemm<3><<<grid, 256, 0, s>>>(A, B, k, ldv, cp, (double*)out);
  } else {
    if (c->cache_dtype == LOVE_BF16) {
      LOVE_TRY((gather_any<__nv_bfloat16, float>(c, ldv, A, s)));
      LOVE_TRY((gather_any<__nv_bfloat16, float>(c, ldv, B, s)));
    } else {
      LOVE_TRY((gather_any<float, float>(c, ldv, A, s)));
      LOVE_TRY((gather_any<float, float>(c, ldv, B, s)));
    }
    dim3 g5((unsigned)((t2 + UM - 1) / UM), (unsigned)((t1 + UN - 1) / UN));
    if (D == 1) {
      LOVE_TRY(allow_smem(k_cov_gemm_tc05<1>, U_SMEM));
      LOVE_COUNT_LAUNCH(); k_cov_gemm_tc05<1><<<g5, 256, U_SMEM, s>>>(A, B, k, ldv, cp, (float*)out, c->status);
    } else if (D == 2) {
      LOVE_TRY(allow_smem(k_cov_gemm_tc05<2>, U_SMEM));
      LOVE_COUNT_LAUNCH(); k_cov_gemm_tc05<2><<<g5, 256, U_SMEM, s>>>(A, B, k, ldv, cp, (float*)out, c->status);
    } else {
      LOVE_TRY(allow_smem(k_cov_gemm_tc05<3>, U_SMEM));
      LOVE_COUNT_LAUNCH(); k_cov_gemm_tc05<3><<<g5, 256, U_SMEM, s>>>(A, B, k, ldv, cp, (float*)out, c->status);
    }
  }
  return cuda_check(cudaGetLastError());
}

}  // namespace love
