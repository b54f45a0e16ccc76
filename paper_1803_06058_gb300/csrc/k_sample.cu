// k_sample.cu -- posterior sampling through the low-rank root (Sec. 3.3).
//
// Pre-compute (eqs. lancapprox, sampling_pre_cholesky, pred_covar_ski_interp_form):
// k' Lanczos steps on M = K_UU - R^T R' (k_lanczos.cu: sampler_lanczos) give
// Q', T' (FP64 vectors); with T' = L' L'^T the root is S = Q' L' (m x k'),
// rounded once to the data dtype.  When T' is not positive definite (M is a
// difference of two nearly equal PSD matrices, so rounding can push small
// eigenvalues below zero) the root is that of T''s positive part, from the
// eigendecomposition T' = V diag(lam) V^T: S = Q' V diag(sqrt(max(lam, 0))),
// with the eigenpairs from cyclic Jacobi rotations (Golub & Van Loan, Sec. 8.5).
// For an FP64 root, whose T' is indefinite only at the rounding level, the
// Cholesky factor of T' + delta I (delta = -lambda_min(T') plus rounding, from
// Sturm-count multisection) is taken first: it differs from the positive part by
// that rounding; the eigen route remains its last resort.
//
// Test phase (eq. sample): F = mu 1^T + (W*^T S Z)^T, F sample-major (s x t):
//   gather   G = W*^T S (t x k') and mu = W*^T a     (4^d rows of S per point)
//   product  F[j, i] = mu_i + sum_c G[i, c] Z[c, j]
// Z (k' x s) is supplied by the caller or drawn on the device from
// Philox4x32-10 (Salmon et al. 2011) with Box-Muller in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include <type_traits>

#include "love_internal.cuh"
#include "umma.cuh"

namespace love {
namespace {


// l_11 = sqrt(alpha_1), e_j = beta_j / l_jj, l_{j+1,j+1} = sqrt(alpha_{j+1} - e_j^2)
__global__ void k_chol_tri(const double* alpha, const double* beta, int k, double* d, double* e, int* ok) {
  if (threadIdx.x || blockIdx.x) return;
  double piv = alpha[0];
  *ok = 1;
  for (int j = 0; j < k; ++j) {
    if (j > 0) {
      e[j - 1] = beta[j - 1] / d[j - 1];
      piv = alpha[j] - e[j - 1] * e[j - 1];
    }
    if (!(piv > 0.0)) {
      *ok = 0;
      return;
    }
    d[j] = sqrt(piv);
  }
}

// T' + delta I for a T' that is not numerically positive definite: the
// smallest eigenvalue of the tridiagonal T' by multisection on Sturm counts
// (the number of negative pivots of the LDL^T factorisation of T' - x I is the
// number of eigenvalues below x), then delta = max(0, -lo) plus 16 units of
// rounding of |T'|, lo the lower end of the final bracket of lambda_min (so
// delta >= -lambda_min: the Cholesky factorisation of the shifted matrix
// succeeds, and delta exceeds -lambda_min by at most the bracket's width);
// alpha_s = alpha + delta.  Used for an FP64 root only (T' indefinite at the
// rounding level).  One CTA: each round its threads count at as many interior
// points of the bracket, and the bracket shrinks to the cell holding
// lambda_min until its width is rel_res |T'| (FP64 resolution).  The counts are FP64 divisions, which
// this part runs at a small fraction of its FP32 rate, so a round costs in
// proportion to the warps per SM sub-partition: it is launched with four warps
// (128 points, 7 bits of the bracket per round).
__device__ int sturm_below(const double* alpha, const double* beta, int k, double x) {
  const double tiny = 1e-300;
  int neg = 0;
  double dd = alpha[0] - x;
  for (int j = 0;;) {
    if (fabs(dd) < tiny) dd = -tiny;
    if (dd < 0.0) ++neg;
    if (++j == k) break;
    dd = alpha[j] - x - beta[j - 1] * beta[j - 1] / dd;
  }
  return neg;
}

__global__ void k_tri_shift(const double* alpha, const double* beta, int k, double* alpha_s, double rel_res) {
  __shared__ double br[2];
  __shared__ int first;
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) {
    double lo = 0.0, hi = 0.0;
    for (int j = 0; j < k; ++j) {   // Gershgorin interval
      const double r = (j > 0 ? fabs(beta[j - 1]) : 0.0) + (j + 1 < k ? fabs(beta[j]) : 0.0);
      lo = j == 0 ? alpha[j] - r : fmin(lo, alpha[j] - r);
      hi = j == 0 ? alpha[j] + r : fmax(hi, alpha[j] + r);
    }
    br[0] = lo;
    br[1] = hi;
  }
  __syncthreads();
  const double nrm = fmax(fabs(br[0]), fabs(br[1]));
  for (int round = 0; round < 12; ++round) {
    const double a = br[0], b = br[1];
    if (!(b - a > rel_res * nrm)) break;
    if (t == 0) first = nt;
    __syncthreads();
    const double x = a + (b - a) * (double)(t + 1) / (double)(nt + 1);
    if (sturm_below(alpha, beta, k, x) >= 1) atomicMin(&first, t);
    __syncthreads();
    if (t == 0) {
      const double h = (b - a) / (double)(nt + 1);
      br[0] = first == 0 ? a : a + h * (double)first;
      br[1] = first == nt ? b : a + h * (double)(first + 1);
    }
    __syncthreads();
  }
  const double delta = fmax(0.0, -br[0]) + 16.0 * 2.2204460492503131e-16 * nrm;
  for (int j = t; j < k; j += nt) alpha_s[j] = alpha[j] + delta;
}

// S[r, c] = d_c Q'[r, c] + e_c Q'[r, c+1]   (S = Q' L', L' lower bidiagonal), row-major ld_s;
// Q' in FP64, S rounded once to T
template <typename T>
__global__ void k_root_from_chol(const double* __restrict__ Q, int64_t ldq, int64_t m, int k, const double* d,
                                 const double* e, T* __restrict__ S, int ld_s) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * ld_s) return;
  int64_t r = idx / ld_s;
  int c = (int)(idx - r * ld_s);
  double v = 0.0;
  if (c < k) {
    v = d[c] * Q[(int64_t)c * ldq + r];
    if (c + 1 < k) v += e[c] * Q[(int64_t)(c + 1) * ldq + r];
  }
  S[idx] = (T)v;
}

// Eigenpairs of the symmetric tridiagonal T' (n <= 200) for the positive-part
// root, one warp per eigenvalue (ascending index i):
//   1  lam_i to ~2^-24 |T'| by multisection on FP32 Sturm counts (the number of
//      negative pivots of the LDL^T factorisation of T' - x I is the number of
//      eigenvalues below x): each round the 32 lanes count at 32 interior points
//      of the bracket, which shrinks to the cell holding lam_i;
//   2  inverse iteration in FP64 with that shift: LU of T' - lam I with partial
//      pivoting (row swaps give U a second superdiagonal), INVIT solves,
//      normalised each time (Golub & Van Loan, Sec. 8.2.2); the shift's error e
//      shrinks the neighbours' components by e / gap per solve.  The start
//      vector differs per index (1 + a SplitMix64 draw in [-1/2, 1/2) per entry),
//      so eigenvalues too close for FP32 to separate, which share a shift, still
//      give independent vectors of their common invariant subspace;
//   3  lam_i = x^T T' x (FP64 Rayleigh quotient).
// V[r * n + i] = x_r (eigenvectors in columns), lam[i].
constexpr int INVIT = 4;
__device__ int sturm_count_f(const float* a, const float* b2, int n, float x) {
  int neg = 0;
  float d = a[0] - x;
  for (int j = 0;;) {
    if (fabsf(d) < 1e-37f) d = -1e-37f;
    if (d < 0.f) ++neg;
    if (++j == n) break;
    d = (a[j] - x) - b2[j - 1] / d;
  }
  return neg;
}

__global__ void __launch_bounds__(32) k_tri_eigpairs(const double* __restrict__ alpha, const double* __restrict__ beta,
                                                     int n, double* __restrict__ lam, double* __restrict__ V) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* u0 = reinterpret_cast<double*>(smem_raw);   // pivots
  double* u1 = u0 + n;                                 // first superdiagonal of U
  double* u2 = u1 + n;                                 // second superdiagonal (after swaps)
  double* ml = u2 + n;                                 // multipliers
  double* xv = ml + n;                                 // iterate
  float* af = reinterpret_cast<float*>(xv + n);        // T' diagonal (FP32)
  float* b2f = af + n;                                 // squared off-diagonal (FP32)
  int* swp = reinterpret_cast<int*>(b2f + n);          // row swap at elimination step j
  const int i = blockIdx.x, lane = threadIdx.x;
  for (int j = lane; j < n; j += 32) {
    af[j] = (float)alpha[j];
    if (j + 1 < n) b2f[j] = (float)(beta[j] * beta[j]);
  }
  __syncwarp();
  // Gershgorin interval (every lane the same)
  double lo = 0.0, hi = 0.0, tn = 0.0;
  for (int j = 0; j < n; ++j) {
    const double r = (j > 0 ? fabs(beta[j - 1]) : 0.0) + (j + 1 < n ? fabs(beta[j]) : 0.0);
    lo = j == 0 ? alpha[j] - r : fmin(lo, alpha[j] - r);
    hi = j == 0 ? alpha[j] + r : fmax(hi, alpha[j] + r);
  }
  tn = fmax(fabs(lo), fabs(hi));
  float flo = (float)lo - 1e-6f * (float)tn, fhi = (float)hi + 1e-6f * (float)tn;
  for (int round = 0; round < 8; ++round) {
    const float w = fhi - flo;
    if (!(w > 2.4e-7f * (float)tn)) break;
    const float x = flo + w * (float)(lane + 1) / 33.f;
    const bool above = sturm_count_f(af, b2f, n, x) >= i + 1;
    const unsigned bal = __ballot_sync(0xffffffffu, above);
    const int f = bal ? __ffs(bal) - 1 : 32;   // first point with >= i + 1 eigenvalues below it
    const float nlo = f == 0 ? flo : flo + w * (float)f / 33.f;
    const float nhi = f == 32 ? fhi : flo + w * (float)(f + 1) / 33.f;
    flo = nlo;
    fhi = nhi;
  }
  const double shift = 0.5 * ((double)flo + (double)fhi);
  // LU with partial pivoting of T' - shift I (lane 0; tridiagonal, so O(n))
  if (lane == 0) {
    const double tiny = 2.2204460492503131e-16 * fmax(tn, 1e-300);
    double d = alpha[0] - shift, e = n > 1 ? beta[0] : 0.0, g = 0.0;   // current row: (d, e, g) at cols j, j+1, j+2
    for (int j = 0; j < n - 1; ++j) {
      const double bl = beta[j];                  // T'[j+1, j]
      const double an = alpha[j + 1] - shift;     // T'[j+1, j+1]
      const double cn = j + 2 < n ? beta[j + 1] : 0.0;
      if (fabs(bl) > fabs(d)) {                   // swap rows j and j+1
        const double mlt = d / bl;
        u0[j] = bl;
        u1[j] = an;
        u2[j] = cn;
        ml[j] = mlt;
        swp[j] = 1;
        d = e - mlt * an;
        e = g - mlt * cn;
        g = 0.0;
      } else {
        const double piv = d == 0.0 ? tiny : d;
        const double mlt = bl / piv;
        u0[j] = piv;
        u1[j] = e;
        u2[j] = g;
        ml[j] = mlt;
        swp[j] = 0;
        d = an - mlt * e;
        e = cn - mlt * g;
        g = 0.0;
      }
    }
    u0[n - 1] = d == 0.0 ? tiny : d;
    u1[n - 1] = 0.0;
    u2[n - 1] = 0.0;
    if (n > 1) u2[n - 2] = 0.0;
  }
  for (int j = lane; j < n; j += 32) {
    uint64_t z = (uint64_t)(i * n + j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    xv[j] = 1.0 + ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
  }
  __syncwarp();
  for (int it = 0; it < INVIT; ++it) {
    if (lane == 0) {
      for (int j = 0; j < n - 1; ++j) {           // L^{-1} with the swaps
        if (swp[j]) {
          const double t = xv[j];
          xv[j] = xv[j + 1];
          xv[j + 1] = t;
        }
        xv[j + 1] -= ml[j] * xv[j];
      }
      for (int j = n - 1; j >= 0; --j) {          // U^{-1}
        double r = xv[j];
        if (j + 1 < n) r -= u1[j] * xv[j + 1];
        if (j + 2 < n) r -= u2[j] * xv[j + 2];
        xv[j] = r / u0[j];
      }
    }
    __syncwarp();
    double ss = 0.0;
    for (int j = lane; j < n; j += 32) ss = fma(xv[j], xv[j], ss);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double sc = 1.0 / sqrt(ss);
    for (int j = lane; j < n; j += 32) xv[j] *= sc;
    __syncwarp();
  }
  // Rayleigh quotient and the sign (largest-magnitude entry positive)
  double rq = 0.0, best = -1.0;
  int bi = 0;
  for (int j = lane; j < n; j += 32) {
    double tx = alpha[j] * xv[j];
    if (j > 0) tx += beta[j - 1] * xv[j - 1];
    if (j + 1 < n) tx += beta[j] * xv[j + 1];
    rq = fma(xv[j], tx, rq);
    if (fabs(xv[j]) > best) {
      best = fabs(xv[j]);
      bi = j;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    rq += __shfl_xor_sync(0xffffffffu, rq, o);
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  const double sgn = xv[bi] < 0.0 ? -1.0 : 1.0;
  for (int j = lane; j < n; j += 32) V[(size_t)j * n + i] = sgn * xv[j];
  if (lane == 0) lam[i] = rq;
}

// Vectors whose eigenvalues lie within 1e-3 |T'| of their neighbour (a cluster)
// are made orthonormal by modified Gram-Schmidt in index order, applied twice
// (LAPACK's stein criterion for the clusters); inverse iteration leaves the
// others orthogonal to ~eps |T'| / gap.  A vector that the projections leave
// (numerically) empty lay in the span of its predecessors: a unit vector takes
// its place before the passes are repeated.  One warp per cluster; lam is only
// read (its Rayleigh quotients already hold to the vectors' accuracy squared).
__global__ void __launch_bounds__(256) k_tri_cluster_mgs(int n, const double* __restrict__ lam,
                                                          double* __restrict__ V) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double tn = 0.0;
  for (int j = 0; j < n; ++j) tn = fmax(tn, fabs(lam[j]));
  const double tol = 1e-3 * tn;
  // clusters: maximal runs [c0, c1) of consecutive eigenvalues with gaps < tol
  int cid = 0;
  for (int c0 = 0; c0 < n;) {
    int c1 = c0 + 1;
    while (c1 < n && lam[c1] - lam[c1 - 1] < tol) ++c1;
    if (c1 - c0 > 1 && (cid++ % nw) == w) {
      for (int q = c0 + 1; q < c1; ++q) {
        for (int attempt = 0; attempt < 2; ++attempt) {
          for (int pass = 0; pass < 2; ++pass)
            for (int p = c0; p < q; ++p) {
              double d = 0.0;
              for (int j = lane; j < n; j += 32) d = fma(V[(size_t)j * n + p], V[(size_t)j * n + q], d);
              for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
              for (int j = lane; j < n; j += 32) V[(size_t)j * n + q] -= d * V[(size_t)j * n + p];
              __syncwarp();
            }
          double ss = 0.0;
          for (int j = lane; j < n; j += 32) ss = fma(V[(size_t)j * n + q], V[(size_t)j * n + q], ss);
          for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
          if (ss > 1e-20) {   // the vector had unit norm before the projections
            const double sc = 1.0 / sqrt(ss);
            for (int j = lane; j < n; j += 32) V[(size_t)j * n + q] *= sc;
            __syncwarp();
            break;
          }
          // empty: restart from the unit vector e_(q - c0 + attempt) mod n
          for (int j = lane; j < n; j += 32) V[(size_t)j * n + q] = j == (q - c0 + attempt) % n ? 1.0 : 0.0;
          __syncwarp();
        }
      }
    }
    c0 = c1;
  }
}

// B[j, c] = V[j, c] sqrt(max(lam_c, 0))
__global__ void k_scale_eig(const double* lam, const double* V, int n, double* B) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  int c = (int)(idx % n);
  double l = lam[c];
  B[idx] = V[idx] * sqrt(l > 0.0 ? l : 0.0);
}

// S[r, c] = sum_j Q'[r, j] B[j, c]  (Q' and B in FP64, arithmetic in T; S row-major
// ld_s).  A CTA takes ROOT_ROWS rows, their Q' entries staged in shared memory,
// and B too when it fits (stage_b); thread (rr, cg) forms the columns cg, cg + 4,
// ... of row rr (the 32 lanes of a warp share c: B's entries are broadcasts).
constexpr int ROOT_ROWS = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_root_from_eig(const double* __restrict__ Q, int64_t ldq, int64_t m, int k,
                                                       const double* __restrict__ B, T* __restrict__ S, int ld_s,
                                                       int stage_b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* Qs = reinterpret_cast<T*>(smem_raw);     // k x ROOT_ROWS
  T* Bs = Qs + (size_t)k * ROOT_ROWS;         // k x k when staged
  const int64_t r0 = (int64_t)blockIdx.x * ROOT_ROWS;
  if (stage_b)
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) Bs[i] = (T)B[i];
  for (int i = threadIdx.x; i < k * ROOT_ROWS; i += blockDim.x) {
    const int j = i / ROOT_ROWS, rr = i - j * ROOT_ROWS;
    const int64_t r = r0 + rr;
    Qs[i] = r < m ? (T)Q[(int64_t)j * ldq + r] : T(0);
  }
  __syncthreads();
  const int rr = threadIdx.x % ROOT_ROWS, cg = threadIdx.x / ROOT_ROWS;   // 4 column groups
  const int64_t r = r0 + rr;
  if (r >= m) return;
  for (int c = cg; c < ld_s; c += 4) {
    T acc = T(0);
    if (c < k) {
      if (stage_b)
        for (int j = 0; j < k; ++j) acc += Qs[j * ROOT_ROWS + rr] * Bs[j * k + c];
      else
        for (int j = 0; j < k; ++j) acc += Qs[j * ROOT_ROWS + rr] * (T)__ldg(B + (size_t)j * k + c);
    }
    S[r * ld_s + c] = acc;
  }
}

// ---- test phase -------------------------------------------------------------
struct SampleGatherArgs {
  GridDev g;
  int64_t t;
  const void* x;
  const void* S;
  int ld_s;
  int ks;
  const void* Rc;    // predict cache (mean in column k) or null
  int ld_c;
  int kc;
  int cache_dtype;
  void* G;           // t x ld_g, or null when Gc is given
  int ld_g;
  unsigned char* Gc; // FP32 data: G split into TF32 hi / lo, 128-point canonical tiles (canon_off)
  int kpad;          // columns of a Gc tile (ks rounded up to 8)
  void* mu;          // t
  DevStatus* status;
};

// The FP32 operands of the tensor-core sample product, split and laid out once:
// tile p holds rows 128 p .. 128 p + 127 (points of G, samples of Z^T) as its
// TF32 hi part, then its lo part, each kpad x 128 in the canonical K-major
// no-swizzle layout of umma_off (K slices of 16 bytes 2 KB apart), so a K
// range of a part is one contiguous run of bytes.
__host__ __device__ __forceinline__ size_t canon_tile_bytes(int kpad) { return (size_t)kpad * 1024; }
__device__ __forceinline__ void canon_store(unsigned char* base, int kpad, int64_t row, int k, float v) {
  uint32_t h, l;
  split_tf32(v, h, l);
  unsigned char* tb = base + (size_t)(row >> 7) * canon_tile_bytes(kpad);
  const uint32_t o = umma_off((int)(row & 127), k);
  *reinterpret_cast<uint32_t*>(tb + o) = h;
  *reinterpret_cast<uint32_t*>(tb + (size_t)kpad * 512 + o) = l;
}

template <typename T>
__device__ __forceinline__ T load_cache_elem(const void* Rc, int64_t idx, int cdt) {
  if (cdt == LOVE_BF16) return (T)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Rc)[idx]);
  if (cdt == LOVE_F64) return (T)reinterpret_cast<const double*>(Rc)[idx];
  return (T)reinterpret_cast<const float*>(Rc)[idx];
}

// one warp per test point; lanes over the columns of S
template <typename T, int D>
__global__ void k_sample_gather(SampleGatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const T* x = reinterpret_cast<const T*>(a.x);
  const T* S = reinterpret_cast<const T*>(a.S);
  T* G = reinterpret_cast<T*>(a.G);
  T* mu = reinterpret_cast<T*>(a.mu);
  constexpr int NR = D == 1 ? 4 : (D == 2 ? 16 : 64);
  for (int64_t pt = w0; pt < a.t; pt += nw) {
    int base[D];
    T w[D][4];
    bool ok = true;
#pragma unroll
    for (int e = 0; e < D; ++e) ok &= keys_weights(grid_coord(x[pt * D + e], a.g, e), a.g.g[e], base[e], w[e]);
    if (!ok) {
      if constexpr (std::is_same<T, float>::value) {
        if (a.Gc)
          for (int c = lane; c < a.kpad; c += 32) canon_store(a.Gc, a.kpad, pt, c, 0.f);
      }
      if (G)
        for (int c = lane; c < a.ld_g; c += 32) G[pt * a.ld_g + c] = T(0);
      if (lane == 0) {
        mu[pt] = (T)NAN;
        atomicAdd(&a.status->domain_errors, 1ull);
        dev_flag(a.status, LOVE_ERR_DOMAIN);
      }
      continue;
    }
    int64_t rows[NR];
    T ww[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      int r0 = q & 3, r1 = (q >> 2) & 3, r2 = (q >> 4) & 3;
      int64_t row;
      T wq;
      if (D == 1) {
        row = base[0] - 1 + r0;
        wq = w[0][r0];
      } else if (a.g.additive) {
        // stacked vector: 4 rows per 1-D block, the rest unused
        const int e = q >> 2 < D ? q >> 2 : 0;
        row = q < 4 * D ? (int64_t)a.g.off[e] + base[e] - 1 + (q & 3) : 0;
        wq = q < 4 * D ? w[e][q & 3] : T(0);
      } else if (D == 2) {
        row = (int64_t)(base[0] - 1 + r1) * a.g.stride[0] + (base[1] - 1 + r0);
        wq = w[0][r1] * w[1][r0];
      } else {
        row = (int64_t)(base[0] - 1 + r2) * a.g.stride[0] + (int64_t)(base[1] - 1 + r1) * a.g.stride[1] +
              (base[2] - 1 + r0);
        wq = w[0][r2] * w[1][r1] * w[2][r0];
      }
      rows[q] = row;
      ww[q] = wq;
    }
    const int cend = G ? a.ld_g : a.kpad;
    for (int c = lane; c < cend; c += 32) {
      T acc = T(0);
      if (c < a.ks) {
#pragma unroll
        for (int q = 0; q < NR; ++q) acc += ww[q] * S[rows[q] * a.ld_s + c];
      }
      if (G) {
        G[pt * a.ld_g + c] = acc;
      } else if constexpr (std::is_same<T, float>::value) {
        canon_store(a.Gc, a.kpad, pt, c, acc);
      }
    }
    if (lane == 0) {
      T m_ = T(0);
      if (a.Rc) {
#pragma unroll
        for (int q = 0; q < NR; ++q) m_ += ww[q] * load_cache_elem<T>(a.Rc, rows[q] * a.ld_c + a.kc, a.cache_dtype);
      }
      mu[pt] = m_;
    }
  }
}

// F[j, i] = mu_i + sum_c G[i, c] Z[c, j];  64 x 64 output tile per CTA, 4 x 4 per thread
template <typename T>
__global__ void __launch_bounds__(256) k_sample_gemm(const T* __restrict__ G, int ld_g, const T* __restrict__ Z,
                                                     int s, int ks, const T* __restrict__ mu, int64_t t,
                                                     T* __restrict__ F) {
  __shared__ T Gs[16][64 + 1];
  __shared__ T Zs[16][64];
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  const int j0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int c0 = 0; c0 < ks; c0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = threadIdx.x + 256 * q;
      int ii = idx >> 4, cc = idx & 15;
      int64_t i = i0 + ii;
      Gs[cc][ii] = (i < t && c0 + cc < ks) ? G[i * ld_g + c0 + cc] : T(0);
      int cz = idx >> 6, jj = idx & 63;
      Zs[cz][jj] = (c0 + cz < ks && j0 + jj < s) ? Z[(int64_t)(c0 + cz) * s + j0 + jj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
      T gv[4], zv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) gv[a] = Gs[cc][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) zv[b] = Zs[cc][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(gv[a], zv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int64_t i = i0 + tx + 16 * a;
    if (i >= t) continue;
    T m_ = mu[i];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int j = j0 + ty + 16 * b;
      if (j < s) F[(int64_t)j * t + i] = m_ + acc[a][b];
    }
  }
}

// ---------------------------------------------------------------------------
// The product on the 5th-generation tensor cores (tcgen05, kind::tf32, one
// CTA, accumulator in tensor memory).  A CTA computes a 128-point x 128-sample
// tile D[i][j] = sum_c G[i][c] Z[c][j] from the pre-split canonical tiles of G
// (A, M = points) and Z^T (B, N = samples).  One thread drives a two-stage
// ring of K chunks (SG_KC columns): it issues the four bulk copies of chunk
// c + 1 (the hi and lo parts of both operands: contiguous runs of the
// canonical tiles) before it waits for chunk c, then issues chunk c's MMAs
// (per K step of 8: hi*hi, hi*lo and lo*hi; the lo*lo term, ~2^-22 relative,
// is dropped) into the 128 x 128 FP32 accumulator in tensor memory and commits
// them to the stage's "empty" mbarrier, which the next copy into that stage
// waits on.  The other warps wait (bounded) for the last commit; then the
// epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32 (w mod 4)
// .., columns 64 (w / 4) ..), adds mu and writes F[j][i] (sample-major, 32
// consecutive points per store).  Two CTAs share an SM (96 KB of shared
// memory each), so one CTA's epilogue overlaps the other's copies and MMAs.
constexpr int SG_KC = 24;
constexpr uint32_t SG_PART = SG_KC * 512;              // one operand part of one chunk
constexpr uint32_t SG_STAGE = 4 * SG_PART;             // A hi, A lo, B hi, B lo
constexpr size_t SG_SMEM = 2 * (size_t)SG_STAGE + 64;  // two stages + barriers
__global__ void __launch_bounds__(256, 2) k_sample_gemm_tc05(const unsigned char* __restrict__ Gc,
                                                              const unsigned char* __restrict__ Zc, int kpad, int s,
                                                              const float* __restrict__ mu, int64_t t,
                                                              float* __restrict__ F, DevStatus* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // barriers: full[2] (copies landed), empty[2] (MMAs done with the stage), done
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * (size_t)SG_STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 5);
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * UM;
  const int j0 = blockIdx.y * UN;
  const unsigned char* ga = Gc + (size_t)blockIdx.x * canon_tile_bytes(kpad);
  const unsigned char* zb = Zc + (size_t)blockIdx.y * canon_tile_bytes(kpad);
  const size_t lo_off = (size_t)kpad * 512;
  const int nch = (kpad + SG_KC - 1) / SG_KC;
  if (warp == 0) tmem_alloc_warp(tmem_slot, UN);
  if (tid == 0) {
    for (int q = 0; q < 5; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
    s_ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    auto load = [&](int c) {
      const int st = c & 1, k0 = c * SG_KC;
      const uint32_t pb = (uint32_t)min(SG_KC, kpad - k0) * 512u;
      unsigned char* d = smem_raw + (size_t)st * SG_STAGE;
      mbar_arrive_expect_tx(&bar[st], 4u * pb);
      bulk_g2s(d, ga + (size_t)k0 * 512, pb, &bar[st]);
      bulk_g2s(d + SG_PART, ga + lo_off + (size_t)k0 * 512, pb, &bar[st]);
      bulk_g2s(d + 2 * SG_PART, zb + (size_t)k0 * 512, pb, &bar[st]);
      bulk_g2s(d + 3 * SG_PART, zb + lo_off + (size_t)k0 * 512, pb, &bar[st]);
    };
    bool ok = true;
    int issued = 0;   // chunks whose copies were issued
    int c = 0;        // chunks whose MMAs were issued
    load(0);
    issued = 1;
    for (; c < nch && ok; ++c) {
      const int st = c & 1;
      if (issued < nch) {
        // stage of chunk c + 1: free once chunk c - 1's MMAs completed
        if (c >= 1) ok = mbar_wait_bounded(&bar[2 + (issued & 1)], ((issued >> 1) - 1) & 1u);
        if (!ok) break;
        load(issued);
        ++issued;
      }
      ok = mbar_wait_bounded(&bar[st], (c >> 1) & 1u);
      if (!ok) break;
      tc_fence_after();
      unsigned char* d = smem_raw + (size_t)st * SG_STAGE;
      umma_chunk(tmem, d, d + SG_PART, d + 2 * SG_PART, d + 3 * SG_PART, min(SG_KC, kpad - c * SG_KC), c == 0);
      umma_commit(&bar[2 + st]);
    }
    if (ok) umma_commit(&bar[4]);   // completes when every MMA issued before it has
    if (!ok) {
      s_ok = 0;
      dev_flag(status, LOVE_ERR_TIMEOUT);
      // copies or MMAs that never signalled may still be in flight: give them a
      // bounded last chance before the shared and tensor memory are released
      for (int x = c; x < issued; ++x) mbar_wait_bounded(&bar[x & 1], (x >> 1) & 1u);
      for (int x = c > 2 ? c - 2 : 0; x < c; ++x) mbar_wait_bounded(&bar[2 + (x & 1)], (x >> 1) & 1u);
    }
  }
  __syncthreads();
  bool ok = s_ok != 0;
  if (ok) ok = mbar_wait_bounded(&bar[4], 0u);
  tc_fence_after();
  if (ok) {
    const int lb = 32 * (warp & 3);            // this warp's tensor-memory lanes (points)
    const int cb = 64 * (warp >> 2);           // and its 64 accumulator columns (samples)
    const int64_t i = i0 + lb + lane;
    const float m_ = i < t ? mu[i] : 0.f;
#pragma unroll 1
    for (int c = 0; c < 64; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)(cb + c), v);
      if (i < t) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + cb + c + q;
          if (j < s) F[(int64_t)j * t + i] = m_ + v[q];
        }
      }
    }
  } else if (s_ok) {
    dev_flag(status, LOVE_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc_warp(tmem, UN);
  }
}

// Z (ks x s, row-major) as the split canonical tiles of Z^T: tile p holds
// samples 128 p .. 128 p + 127; zero past ks and past s
__global__ void k_z_canon(const float* __restrict__ Z, int ks, int s, int kpad, int ntiles,
                          unsigned char* __restrict__ Zc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ntiles * kpad * 128) return;
  const int n = (int)(idx & 127);
  const int64_t rest = idx >> 7;
  const int k = (int)(rest % kpad);
  const int64_t tile = rest / kpad;
  const int64_t j = tile * 128 + n;
  const float v = (k < ks && j < s) ? Z[(int64_t)k * s + j] : 0.f;
  canon_store(Zc, kpad, j, k, v);
}

// Philox4x32-10: 10 rounds of (hi0,lo0) = M0 x0, (hi1,lo1) = M1 x2,
// x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0), key += Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * x[0], hi0 = __umulhi(0xD2511F53u, x[0]);
    uint32_t lo1 = 0xCD9E8D57u * x[2], hi1 = __umulhi(0xCD9E8D57u, x[2]);
    uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}
// element e: block e / 4 of counter (lo, hi, 0, 0), key = seed; u = (r + 1/2) 2^-32;
// Box-Muller pairs (r0, r1), (r2, r3): (cos, sin) of each
template <typename T>
__global__ void k_philox_normals(int64_t count, uint64_t seed, T* __restrict__ out) {
  int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk * 4 >= count) return;
  uint32_t x[4] = {(uint32_t)(uint64_t)blk, (uint32_t)((uint64_t)blk >> 32), 0u, 0u};
  philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
  double z[4];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    double u1 = ((double)x[2 * p] + 0.5) * 2.3283064365386963e-10;
    double u2 = ((double)x[2 * p + 1] + 0.5) * 2.3283064365386963e-10;
    double rad = sqrt(-2.0 * log(u1));
    double sn, cn;
    sincospi(2.0 * u2, &sn, &cn);
    z[2 * p] = rad * cn;
    z[2 * p + 1] = rad * sn;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (blk * 4 + q < count) out[blk * 4 + q] = (T)z[q];
}

struct Buf {
  const Allocator* al;
  cudaStream_t s;
  void* p = nullptr;
  size_t b = 0;
  Buf(const Allocator& a, cudaStream_t st) : al(&a), s(st) {}
  bool get(size_t bytes) {
    b = bytes;
    p = scratch_alloc(*al, bytes, s);
    return p != nullptr;
  }
  ~Buf() {
    if (p) scratch_free(*al, p, b, s);
  }
  template <typename X> X* as() const { return (X*)p; }
};

}  // namespace

template <typename T>
love_status sampler_build(const GridHost& g, const FftPlan* fft, const Allocator& al, love_cache* c, const T* Rt,
                          int ks, uint64_t seed, double tau, cudaStream_t s) {
  const int64_t m = g.m;
  const int64_t m_pad = (m + 255) / 256 * 256;
  Buf Qb(al, s), ab(al, s), okb(al, s);
  if (!Qb.get(sizeof(double) * m_pad * ks) || !ab.get(sizeof(double) * 5 * (ks + 1)) || !okb.get(sizeof(int)))
    return LOVE_ERR_OOM;
  std::vector<double> alpha(ks + 1), beta(ks + 1);
  int keff = 0;
  // one persistent launch where the grid allows it (1-D), else the multi-launch run
  love_status lrc = sampler_lanczos_fused<T>(g, fft, al, Rt, m, c->k_eff, ks, seed, tau, Qb.as<double>(), m_pad,
                                             alpha.data(), beta.data(), &keff, c->status, s);
  if (lrc == LOVE_ERR_UNSUPPORTED)
    lrc = sampler_lanczos<T>(g, fft, al, Rt, m, c->k_eff, ks, seed, tau, Qb.as<double>(), m_pad, alpha.data(),
                             beta.data(), &keff, c->status, s);
  LOVE_TRY(lrc);
  if (keff < 1) return LOVE_ERR_NAN;
  double* ad = ab.as<double>();
  double* bd = ad + (ks + 1);
  double* dd = bd + (ks + 1);
  double* ed = dd + (ks + 1);
  LOVE_CUDA(cudaMemcpyAsync(ad, alpha.data(), sizeof(double) * keff, cudaMemcpyHostToDevice, s));
  if (keff > 1) LOVE_CUDA(cudaMemcpyAsync(bd, beta.data(), sizeof(double) * (keff - 1), cudaMemcpyHostToDevice, s));
  LOVE_COUNT_LAUNCH(); k_chol_tri<<<1, 32, 0, s>>>(ad, bd, keff, dd, ed, okb.as<int>());
  LOVE_LAUNCH_CHECK();
  int ok = 0;
  LOVE_CUDA(cudaMemcpyAsync(&ok, okb.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  int shifted = 0;
  // An FP64 root whose T' is not PD is indefinite at the rounding level of K_UU -
  // Rt Rt^T: the shifted Cholesky below differs from the positive part of T' by
  // the size of that rounding.  An FP32 cache's Rt carries FP32 rounding, and
  // K_UU - Rt Rt^T can then be indefinite by a sizeable fraction of |T'| (on the
  // 1-D n = 1e6 workload: 32 negative eigenvalues, the lowest -0.12 |T'|), where a
  // shift would add that much to every direction: the root is the positive part
  // of T' instead (eigen fallback below), as the paper's covariance requires.
  if (!ok && sizeof(T) == 8) {
    // T' not numerically PD (K_UU - Rt Rt^T has eigenvalues at the rounding
    // level): Cholesky of T' + delta I, delta = -lambda_min(T') + rounding
    double* as = ed + (ks + 1);
    const double rel_res = 2.0 * 2.2204460492503131e-16;
    LOVE_COUNT_LAUNCH(); k_tri_shift<<<1, 128, 0, s>>>(ad, bd, keff, as, rel_res);
    LOVE_COUNT_LAUNCH(); k_chol_tri<<<1, 32, 0, s>>>(as, bd, keff, dd, ed, okb.as<int>());
    LOVE_LAUNCH_CHECK();
    LOVE_CUDA(cudaMemcpyAsync(&ok, okb.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    shifted = ok;
  }
  const int vec = 16 / (int)sizeof(T);
  // the root belongs to the cache: taken from (and later freed by) its allocator;
  // a root computed earlier is replaced
  if (c->S) c->alloc.free(c->S, sizeof(T) * (size_t)m * c->ld_s, s);
  c->S = nullptr;
  c->ks = 0;
  c->ld_s = (keff + vec - 1) / vec * vec;
  c->S = c->alloc.alloc(sizeof(T) * (size_t)m * c->ld_s, s);
  if (!c->S) return LOVE_ERR_OOM;
  c->ks = keff;
  if (ok) {
    LOVE_COUNT_LAUNCH(); k_root_from_chol<T><<<ceil_div(m * c->ld_s, 256), 256, 0, s>>>(Qb.as<double>(), m_pad, m, keff, dd, ed, (T*)c->S, c->ld_s);
    c->sampler_fallback = shifted;
  } else {
    Buf V(al, s), B(al, s), L(al, s);
    const int64_t nn = (int64_t)keff * keff;
    if (!V.get(sizeof(double) * nn) || !B.get(sizeof(double) * nn) || !L.get(sizeof(double) * keff))
      return LOVE_ERR_OOM;
    const size_t sme = sizeof(double) * 5 * (size_t)keff + sizeof(float) * 2 * (size_t)keff + sizeof(int) * keff;
    LOVE_COUNT_LAUNCH(); k_tri_eigpairs<<<keff, 32, sme, s>>>(ad, bd, keff, L.as<double>(), V.as<double>());
    LOVE_COUNT_LAUNCH(); k_tri_cluster_mgs<<<1, 256, 0, s>>>(keff, L.as<double>(), V.as<double>());
    LOVE_COUNT_LAUNCH(); k_scale_eig<<<ceil_div(nn, 256), 256, 0, s>>>(L.as<double>(), V.as<double>(), keff, B.as<double>());
    const size_t smq = sizeof(T) * (size_t)keff * ROOT_ROWS, smbb = sizeof(T) * (size_t)nn;
    const int stage_b = smq + smbb <= 100 * 1024;
    const size_t smb = smq + (stage_b ? smbb : 0);
    LOVE_TRY(allow_smem(k_root_from_eig<T>, smb));
    LOVE_COUNT_LAUNCH(); k_root_from_eig<T><<<ceil_div(m, ROOT_ROWS), 256, smb, s>>>(Qb.as<double>(), m_pad, m, keff, B.as<double>(), (T*)c->S, c->ld_s, stage_b);
    LOVE_LAUNCH_CHECK();
    LOVE_CUDA(cudaStreamSynchronize(s));
    c->sampler_fallback = 1;
  }
  LOVE_LAUNCH_CHECK();
  return cuda_check(cudaStreamSynchronize(s));
}

template love_status sampler_build<float>(const GridHost&, const FftPlan*, const Allocator&, love_cache*,
                                          const float*, int, uint64_t, double, cudaStream_t);
template love_status sampler_build<double>(const GridHost&, const FftPlan*, const Allocator&, love_cache*,
                                           const double*, int, uint64_t, double, cudaStream_t);

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }
// FP32: the canonical tiles of G, mu, Z and the canonical tiles of Z^T; FP64: G, mu, Z
static int canon_kpad(int ks) { return (ks + 7) / 8 * 8; }
template <typename T>
static size_t sample_ws_bytes_t(const love_cache* c, int64_t t, int s_count) {
  const int vec = 16 / (int)sizeof(T);
  const int ld_g = (c->ks + vec - 1) / vec * vec;
  if (sizeof(T) == 4) {
    const size_t tb = canon_tile_bytes(canon_kpad(c->ks));
    return round256(tb * (size_t)ceil_div(t, UM)) + round256(sizeof(T) * (size_t)t) +
           round256(sizeof(T) * (size_t)c->ks * s_count) + round256(tb * (size_t)ceil_div(s_count, UN));
  }
  return round256(sizeof(T) * (size_t)t * ld_g) + round256(sizeof(T) * (size_t)t) +
         round256(sizeof(T) * (size_t)c->ks * s_count);
}

// ws: optional work space of sample_ws_bytes_t bytes (then nothing is allocated)
template <typename T>
static love_status sample_impl(love_cache* c, int64_t t, const void* x, int s_count, const void* z, uint64_t seed,
                               void* out, cudaStream_t s, void* ws = nullptr) {
  const Allocator& al = c->alloc;
  const int ks = c->ks;
  const int vec = 16 / (int)sizeof(T);
  const int ld_g = (ks + vec - 1) / vec * vec;
  constexpr bool tc = std::is_same<T, float>::value;   // the tensor-core product on canonical tiles
  const int kpad = canon_kpad(ks);
  const size_t tb = canon_tile_bytes(kpad);
  const int64_t nti = ceil_div(t, UM), ntj = ceil_div((int64_t)s_count, UN);
  const size_t gbytes = tc ? tb * (size_t)nti : sizeof(T) * (size_t)t * ld_g;
  Buf Gb(al, s), mub(al, s), zb(al, s), zcb(al, s);
  T *Gp, *mup, *zp = nullptr;
  unsigned char* zc = nullptr;
  if (ws) {
    char* w = (char*)ws;
    Gp = (T*)w;
    mup = (T*)(w + round256(gbytes));
    zp = (T*)((char*)mup + round256(sizeof(T) * (size_t)t));
    if (tc) zc = (unsigned char*)zp + round256(sizeof(T) * (size_t)ks * s_count);
  } else {
    if (!Gb.get(gbytes) || !mub.get(sizeof(T) * (size_t)t)) return LOVE_ERR_OOM;
    if (tc && !zcb.get(tb * (size_t)ntj)) return LOVE_ERR_OOM;
    Gp = Gb.as<T>();
    mup = mub.as<T>();
    zc = zcb.as<unsigned char>();
  }
  const T* Z = (const T*)z;
  if (!Z) {
    int64_t cnt = (int64_t)ks * s_count;
    if (!zp) {
      if (!zb.get(sizeof(T) * cnt)) return LOVE_ERR_OOM;
      zp = zb.as<T>();
    }
    int64_t blocks4 = (cnt + 3) / 4;
    LOVE_COUNT_LAUNCH(); k_philox_normals<T><<<ceil_div(blocks4, 256), 256, 0, s>>>(cnt, seed, zp);
    Z = zp;
  }
  SampleGatherArgs a{};
  a.g = c->grid.dev();
  a.t = t;
  a.x = x;
  a.S = c->S;
  a.ld_s = c->ld_s;
  a.ks = ks;
  a.Rc = (c->flags & LOVE_WANT_MEAN) ? c->Rc : nullptr;
  a.ld_c = c->ld;
  a.kc = c->k_eff;
  a.cache_dtype = c->cache_dtype;
  a.G = tc ? nullptr : Gp;
  a.ld_g = ld_g;
  a.Gc = tc ? reinterpret_cast<unsigned char*>(Gp) : nullptr;
  a.kpad = kpad;
  a.mu = mup;
  a.status = c->status;
  int blocks = (int)std::min<int64_t>((t * 32 + 255) / 256, (int64_t)num_sms() * 16);
  switch (a.g.dim) {
    case 1: LOVE_COUNT_LAUNCH(); k_sample_gather<T, 1><<<blocks, 256, 0, s>>>(a); break;
    case 2: LOVE_COUNT_LAUNCH(); k_sample_gather<T, 2><<<blocks, 256, 0, s>>>(a); break;
    default: LOVE_COUNT_LAUNCH(); k_sample_gather<T, 3><<<blocks, 256, 0, s>>>(a);
  }
  if constexpr (tc) {
    const int64_t nz = ntj * kpad * 128;
    LOVE_COUNT_LAUNCH();
    k_z_canon<<<(unsigned)ceil_div(nz, 256), 256, 0, s>>>(Z, ks, s_count, kpad, (int)ntj, zc);
    dim3 grid((unsigned)nti, (unsigned)ntj);
    LOVE_TRY(allow_smem(k_sample_gemm_tc05, SG_SMEM));
    LOVE_COUNT_LAUNCH();
    k_sample_gemm_tc05<<<grid, 256, SG_SMEM, s>>>(reinterpret_cast<const unsigned char*>(Gp), zc, kpad, s_count,
                                                    mup, t, (float*)out, c->status);
  } else {
    dim3 grid((unsigned)((t + 63) / 64), (unsigned)((s_count + 63) / 64));
    LOVE_COUNT_LAUNCH(); k_sample_gemm<T><<<grid, 256, 0, s>>>(Gp, ld_g, Z, s_count, ks, mup, t, (T*)out);
  }
  return cuda_check(cudaGetLastError());
}

love_status sample_launch(love_cache* c, int64_t t, const void* x, int s_count, const void* z, uint64_t seed,
                          void* out, cudaStream_t s) {
  if (c->dtype == LOVE_F64) return sample_impl<double>(c, t, x, s_count, z, seed, out, s);
  return sample_impl<float>(c, t, x, s_count, z, seed, out, s);
}

size_t sample_ws_bytes(const love_cache* c, int64_t t, int s_count) {
  return c->dtype == LOVE_F64 ? sample_ws_bytes_t<double>(c, t, s_count) : sample_ws_bytes_t<float>(c, t, s_count);
}
love_status sample_launch_z_ws(love_cache* c, int64_t t, const void* x, int s_count, const void* z, uint64_t seed,
                               void* out, void* ws, cudaStream_t s) {
  if (t == 0 || s_count == 0) return LOVE_OK;
  if (c->dtype == LOVE_F64) return sample_impl<double>(c, t, x, s_count, z, seed, out, s, ws);
  return sample_impl<float>(c, t, x, s_count, z, seed, out, s, ws);
}
love_status sample_launch_ws(love_cache* c, int64_t t, const void* x, int s_count, uint64_t seed, void* out,
                             void* ws, cudaStream_t s) {
  if (t == 0 || s_count == 0) return LOVE_OK;
  if (c->dtype == LOVE_F64) return sample_impl<double>(c, t, x, s_count, nullptr, seed, out, s, ws);
  return sample_impl<float>(c, t, x, s_count, nullptr, seed, out, s, ws);
}

}  // namespace love
