// k_sampler.cu -- the sampler's Lanczos run (Sec. 3.3, eq. lancapprox) on a 1-D
// grid as ONE persistent cooperative kernel.
//
// k' steps of Lanczos with full reorthogonalisation (classical Gram-Schmidt
// twice, as the main run and the oracle) on the m x m operator
//     M = K_UU - Rt Rt^T        (K_UU Toeplitz, Rt m x k)
// from the SplitMix64 Rademacher probe.  The arithmetic is double-float
// (~2^-48 relative, on the FP32 pipes), with the per-step scalars in FP64: M's
// two terms cancel to ~1e-7 of their size on the 1-D n = 1e6 workload, so FP32
// alone would leave nothing of M.  The multi-launch form of the same run (k_lanczos.cu,
// FP64) spends ~8
// short launches per step, each latency-bound on m = 1e4 vectors; here one
// launch runs every step, with bounded grid barriers between its phases.
//
// Layout.  K_UU v is the circulant-embedding product of length N = N1 N2
// (power of two >= 2m - 1), computed by the four-step split of the K_UU
// product (k_fft.cu):
//   A  for each n1: FFT over n2 of x[n1 + N1 n2], times W_N^{n1 k2}
//   B  for each k2: FFT over n1, times lambda / N, inverse FFT over k1
//   C  for each n1: conjugate twiddles, inverse FFT over k2, real part.
// CTA b owns the columns n1 in [b NB, (b+1) NB) of passes A and C, and with
// them the grid rows r = n1 + N1 n2 (r < m): the rows its column transforms
// read and write.  Those rows' entries of every Lanczos vector, of Rt and of
// the working vector stay in the CTA's shared memory for the whole run (local
// row lr = f R2 + n2, f = n1 - b NB, R2 = ceil(m / N1); entries with r >= m are
// zero), so the reorthogonalisation never leaves the SM.  Rows of pass B
// (k2 in [b FB, (b+1) FB)) go through a global work array.
//
// One step j (5 grid barriers):
//   1  q_j = v / beta_{j-1} (own rows, also to Q' in HBM); pass A on q_j;
//      partial sums of Rt^T q_j over own rows                         | barrier
//   2  pass B; CTA b adds the partials of columns c = b, b + G, ... -> t = Rt^T q_j | barrier
//   3  pass C -> (K_UU q_j) on own rows; v = K_UU q_j - Rt t;
//      partials of c1 = Q_j^T v                                        | barrier
//   4  c1 summed (every CTA, same order); alpha_j = c1[j]; v -= Q_j c1;
//      partials of c2 = Q_j^T v                                        | barrier
//   5  c2 summed; v -= Q_j c2; partial of |v|^2                       | barrier
//   then beta_j = |v| in every CTA; stop at k', on NaN, or on breakdown
//   beta_j <= tau max|alpha| (the rule of the main run).
// Every sum is taken in a fixed order, so the run is bit-reproducible and all
// CTAs take the same stop decision.
#include <algorithm>
#include <cmath>

#include "lanczos_common.cuh"
#include "fft_core.cuh"

namespace love {
namespace {
using namespace fftcore;

constexpr int SAMP_THREADS = 512;
constexpr int SAMP_WARPS = SAMP_THREADS / 32;
constexpr int KP = LOVE_MAX_K + 8;   // stride of the per-CTA partial rows
constexpr int RQ = 4;                  // quarters of the cross-CTA sums (reduce_parts)
constexpr int SCRATCH = RQ * KP;       // doubles: rows_sub partials (<= SAMP_THREADS) or RQ x KP df pairs

template <typename RT>
struct SamplerArgs {
  int m, k, ks;
  const RT* Rt;          // m x k column-major, leading dimension ldr
  int64_t ldr;
  double* Q;             // m_pad x ks column-major (ldq): the Lanczos vectors, natural row order
  int64_t ldq;
  int N, N1, N2, logN1, logN2, logNB;
  int NB, FB, R2;        // n1 per CTA, k2 rows per CTA in pass B, rows per n1
  const float4* twdf;    // W_N^j, df complex
  const float2* lamdf;   // circulant spectrum / N, df
  float4* work;          // N df complex
  float2* part_t;        // G x KP df pairs: partial sums of Rt^T q
  float2* part_c1;       // G x KP df pairs
  float2* part_c2;       // G x KP df pairs
  float2* part_nn;       // G df pairs
  float2* tvec;          // k df pairs
  double* alpha;         // ks
  double* beta;          // ks
  int* k_eff;
  uint64_t seed;
  double tau;
  GridSync* gs;
  DevStatus* status;
};

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// GB300 runs FP64 at a small fraction of its FP32 rate, so the run keeps its
// vectors, products and transforms in double-float (a value as an unevaluated
// float pair hi + lo, ~2^-48 relative; error-free transformations on the FP32
// pipes): FP64 is left to the per-step scalars (alpha_j, beta_j, the stop rule)
// and to the rows of Q' written out.

// sum of exact products of double-float factors (Dot2 with the cross terms)
struct DotDF {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float2 a, float2 b) {
    const float p = a.x * b.x;
    float pe = fmaf(a.x, b.x, -p);
    pe = fmaf(a.x, b.y, pe);
    pe = fmaf(a.y, b.x, pe);
    const float t = s + p;
    const float z = t - s;
    c += pe + ((s - (t - z)) + (p - z));
    s = t;
  }
  __device__ __forceinline__ df get() const { return fast_two_sum(s, c); }
};
__device__ __forceinline__ df ld_df(const float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ float2 st_df(const df v) { return make_float2(v.hi, v.lo); }
__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.hi, o), l = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, df{h, l});
  }
  return v;
}
__device__ __forceinline__ dfc ld_dfc(const float4* p) {
  const float4 v = __ldcg(p);
  return dfc{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void st_dfc(float4* p, const dfc& v) { __stcg(p, make_float4(v.rh, v.rl, v.ih, v.il)); }
// a complex double-float times a real one
__device__ __forceinline__ dfc dfc_scale(const dfc& a, float2 l) {
  const df re = df_mul(df{a.rh, a.rl}, ld_df(l)), im = df_mul(df{a.ih, a.il}, ld_df(l));
  return dfc{re.hi, re.lo, im.hi, im.lo};
}
// the twiddles W_L^j (j < L/2) of one transform length from the df table of W_N
__device__ __forceinline__ void load_twiddles_tab(dfc* w, int L, const float4* __restrict__ twdf, int N) {
  const int step = N / L;
  for (int j = threadIdx.x; j < (L >> 1); j += blockDim.x) {
    const float4 v = twdf[(int64_t)j * step];
    w[j] = dfc{v.x, v.y, v.z, v.w};
  }
}

// part[i] = sum over own rows of Ms[i][lr] v[lr] for i < ncols: 4 threads per
// column take every 4th row, then two shuffles add them
__device__ __forceinline__ void cols_dot(const float2* Ms, int RL, int ncols, const float2* v, float2* part) {
  const int sub = threadIdx.x & 3;
  for (int i = threadIdx.x >> 2; i < ((ncols + 7) & ~7); i += SAMP_THREADS / 4) {
    DotDF acc;
    acc.zero();
    if (i < ncols) {
      const float2* col = Ms + (size_t)i * RL;
      for (int lr = sub; lr < RL; lr += 4) acc.add(col[lr], v[lr]);
    }
    df r = acc.get();
    for (int o = 1; o <= 2; o <<= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, r.hi, o), l = __shfl_xor_sync(0xffffffffu, r.lo, o);
      r = df_add(r, df{h, l});
    }
    if (sub == 0 && i < ncols) __stcg(part + i, st_df(r));
  }
}

// out[lr] = base[lr] - sum_{i < ncols} Ms[i][lr] c[i] for own rows: NG groups of
// RL threads split the columns, the group partials are added in group order
__device__ __forceinline__ void rows_sub(const float2* Ms, int RL, int ncols, const float2* c, const float2* base,
                                         float2* out, float2* scratch) {
  const int NG = SAMP_THREADS / RL;   // RL <= SAMP_THREADS is enforced on the host
  const int g = threadIdx.x / RL, lr = threadIdx.x - g * RL;
  if (g < NG) {
    DotDF acc;
    acc.zero();
    for (int i = g; i < ncols; i += NG) acc.add(Ms[(size_t)i * RL + lr], c[i]);
    scratch[g * RL + lr] = st_df(acc.get());
  }
  __syncthreads();
  for (int r = threadIdx.x; r < RL; r += SAMP_THREADS) {
    df s = ld_df(scratch[r]);
    for (int q = 1; q < NG; ++q) s = df_add(s, ld_df(scratch[q * RL + r]));
    out[r] = st_df(df_add(ld_df(base[r]), df_neg(s)));
  }
  __syncthreads();
}

// out[i] = sum_b part[b][i] for i < n (df pairs from every CTA), the same in
// every CTA: thread (q, i) adds the partials of CTAs q, q + 4, ... in order
// (all its loads issued first), then thread i adds the four quarter sums
__device__ __forceinline__ void reduce_parts(const float2* part, int G, int n, float2* out, float2* scratch) {
  for (int t = threadIdx.x; t < RQ * n; t += SAMP_THREADS) {
    const int q = t / n, i = t - q * n;
    df acc{0.f, 0.f};
    int bb = q;
    for (; bb + 3 * RQ < G; bb += 4 * RQ) {
      float2 p0 = __ldcg(part + (size_t)bb * KP + i), p1 = __ldcg(part + (size_t)(bb + RQ) * KP + i);
      float2 p2 = __ldcg(part + (size_t)(bb + 2 * RQ) * KP + i), p3 = __ldcg(part + (size_t)(bb + 3 * RQ) * KP + i);
      acc = df_add(acc, ld_df(p0));
      acc = df_add(acc, ld_df(p1));
      acc = df_add(acc, ld_df(p2));
      acc = df_add(acc, ld_df(p3));
    }
    for (; bb < G; bb += RQ) acc = df_add(acc, ld_df(__ldcg(part + (size_t)bb * KP + i)));
    scratch[t] = st_df(acc);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += SAMP_THREADS) {
    df acc = ld_df(scratch[i]);
    for (int q = 1; q < RQ; ++q) acc = df_add(acc, ld_df(scratch[q * n + i]));
    out[i] = st_df(acc);
  }
  __syncthreads();
}

template <typename RT> __device__ __forceinline__ float2 to_df(RT v);
template <> __device__ __forceinline__ float2 to_df<float>(float v) { return make_float2(v, 0.f); }

template <typename RT>
__global__ void __launch_bounds__(SAMP_THREADS, 1) k_sampler_lanczos(const __grid_constant__ SamplerArgs<RT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int NB = a.NB, R2 = a.R2, RL = NB * R2;
  const int n1_0 = b * NB;
  // shared memory: x [N / G] complex, wA [N2 / 2], wB [N1 / 2] (complex first: 16-byte
  // aligned), scratch [SCRATCH], cvec [KP], tv [KP], v [RL], kq [RL], Qs [ks][RL],
  // then Rs [k][RL]; every real entry a df pair
  dfc* x = reinterpret_cast<dfc*>(smem_raw);
  dfc* wA = x + a.N / G;
  dfc* wB = wA + a.N2 / 2;
  float2* scratch = reinterpret_cast<float2*>(wB + a.N1 / 2);
  float2* cvec = scratch + SCRATCH;
  float2* tv = cvec + KP;
  float2* v = tv + KP;
  float2* kq = v + RL;
  float2* Qs = kq + RL;
  float2* Rs = Qs + (size_t)a.ks * RL;   // Rt's own rows
  __shared__ double s_beta, s_amax;
  __shared__ int s_stop;

  load_twiddles_tab(wA, a.N2, a.twdf, a.N);
  load_twiddles_tab(wB, a.N1, a.twdf, a.N);
  // own rows of Rt (zero past m) and of the probe v_0 (Rademacher, 1 / sqrt(m) after scaling)
  for (int i = tid; i < a.k * RL; i += SAMP_THREADS) {
    const int c = i / RL, lr = i - c * RL;
    const int f = lr / R2, n2 = lr - f * R2;
    const int r = n1_0 + f + a.N1 * n2;
    Rs[i] = r < a.m ? to_df<RT>(a.Rt[(int64_t)c * a.ldr + r]) : make_float2(0.f, 0.f);
  }
  for (int lr = tid; lr < RL; lr += SAMP_THREADS) {
    const int f = lr / R2, n2 = lr - f * R2;
    const int r = n1_0 + f + a.N1 * n2;
    v[lr] = make_float2(r < a.m ? ((splitmix64_at(a.seed, (uint64_t)r) & 1ull) ? 1.f : -1.f) : 0.f, 0.f);
  }
  if (tid == 0) {
    s_beta = sqrt((double)a.m);
    s_amax = 0.0;
    s_stop = 0;
  }
  __syncthreads();
  unsigned int gen = 0;
  int keff = a.ks;
  for (int j = 0; j < a.ks; ++j) {
    // ---- 1: q_j, pass A, partials of Rt^T q_j
    const df inv = df_from_double(1.0 / s_beta);
    float2* qj = Qs + (size_t)j * RL;
    for (int lr = tid; lr < RL; lr += SAMP_THREADS) {
      const df q = df_mul(ld_df(v[lr]), inv);
      qj[lr] = st_df(q);
      const int f = lr / R2, n2 = lr - f * R2;
      const int r = n1_0 + f + a.N1 * n2;
      if (r < a.m) a.Q[(int64_t)j * a.ldq + r] = df_to_double(q);
    }
    __syncthreads();
    for (int t = tid; t < (a.N2 << a.logNB); t += SAMP_THREADS) {
      const int f = t & (NB - 1), n2 = t >> a.logNB;
      const float2 q = n2 < R2 ? qj[f * R2 + n2] : make_float2(0.f, 0.f);
      x[(bitrev(n2, a.logN2) << a.logNB) + f] = dfc{q.x, q.y, 0.f, 0.f};
    }
    __syncthreads();
    fft_dit_df(x, a.N2, a.logNB, wA, false);
    for (int t = tid; t < (a.N2 << a.logNB); t += SAMP_THREADS) {
      const int f = t & (NB - 1), k2 = t >> a.logNB;
      const int n1 = n1_0 + f;
      const float4 w = a.twdf[((int64_t)n1 * k2) & (a.N - 1)];
      st_dfc(a.work + (int64_t)k2 * a.N1 + n1, dfc_mul(x[t], dfc{w.x, w.y, w.z, w.w}, false));
    }
    cols_dot(Rs, RL, a.k, qj, a.part_t + (size_t)b * KP);
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 2: pass B (rows k2 of this CTA); t = Rt^T q_j for columns b, b + G, ...
    {
      const int FB = a.FB, logFB = a.logN2 - (a.logN1 - a.logNB);   // FB = N2 / G
      const int k2_0 = b * FB;
      for (int t = tid; t < (a.N1 << logFB); t += SAMP_THREADS) {
        const int n1 = t & (a.N1 - 1), f = t >> a.logN1;
        x[(bitrev(n1, a.logN1) << logFB) + f] = ld_dfc(a.work + (int64_t)(k2_0 + f) * a.N1 + n1);
      }
      __syncthreads();
      fft_dit_df(x, a.N1, logFB, wB, false);
      for (int t = tid; t < (a.N1 << logFB); t += SAMP_THREADS) {
        const int f = t & (FB - 1), k1 = t >> logFB;
        x[t] = dfc_scale(x[t], a.lamdf[(k2_0 + f) + a.N2 * k1]);
      }
      __syncthreads();
      fft_dif_df(x, a.N1, logFB, wB, true);
      for (int t = tid; t < (a.N1 << logFB); t += SAMP_THREADS) {
        const int n1 = t & (a.N1 - 1), f = t >> a.logN1;
        st_dfc(a.work + (int64_t)(k2_0 + f) * a.N1 + n1, x[(bitrev(n1, a.logN1) << logFB) + f]);
      }
    }
    for (int c = b + G * (tid >> 5); c < a.k && (tid >> 5) < SAMP_WARPS; c += G * SAMP_WARPS) {
      // warp (tid >> 5) adds column c's partials over the CTAs: lane l those of
      // CTAs l, l + 32, ..., then a fixed df butterfly across the lanes
      const int lane = tid & 31;
      df acc{0.f, 0.f};
      for (int bb = lane; bb < G; bb += 32) acc = df_add(acc, ld_df(__ldcg(a.part_t + (size_t)bb * KP + c)));
      acc = warp_sum_df(acc);
      if (lane == 0) __stcg(a.tvec + c, st_df(acc));
    }
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 3: pass C -> K_UU q_j on own rows; v = K_UU q_j - Rt t; partials of c1
    for (int c = tid; c < a.k; c += SAMP_THREADS) tv[c] = __ldcg(a.tvec + c);
    for (int t = tid; t < (a.N2 << a.logNB); t += SAMP_THREADS) {
      const int f = t & (NB - 1), k2 = t >> a.logNB;
      const int n1 = n1_0 + f;
      const float4 w = a.twdf[((int64_t)n1 * k2) & (a.N - 1)];
      x[t] = dfc_mul(ld_dfc(a.work + (int64_t)k2 * a.N1 + n1), dfc{w.x, w.y, w.z, w.w}, true);
    }
    __syncthreads();
    fft_dif_df(x, a.N2, a.logNB, wA, true);
    for (int lr = tid; lr < RL; lr += SAMP_THREADS) {
      const int f = lr / R2, n2 = lr - f * R2;
      const int r = n1_0 + f + a.N1 * n2;
      const dfc& o = x[(bitrev(n2, a.logN2) << a.logNB) + f];
      kq[lr] = r < a.m ? make_float2(o.rh, o.rl) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    rows_sub(Rs, RL, a.k, tv, kq, v, scratch);
    cols_dot(Qs, RL, j + 1, v, a.part_c1 + (size_t)b * KP);
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 4: c1; alpha_j; v -= Q_j c1; partials of c2
    reduce_parts(a.part_c1, G, j + 1, cvec, scratch);
    const double alpha_j = df_to_double(ld_df(cvec[j]));
    rows_sub(Qs, RL, j + 1, cvec, v, v, scratch);
    cols_dot(Qs, RL, j + 1, v, a.part_c2 + (size_t)b * KP);
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 5: c2; v -= Q_j c2; partial of |v|^2
    reduce_parts(a.part_c2, G, j + 1, cvec, scratch);
    rows_sub(Qs, RL, j + 1, cvec, v, v, scratch);
    {
      const int lane = tid & 31, w = tid >> 5;
      DotDF acc;
      acc.zero();
      for (int lr = tid; lr < RL; lr += SAMP_THREADS) acc.add(v[lr], v[lr]);
      const df s = warp_sum_df(acc.get());
      if (lane == 0) scratch[w] = st_df(s);
      __syncthreads();
      if (tid == 0) {
        df t = ld_df(scratch[0]);
        for (int q = 1; q < SAMP_WARPS; ++q) t = df_add(t, ld_df(scratch[q]));
        __stcg(a.part_nn + b, st_df(t));
      }
    }
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- beta_j and the stop rule (identical in every CTA)
    if (tid < 32) {
      df nn{0.f, 0.f};
      for (int bb = tid; bb < G; bb += 32) nn = df_add(nn, ld_df(__ldcg(a.part_nn + bb)));
      nn = warp_sum_df(nn);
      if (tid == 0) scratch[0] = st_df(nn);
    }
    __syncthreads();
    if (tid == 0) {
      const double beta_j = sqrt(df_to_double(ld_df(scratch[0])));
      s_amax = fmax(s_amax, fabs(alpha_j));
      if (b == 0) {
        a.alpha[j] = alpha_j;
        a.beta[j] = beta_j;
      }
      s_stop = 0;
      if (!isfinite(beta_j) || !isfinite(alpha_j)) {
        s_stop = 2;
      } else if (j + 1 < a.ks && beta_j <= a.tau * s_amax) {
        s_stop = 1;
      }
      s_beta = beta_j;
    }
    __syncthreads();
    if (s_stop == 2) {
      keff = j;
      if (b == 0 && tid == 0) dev_flag(a.status, LOVE_ERR_NAN);
      break;
    }
    if (s_stop == 1) {
      keff = j + 1;
      break;
    }
  }
  if (b == 0 && tid == 0) *a.k_eff = keff;
}

int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

size_t sampler_smem_bytes(int ks, int k, int RL, int N, int G, int N1, int N2) {
  return sizeof(dfc) * ((size_t)N / G + N2 / 2 + N1 / 2) +
         sizeof(float2) * (SCRATCH + 2 * (size_t)KP + 2 * (size_t)RL + (size_t)(ks + k) * RL);
}

}  // namespace

template <typename T>
love_status sampler_lanczos_fused(const GridHost& gh, const FftPlan* fft, const Allocator& al, const T* Rt,
                                  int64_t ldr, int k, int ks, uint64_t seed, double tau, double* Q, int64_t ldq,
                                  double* alpha_h, double* beta_h, int* ks_eff, DevStatus* status, cudaStream_t s) {
  // FP64 caches keep FP64 Lanczos vectors (the multi-launch run): double-float
  // moves their late sampler columns by ~1e-7 relative
  if (gh.dim != 1 || gh.additive || sizeof(T) != sizeof(float)) return LOVE_ERR_UNSUPPORTED;
  if (ks < 1 || ks > LOVE_MAX_K || k < 1 || k > LOVE_MAX_K) return LOVE_ERR_ARG;
  const FftPlan& p = fft[0];
  const int m = (int)gh.m;
  const int N = (int)p.N;
  if (N < 64 || !p.tw_d || !p.lam_d) return LOVE_ERR_UNSUPPORTED;
  const int l = ilog2i(N);
  const int N1 = 1 << (l / 2), N2 = N >> (l / 2);   // N2 = N1 or 2 N1
  const int R2 = (m + N1 - 1) / N1;
  int dev = 0, coop = 0;
  LOVE_CUDA(cudaGetDevice(&dev));
  LOVE_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return LOVE_ERR_UNSUPPORTED;
  // the most CTAs that can be co-resident: one per SM (the kernel takes over 48 KB of
  // shared memory and SAMP_THREADS threads); a power of two dividing N1
  int G = N1;
  while (G > num_sms()) G >>= 1;
  const int NB = N1 / G, FB = N2 / G, RL = NB * R2;
  if (RL > SAMP_THREADS) return LOVE_ERR_UNSUPPORTED;
  const size_t smem = sampler_smem_bytes(ks, k, RL, N, G, N1, N2);
  const int limit = smem_limit(reinterpret_cast<const void*>(k_sampler_lanczos<T>));
  if (limit < 0) return LOVE_ERR_CUDA;
  if (smem > (size_t)limit) return LOVE_ERR_UNSUPPORTED;
  LOVE_TRY(allow_smem(k_sampler_lanczos<T>, smem));
  int per_sm = 0;
  LOVE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sampler_lanczos<T>, SAMP_THREADS, smem));
  if (per_sm < 1 || (int64_t)per_sm * num_sms() < G) return LOVE_ERR_UNSUPPORTED;

  // work: N df complex | N df twiddles | N df spectrum | 3 G KP partials | G | k |
  // ks alpha | ks beta | k_eff | GridSync
  const size_t off_tab = sizeof(float4) * (size_t)N;
  const size_t off_part = off_tab + (sizeof(float4) + sizeof(float2)) * (size_t)N;
  const size_t n_dbl = 3 * (size_t)G * KP + G + KP + 2 * (size_t)KP;
  const size_t off_int = off_part + sizeof(double) * n_dbl;
  const size_t bytes = off_int + 64 + sizeof(GridSync);
  char* w = (char*)scratch_alloc(al, bytes, s);
  if (!w) return LOVE_ERR_OOM;
  SamplerArgs<T> a{};
  a.m = m;
  a.k = k;
  a.ks = ks;
  a.Rt = Rt;
  a.ldr = ldr;
  a.Q = Q;
  a.ldq = ldq;
  a.N = N;
  a.N1 = N1;
  a.N2 = N2;
  a.logN1 = ilog2i(N1);
  a.logN2 = ilog2i(N2);
  a.logNB = ilog2i(NB);
  a.NB = NB;
  a.FB = FB;
  a.R2 = R2;
  a.work = (float4*)w;
  a.twdf = (const float4*)(w + off_tab);
  a.lamdf = (const float2*)(w + off_tab + sizeof(float4) * (size_t)N);
  double* d = (double*)(w + off_part);
  a.part_t = reinterpret_cast<float2*>(d);   // a float2 is one double's bytes
  a.part_c1 = a.part_t + (size_t)G * KP;
  a.part_c2 = a.part_c1 + (size_t)G * KP;
  a.part_nn = a.part_c2 + (size_t)G * KP;
  a.tvec = a.part_nn + G;
  a.alpha = d + 3 * (size_t)G * KP + G + KP;
  a.beta = a.alpha + KP;
  a.k_eff = (int*)(w + off_int);
  a.gs = (GridSync*)(w + off_int + 64);
  a.seed = seed;
  a.tau = tau;
  a.status = status;
  // rows m .. ldq of Q' are not written: the root kernels read rows below m only
  love_status rc = fft_df_tables(p, (float4*)(w + off_tab), (float2*)(w + off_tab + sizeof(float4) * (size_t)N), s);
  if (rc == LOVE_OK) rc = cuda_check(cudaMemsetAsync(w + off_int, 0, 64 + sizeof(GridSync), s));
  if (rc == LOVE_OK) rc = cuda_check(cudaMemsetAsync(a.alpha, 0, sizeof(double) * 2 * KP, s));
  if (rc == LOVE_OK) {
    void* args[] = {(void*)&a};
    LOVE_COUNT_LAUNCH();
    rc = cuda_check(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_sampler_lanczos<T>), dim3(G),
                                                dim3(SAMP_THREADS), args, smem, s));
  }
  int keff = 0;
  GridSync gsh{};
  if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(&keff, a.k_eff, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(&gsh, a.gs, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(alpha_h, a.alpha, sizeof(double) * ks, cudaMemcpyDeviceToHost, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(beta_h, a.beta, sizeof(double) * ks, cudaMemcpyDeviceToHost, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  scratch_free(al, w, bytes, s);
  if (rc != LOVE_OK) return rc;
  if (gsh.abort) return LOVE_ERR_TIMEOUT;   // a grid barrier gave up waiting
  *ks_eff = keff;
  return LOVE_OK;
}

template love_status sampler_lanczos_fused<float>(const GridHost&, const FftPlan*, const Allocator&, const float*,
                                                  int64_t, int, int, uint64_t, double, double*, int64_t, double*,
                                                  double*, int*, DevStatus*, cudaStream_t);
template <>
love_status sampler_lanczos_fused<double>(const GridHost&, const FftPlan*, const Allocator&, const double*, int64_t,
                                          int, int, uint64_t, double, double*, int64_t, double*, double*, int*,
                                          DevStatus*, cudaStream_t) {
  return LOVE_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------------------
// The same sampler run as a sequence of launches, for the cases the persistent
// kernel above does not take (FP64 caches, 2-D and 3-D grids, additive
// compositions): k' steps on M = K_UU - Rt Rt^T, an m x m operator, in FP64
// with the n-space run's CGS2 reorthogonalisation sweeps.
// M's entries are differences of nearly equal numbers (K_UU ~ 1, posterior
// ~ 1e-7 on the 1-D n = 1e6 workload), so FP32 would lose them entirely.
// The probe (not given by the paper) is the Rademacher vector
// r_i = +1 if the low bit of SplitMix64 output i (seeded with `seed`) is 1, else -1.
namespace {

template <typename QT>
__global__ void k_rademacher(int64_t m, int64_t m_pad, uint64_t seed, QT* __restrict__ q0, LanczosState* st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m_pad) q0[i] = i < m ? ((splitmix64_at(seed, (uint64_t)i) & 1ull) ? QT(1) : QT(-1)) : QT(0);
  if (i == 0) st->scal[0] = 1.0 / sqrt((double)m);
}
// Partial products of the sampler operator's low-rank term (R = Rt, m x k,
// column-major): tp[c * RS + rs] = sum over rows of slice rs of R[r, c] q[r],
// a block per (column, slice of GEMV_SLICE rows), each thread 4 rows.
constexpr int GEMV_SLICE = 1024;
template <typename T>
__global__ void k_gemv_t(const T* __restrict__ R, int64_t ldr, int64_t m, const double* __restrict__ q,
                         double* __restrict__ tp, const LanczosState* st) {
  __shared__ DotAccD red[32];
  if (st->done) return;
  const int c = blockIdx.x, rs = blockIdx.y;
  const int64_t r0 = (int64_t)rs * GEMV_SLICE;
  DotAccD a;
  a.zero();
#pragma unroll
  for (int u = 0; u < GEMV_SLICE / 256; ++u) {
    const int64_t r = r0 + u * 256 + threadIdx.x;
    if (r < m) a.add_prod((double)R[(int64_t)c * ldr + r], q[r]);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) tp[(int64_t)c * gridDim.y + rs] = a.value();
}
// y[r] = Kq[r] - sum_c R[r, c] t[c]  (0 on padding rows); t[c] = the sum of
// the RS slice partials (fixed order).  A block covers 32 rows: warp w takes
// the columns w, w + 8, ..., lane l row l, then the 8 warp sums are added.
// (y in the storage type of the Lanczos vectors: the FP64 difference rounded once)
template <typename T, typename YT>
__global__ void k_gemv_n_sub(const T* __restrict__ R, int64_t ldr, int64_t m, int64_t m_pad, int k, int RS,
                             const double* __restrict__ tp, const double* __restrict__ Kq, YT* __restrict__ y,
                             const LanczosState* st) {
  extern __shared__ double t_s[];   // [k] then [8][32]
  if (st->done) return;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double v = 0.0;
    for (int rs = 0; rs < RS; ++rs) v += tp[(int64_t)c * RS + rs];
    t_s[c] = v;
  }
  __syncthreads();
  double* ws = t_s + k;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (r < m) {
#pragma unroll 4
    for (int c = w; c < k; c += 8) acc = fma((double)R[(int64_t)c * ldr + r], t_s[c], acc);
  }
  ws[w * 32 + lane] = acc;
  __syncthreads();
  if (w == 0 && r < m_pad) {
    double sum = 0.0;
#pragma unroll
    for (int v = 0; v < 8; ++v) sum += ws[v * 32 + lane];
    y[r] = r < m ? (YT)(Kq[r] - sum) : YT(0);
  }
}

}  // namespace

// The Lanczos vectors Q' are FP64 whatever the data dtype T of Rt: the run is
// m-sized, and M q (K_UU q and Rt (Rt^T q) cancel to ~1e-7 of their size on the
// 1-D n = 1e6 workload) is formed and kept in FP64, so the root is that of the
// operator the cache defines to FP64 accuracy before it is rounded to T.
template <typename T>
love_status sampler_lanczos(const GridHost& gh, const FftPlan* fft, const Allocator& al, const T* Rt, int64_t ldr,
                            int k, int ks, uint64_t seed, double tau, double* Q, int64_t ldq, double* alpha_h,
                            double* beta_h, int* ks_eff, DevStatus* status, cudaStream_t s) {
  const int64_t m = gh.m, m_pad = ldq;
  if (ks < 1 || ks > LOVE_MAX_K || m_pad % TILE_R) return LOVE_ERR_ARG;
  const int bc = box_cols(sizeof(double));
  const int max_grid = std::max(TILE_CTAS_PER_SM * num_sms(), 1024);
  DevBuf stb(al, s), part(al, s), kq(al, s), y(al, s), tv(al, s), fw(al, s);
  size_t fwb = fft_work_bytes(gh, fft, 1, true);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * (size_t)max_grid * (ks + 1)) ||
      !kq.get(sizeof(double) * m) || !y.get(sizeof(double) * m_pad) ||
      !tv.get(sizeof(double) * (size_t)(k + 1) * (size_t)ceil_div(m, GEMV_SLICE)) ||
      !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, ks, tau);
  LOVE_COUNT_LAUNCH(); k_rademacher<double><<<ceil_div(m_pad, 256), 256, 0, s>>>(m, m_pad, seed, Q, st);
  LOVE_LAUNCH_CHECK();
  TileArgs<double> ta{};
  ta.n_pad = m_pad;
  ta.kcols = ks;
  ta.bc = bc;
  ta.Q = Q;
  ta.ldq = ldq;
  ta.y = y.as<double>();
  ta.partial = part.as<double2>();
  ta.st = st;
  ta.status = status;
  const int nb = std::min(4 * num_sms(), ceil_div(m_pad, 256));
  const int RS = ceil_div(m, GEMV_SLICE);
  const size_t nsub_smem = sizeof(double) * ((size_t)k + 8 * 32);
  LOVE_TRY(allow_smem(k_gemv_n_sub<T, double>, nsub_smem));
  for (int j = 0; j < ks; ++j) {
    double* qj = Q + (int64_t)j * ldq;
    LOVE_COUNT_LAUNCH(); k_normalize_col<double><<<nb, 256, 0, s>>>(qj, m_pad, st->scal + j, st);
    LOVE_TRY(kuu_apply<double>(gh, fft, qj, kq.as<double>(), 1, m, fw.p, -1, s));
    LOVE_COUNT_LAUNCH(); k_gemv_t<T><<<dim3(k, RS), 256, 0, s>>>(Rt, ldr, m, qj, tv.as<double>(), st);
    LOVE_COUNT_LAUNCH(); k_gemv_n_sub<T, double><<<ceil_div(m_pad, 32), 256, nsub_smem, s>>>(Rt, ldr, m, m_pad, k, RS, tv.as<double>(), kq.as<double>(), y.as<double>(), st);
    LOVE_LAUNCH_CHECK();
    ta.j = j;
    LOVE_TRY(reorth_sweep<double, MODE_DOT>(ta, s));
    LOVE_TRY(reorth_sweep<double, MODE_UPDATE_DOT>(ta, s));
    LOVE_TRY(reorth_sweep<double, MODE_UPDATE_NORM>(ta, s));
  }
  int keff = 0;
  LOVE_CUDA(cudaMemcpyAsync(&keff, &st->k_eff, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaMemcpyAsync(alpha_h, st->alpha, sizeof(double) * ks, cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaMemcpyAsync(beta_h, st->beta, sizeof(double) * ks, cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  *ks_eff = keff;
  return LOVE_OK;
}

template love_status sampler_lanczos<float>(const GridHost&, const FftPlan*, const Allocator&, const float*, int64_t,
                                            int, int, uint64_t, double, double*, int64_t, double*, double*, int*,
                                            DevStatus*, cudaStream_t);
template love_status sampler_lanczos<double>(const GridHost&, const FftPlan*, const Allocator&, const double*,
                                             int64_t, int, int, uint64_t, double, double*, int64_t, double*, double*,
                                             int*, DevStatus*, cudaStream_t);

}  // namespace love
