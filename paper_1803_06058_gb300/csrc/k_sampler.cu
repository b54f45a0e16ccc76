// k_sampler.cu -- the sampler's Lanczos run (Sec. 3.3, eq. lancapprox) on a 1-D
// grid as ONE persistent cooperative kernel.
//
// k' steps of Lanczos with full reorthogonalisation (classical Gram-Schmidt
// twice, as the main run and the oracle) on the m x m operator
//     M = K_UU - Rt Rt^T        (K_UU Toeplitz, Rt m x k)
// from the SplitMix64 Rademacher probe.  All arithmetic is FP64: the work is
// m-sized, and M's two terms cancel to ~1e-7 of their size on the 1-D n = 1e6
// workload.  The multi-launch form of the same run (k_lanczos.cu) spends ~8
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

#include "love_internal.cuh"
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
  const double2* tw;     // W_N^j
  const double* lam;     // circulant spectrum / N
  double2* work;         // N complex
  float2* part_t;        // G x KP df pairs: partial sums of Rt^T q
  float2* part_c1;       // G x KP df pairs
  float2* part_c2;       // G x KP df pairs
  double* part_nn;       // G
  double* tvec;          // k
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// This part runs FP64 at a small fraction of its FP32 rate, and the run is
// bound by the FP64 pipe: the dots below keep their FP64 work to one FMA per
// row and column (plus two adds per column), and the per-CTA partials that
// every CTA must add up go out as double-float pairs, summed on the FP32 pipes
// (error-free transformations, ~2^-48 relative).

// part[i] = sum over own rows of Ms[i][lr] v[lr] for i < ncols, as a df pair:
// 4 threads per column take every 4th row, then two shuffles add them
__device__ __forceinline__ void cols_dot(const double* Ms, int RL, int ncols, const double* v, float2* part) {
  const int sub = threadIdx.x & 3;
  for (int i = threadIdx.x >> 2; i < ((ncols + 7) & ~7); i += SAMP_THREADS / 4) {
    double s = 0.0;
    if (i < ncols) {
      const double* col = Ms + (size_t)i * RL;
      for (int lr = sub; lr < RL; lr += 4) s = fma(col[lr], v[lr], s);
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (sub == 0 && i < ncols) {
      const float hi = (float)s;
      __stcg(part + i, make_float2(hi, (float)(s - (double)hi)));
    }
  }
}

// out[lr] = base[lr] - sum_{i < ncols} Ms[i][lr] c[i] for own rows: NG groups of
// RL threads split the columns, the group partials are added in group order
__device__ __forceinline__ void rows_sub(const double* Ms, int RL, int ncols, const double* c, const double* base,
                                         double* out, double* scratch) {
  const int NG = SAMP_THREADS / RL;   // RL <= SAMP_THREADS is enforced on the host
  const int g = threadIdx.x / RL, lr = threadIdx.x - g * RL;
  if (g < NG) {
    double s = 0.0;
    for (int i = g; i < ncols; i += NG) s = fma(Ms[(size_t)i * RL + lr], c[i], s);
    scratch[g * RL + lr] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < RL; r += SAMP_THREADS) {
    double s = 0.0;
    for (int q = 0; q < NG; ++q) s += scratch[q * RL + r];
    out[r] = base[r] - s;
  }
  __syncthreads();
}

// out[i] = sum_b part[b][i] for i < n (df pairs from every CTA), the same in
// every CTA: thread (q, i) adds the partials of CTAs q, q + 4, ... in order
// (all its loads issued first), then thread i adds the four quarter sums

__device__ __forceinline__ void reduce_parts(const float2* part, int G, int n, double* out, float2* scratch) {
  for (int t = threadIdx.x; t < RQ * n; t += SAMP_THREADS) {
    const int q = t / n, i = t - q * n;
    df acc{0.f, 0.f};
    int bb = q;
    for (; bb + 3 * RQ < G; bb += 4 * RQ) {
      float2 p0 = __ldcg(part + (size_t)bb * KP + i), p1 = __ldcg(part + (size_t)(bb + RQ) * KP + i);
      float2 p2 = __ldcg(part + (size_t)(bb + 2 * RQ) * KP + i), p3 = __ldcg(part + (size_t)(bb + 3 * RQ) * KP + i);
      acc = df_add(acc, df{p0.x, p0.y});
      acc = df_add(acc, df{p1.x, p1.y});
      acc = df_add(acc, df{p2.x, p2.y});
      acc = df_add(acc, df{p3.x, p3.y});
    }
    for (; bb < G; bb += RQ) {
      const float2 p = __ldcg(part + (size_t)bb * KP + i);
      acc = df_add(acc, df{p.x, p.y});
    }
    scratch[t] = make_float2(acc.hi, acc.lo);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += SAMP_THREADS) {
    df acc{scratch[i].x, scratch[i].y};
    for (int q = 1; q < RQ; ++q) acc = df_add(acc, df{scratch[q * n + i].x, scratch[q * n + i].y});
    out[i] = (double)acc.hi + (double)acc.lo;
  }
  __syncthreads();
}

template <typename RT>
__global__ void __launch_bounds__(SAMP_THREADS, 1) k_sampler_lanczos(const __grid_constant__ SamplerArgs<RT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int NB = a.NB, R2 = a.R2, RL = NB * R2;
  const int n1_0 = b * NB;
  // shared memory: x [N / G] complex, wA [N2 / 2], wB [N1 / 2] (complex first: 16-byte
  // aligned), scratch [SAMP_THREADS], cvec [KP], tv [KP], v [RL], kq [RL], Qs [ks][RL],
  // then Rs [k][RL] (RT)
  double2* x = reinterpret_cast<double2*>(smem_raw);
  double2* wA = x + a.N / G;
  double2* wB = wA + a.N2 / 2;
  double* scratch = reinterpret_cast<double*>(wB + a.N1 / 2);   // SCRATCH doubles
  double* cvec = scratch + SCRATCH;
  double* tv = cvec + KP;
  double* v = tv + KP;
  double* kq = v + RL;
  double* Qs = kq + RL;
  double* Rs = Qs + (size_t)a.ks * RL;   // Rt's own rows, in FP64
  __shared__ double s_beta, s_amax;
  __shared__ int s_stop;

  load_twiddles(wA, a.N2, a.tw, a.N);
  load_twiddles(wB, a.N1, a.tw, a.N);
  // own rows of Rt (zero past m) and of the probe v_0 (Rademacher, 1 / sqrt(m) after scaling)
  for (int i = tid; i < a.k * RL; i += SAMP_THREADS) {
    const int c = i / RL, lr = i - c * RL;
    const int f = lr / R2, n2 = lr - f * R2;
    const int r = n1_0 + f + a.N1 * n2;
    Rs[i] = r < a.m ? (double)a.Rt[(int64_t)c * a.ldr + r] : 0.0;
  }
  for (int lr = tid; lr < RL; lr += SAMP_THREADS) {
    const int f = lr / R2, n2 = lr - f * R2;
    const int r = n1_0 + f + a.N1 * n2;
    v[lr] = r < a.m ? ((splitmix64_at(a.seed, (uint64_t)r) & 1ull) ? 1.0 : -1.0) : 0.0;
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
    const double inv = 1.0 / s_beta;
    double* qj = Qs + (size_t)j * RL;
    for (int lr = tid; lr < RL; lr += SAMP_THREADS) {
      const double q = v[lr] * inv;
      qj[lr] = q;
      const int f = lr / R2, n2 = lr - f * R2;
      const int r = n1_0 + f + a.N1 * n2;
      if (r < a.m) a.Q[(int64_t)j * a.ldq + r] = q;
    }
    __syncthreads();
    for (int t = tid; t < (a.N2 << a.logNB); t += SAMP_THREADS) {
      const int f = t & (NB - 1), n2 = t >> a.logNB;
      double2 c;
      c.x = n2 < R2 ? qj[f * R2 + n2] : 0.0;
      c.y = 0.0;
      x[(bitrev(n2, a.logN2) << a.logNB) + f] = c;
    }
    __syncthreads();
    fft_dit(x, a.N2, a.logNB, wA, false);
    for (int t = tid; t < (a.N2 << a.logNB); t += SAMP_THREADS) {
      const int f = t & (NB - 1), k2 = t >> a.logNB;
      const int n1 = n1_0 + f;
      __stcg(a.work + (int64_t)k2 * a.N1 + n1, cmul(x[t], a.tw[((int64_t)n1 * k2) & (a.N - 1)]));
    }
    cols_dot(Rs, RL, a.k, qj, a.part_t + (size_t)b * KP);
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 2: pass B (rows k2 of this CTA); t = Rt^T q_j for columns b, b + G, ...
    {
      const int FB = a.FB, logFB = a.logN2 - (a.logN1 - a.logNB);   // FB = N2 / G
      const int k2_0 = b * FB;
      for (int t = tid; t < (a.N1 << logFB); t += SAMP_THREADS) {
        const int n1 = t & (a.N1 - 1), f = t >> a.logN1;
        x[(bitrev(n1, a.logN1) << logFB) + f] = __ldcg(a.work + (int64_t)(k2_0 + f) * a.N1 + n1);
      }
      __syncthreads();
      fft_dit(x, a.N1, logFB, wB, false);
      for (int t = tid; t < (a.N1 << logFB); t += SAMP_THREADS) {
        const int f = t & (FB - 1), k1 = t >> logFB;
        const double l = a.lam[(k2_0 + f) + a.N2 * k1];
        x[t].x *= l;
        x[t].y *= l;
      }
      __syncthreads();
      fft_dif(x, a.N1, logFB, wB, true);
      for (int t = tid; t < (a.N1 << logFB); t += SAMP_THREADS) {
        const int n1 = t & (a.N1 - 1), f = t >> a.logN1;
        __stcg(a.work + (int64_t)(k2_0 + f) * a.N1 + n1, x[(bitrev(n1, a.logN1) << logFB) + f]);
      }
    }
    for (int c = b + G * (tid >> 5); c < a.k && (tid >> 5) < SAMP_WARPS; c += G * SAMP_WARPS) {
      // warp (tid >> 5) adds column c's partials over the CTAs: lane l those of
      // CTAs l, l + 32, ..., then a fixed df butterfly across the lanes
      const int lane = tid & 31;
      df acc{0.f, 0.f};
      for (int bb = lane; bb < G; bb += 32) {
        const float2 p = __ldcg(a.part_t + (size_t)bb * KP + c);
        acc = df_add(acc, df{p.x, p.y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, acc.hi, o), l = __shfl_xor_sync(0xffffffffu, acc.lo, o);
        acc = df_add(acc, df{h, l});
      }
      if (lane == 0) __stcg(a.tvec + c, (double)acc.hi + (double)acc.lo);
    }
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 3: pass C -> K_UU q_j on own rows; v = K_UU q_j - Rt t; partials of c1
    for (int c = tid; c < a.k; c += SAMP_THREADS) tv[c] = __ldcg(a.tvec + c);
    for (int t = tid; t < (a.N2 << a.logNB); t += SAMP_THREADS) {
      const int f = t & (NB - 1), k2 = t >> a.logNB;
      const int n1 = n1_0 + f;
      double2 w = a.tw[((int64_t)n1 * k2) & (a.N - 1)];
      w.y = -w.y;
      x[t] = cmul(__ldcg(a.work + (int64_t)k2 * a.N1 + n1), w);
    }
    __syncthreads();
    fft_dif(x, a.N2, a.logNB, wA, true);
    for (int lr = tid; lr < RL; lr += SAMP_THREADS) {
      const int f = lr / R2, n2 = lr - f * R2;
      const int r = n1_0 + f + a.N1 * n2;
      kq[lr] = r < a.m ? x[(bitrev(n2, a.logN2) << a.logNB) + f].x : 0.0;
    }
    __syncthreads();
    rows_sub(Rs, RL, a.k, tv, kq, v, scratch);
    cols_dot(Qs, RL, j + 1, v, a.part_c1 + (size_t)b * KP);
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 4: c1; alpha_j; v -= Q_j c1; partials of c2
    reduce_parts(a.part_c1, G, j + 1, cvec, reinterpret_cast<float2*>(scratch));
    const double alpha_j = cvec[j];
    rows_sub(Qs, RL, j + 1, cvec, v, v, scratch);
    cols_dot(Qs, RL, j + 1, v, a.part_c2 + (size_t)b * KP);
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- 5: c2; v -= Q_j c2; partial of |v|^2
    reduce_parts(a.part_c2, G, j + 1, cvec, reinterpret_cast<float2*>(scratch));
    rows_sub(Qs, RL, j + 1, cvec, v, v, scratch);
    {
      const int lane = tid & 31, w = tid >> 5;
      double s = 0.0;
      for (int lr = tid; lr < RL; lr += SAMP_THREADS) s = fma(v[lr], v[lr], s);
      s = warp_sum(s);
      if (lane == 0) scratch[w] = s;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < SAMP_WARPS; ++q) t += scratch[q];
        __stcg(a.part_nn + b, t);
      }
    }
    if (!grid_barrier(a.gs, gen, a.status)) return;
    // ---- beta_j and the stop rule (identical in every CTA)
    if (tid < 32) {
      double nn = 0.0;
      for (int bb = tid; bb < G; bb += 32) nn += __ldcg(a.part_nn + bb);
      nn = warp_sum(nn);
      if (tid == 0) scratch[0] = nn;
    }
    __syncthreads();
    if (tid == 0) {
      const double beta_j = sqrt(scratch[0]);
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
  return sizeof(double2) * ((size_t)N / G + N2 / 2 + N1 / 2) +
         sizeof(double) * (SCRATCH + 2 * (size_t)KP + 2 * (size_t)RL + (size_t)(ks + k) * RL);
}

}  // namespace

template <typename T>
love_status sampler_lanczos_fused(const GridHost& gh, const FftPlan* fft, const Allocator& al, const T* Rt,
                                  int64_t ldr, int k, int ks, uint64_t seed, double tau, double* Q, int64_t ldq,
                                  double* alpha_h, double* beta_h, int* ks_eff, DevStatus* status, cudaStream_t s) {
  if (gh.dim != 1 || gh.additive) return LOVE_ERR_UNSUPPORTED;
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

  // work: N complex | 3 G KP partials | G | k | ks alpha | ks beta | k_eff | GridSync
  const size_t off_part = sizeof(double2) * (size_t)N;
  const size_t n_dbl = 3 * (size_t)G * KP + G + KP + 2 * (size_t)KP;
  const size_t off_int = off_part + sizeof(double) * n_dbl;
  const size_t bytes = off_int + 64 + sizeof(GridSync);
  char* w = (char*)al.alloc(bytes, s);
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
  a.tw = (const double2*)p.tw_d;
  a.lam = (const double*)p.lam_d;
  a.work = (double2*)w;
  double* d = (double*)(w + off_part);
  a.part_t = reinterpret_cast<float2*>(d);   // a float2 is one double's bytes
  a.part_c1 = a.part_t + (size_t)G * KP;
  a.part_c2 = a.part_c1 + (size_t)G * KP;
  a.part_nn = d + 3 * (size_t)G * KP;
  a.tvec = a.part_nn + G;
  a.alpha = a.tvec + KP;
  a.beta = a.alpha + KP;
  a.k_eff = (int*)(w + off_int);
  a.gs = (GridSync*)(w + off_int + 64);
  a.seed = seed;
  a.tau = tau;
  a.status = status;
  // rows m .. ldq of Q' are not written: the root kernels read rows below m only
  love_status rc = cuda_check(cudaMemsetAsync(w + off_int, 0, 64 + sizeof(GridSync), s));
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
  al.free(w, bytes, s);
  if (rc != LOVE_OK) return rc;
  if (gsh.abort) return LOVE_ERR_TIMEOUT;   // a grid barrier gave up waiting
  *ks_eff = keff;
  return LOVE_OK;
}

template love_status sampler_lanczos_fused<float>(const GridHost&, const FftPlan*, const Allocator&, const float*,
                                                  int64_t, int, int, uint64_t, double, double*, int64_t, double*,
                                                  double*, int*, DevStatus*, cudaStream_t);
template love_status sampler_lanczos_fused<double>(const GridHost&, const FftPlan*, const Allocator&, const double*,
                                                   int64_t, int, int, uint64_t, double, double*, int64_t, double*,
                                                   double*, int*, DevStatus*, cudaStream_t);

}  // namespace love
