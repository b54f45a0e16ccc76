// k_fft.cu -- K_UU matrix-vector products by FFT (Sec. 2.3: a regular grid makes
// K_UU Toeplitz, or a Kronecker product of Toeplitz factors, so K_UU v costs
// O(m log m)).
//
// Each factor T_e (g x g, symmetric Toeplitz, first column c) is embedded in a
// circulant of power-of-two length N >= 2g - 1 whose first column is
// c[0..g-1], zeros, c[g-1..1].  T_e v = first g entries of
// IFFT(lambda .* FFT([v; 0])) with lambda = FFT(circulant column), real because
// the column is symmetric.  A Kronecker K_UU applies one such product per mode
// to every fibre of that mode.
//
// Two kernel shapes:
//   * short modes (N <= 4096): one CTA transforms F fibres entirely in shared
//     memory (DIT forward on bit-reversed input, pointwise lambda, DIF inverse
//     giving bit-reversed output) -- one launch per mode.
//   * long modes: the four-step split N = N1 N2 in three launches:
//     A  length-N2 FFTs over n2 for each n1, times the twiddle W_N^{n1 k2}
//     B  length-N1 FFTs over n1 for each k2, times lambda, inverse length-N1 FFTs
//     C  conjugate twiddles, inverse length-N2 FFTs, real part, crop to g.
// The twiddle table W_N^j and lambda are computed once per grid in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "love_internal.cuh"
#include "fft_core.cuh"

namespace love {
namespace {
using namespace fftcore;

// address of element i of fibre `fid` of column `col` along mode e
struct ModeGeom {
  int64_t g;        // length of the mode
  int64_t stride;   // stride of the mode
  int64_t nfib;     // fibres per column = m / g
  int64_t ldc;      // column stride
  __device__ __forceinline__ int64_t offset(int64_t col, int64_t fid, int64_t i) const {
    int64_t outer = fid / stride, inner = fid - outer * stride;
    return col * ldc + outer * (g * stride) + i * stride + inner;
  }
};

// ----- short modes: whole transform in shared memory -----------------------
template <typename IO, typename R>
__global__ void k_toep_small(const IO* __restrict__ in, IO* __restrict__ out, ModeGeom mg, int64_t total_fib,
                             int N, int logN, int logF, const typename Cplx<R>::type* __restrict__ tw,
                             const R* __restrict__ lam) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const int F = 1 << logF;
  C* w = x + ((size_t)N << logF);   // [N / 2] twiddles
  load_twiddles(w, N, tw, N);
  const int64_t fib0 = (int64_t)blockIdx.x * F;
  // load (fibre fastest), zero padded, into bit-reversed slots
  for (int t = threadIdx.x; t < (N << logF); t += blockDim.x) {
    int f = t & (F - 1), i = t >> logF;
    int64_t fb = fib0 + f;
    R v = R(0);
    if (i < mg.g && fb < total_fib) {
      int64_t col = fb / mg.nfib, fid = fb - col * mg.nfib;
      v = (R)in[mg.offset(col, fid, i)];
    }
    C c;
    c.x = v;
    c.y = R(0);
    x[(bitrev(i, logN) << logF) + f] = c;
  }
  __syncthreads();
  fft_dit(x, N, logF, w, false);
  for (int t = threadIdx.x; t < (N << logF); t += blockDim.x) {
    int i = t >> logF;
    R l = lam[i];
    x[t].x *= l;
    x[t].y *= l;
  }
  __syncthreads();
  fft_dif(x, N, logF, w, true);
  for (int t = threadIdx.x; t < (N << logF); t += blockDim.x) {
    int f = t & (F - 1), i = t >> logF;
    int64_t fb = fib0 + f;
    if (i < mg.g && fb < total_fib) {
      int64_t col = fb / mg.nfib, fid = fb - col * mg.nfib;
      out[mg.offset(col, fid, i)] = (IO)x[(bitrev(i, logN) << logF) + f].x;
    }
  }
}

// ----- long modes: four-step -------------------------------------------------
// A: for each n1 in a group of FA, FFT over n2 of x[n1 + N1 n2], times W_N^{n1 k2};
//    work[fb][k2 * N1 + n1]
template <typename IO, typename R>
__global__ void k_four_a(const IO* __restrict__ in, typename Cplx<R>::type* __restrict__ work, ModeGeom mg,
                         int N, int N1, int N2, int logN2, int logFA,
                         const typename Cplx<R>::type* __restrict__ tw) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const int FA = 1 << logFA;
  C* w = x + ((size_t)N2 << logFA);   // [N2 / 2] twiddles
  load_twiddles(w, N2, tw, N);
  const int n1_0 = blockIdx.x * FA;
  const int64_t fb = blockIdx.y;
  const int64_t col = fb / mg.nfib, fid = fb - col * mg.nfib;
  for (int t = threadIdx.x; t < (N2 << logFA); t += blockDim.x) {
    int f = t & (FA - 1), n2 = t >> logFA;
    int64_t idx = (int64_t)(n1_0 + f) + (int64_t)N1 * n2;
    C c;
    c.x = R(0);
    c.y = R(0);
    if (idx < mg.g) c.x = (R)in[mg.offset(col, fid, idx)];
    x[(bitrev(n2, logN2) << logFA) + f] = c;
  }
  __syncthreads();
  fft_dit(x, N2, logFA, w, false);
  C* wdst = work + fb * (int64_t)N;
  for (int t = threadIdx.x; t < (N2 << logFA); t += blockDim.x) {
    int f = t & (FA - 1), k2 = t >> logFA;
    int n1 = n1_0 + f;
    C v = x[t];
    C w = tw[((int64_t)n1 * k2) & (N - 1)];
    wdst[(int64_t)k2 * N1 + n1] = cmul(v, w);
  }
}

// B: for each k2 in a group of FB rows: FFT over n1, times lambda, inverse FFT
//    over k1 (or, with lam == nullptr, write X[k2 + N2 k1] to xout).
template <typename R>
__global__ void k_four_b(typename Cplx<R>::type* __restrict__ work, int N, int N1, int N2, int logN1, int logFB,
                         const typename Cplx<R>::type* __restrict__ tw, const R* __restrict__ lam,
                         typename Cplx<R>::type* __restrict__ xout) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const int FB = 1 << logFB;
  C* w = x + ((size_t)N1 << logFB);   // [N1 / 2] twiddles
  load_twiddles(w, N1, tw, N);
  const int k2_0 = blockIdx.x * FB;
  const int64_t fb = blockIdx.y;
  C* wrow = work + fb * (int64_t)N;
  // load row-major (n1 fastest) for coalescing; store transposed in smem
  for (int t = threadIdx.x; t < (N1 << logFB); t += blockDim.x) {
    int n1 = t & (N1 - 1), f = t >> logN1;
    x[(bitrev(n1, logN1) << logFB) + f] = wrow[(int64_t)(k2_0 + f) * N1 + n1];
  }
  __syncthreads();
  fft_dit(x, N1, logFB, w, false);
  if (lam == nullptr) {
    for (int t = threadIdx.x; t < (N1 << logFB); t += blockDim.x) {
      int f = t & (FB - 1), k1 = t >> logFB;
      xout[fb * (int64_t)N + (int64_t)(k2_0 + f) + (int64_t)N2 * k1] = x[t];
    }
    return;
  }
  for (int t = threadIdx.x; t < (N1 << logFB); t += blockDim.x) {
    int f = t & (FB - 1), k1 = t >> logFB;
    R l = lam[(k2_0 + f) + N2 * k1];
    x[t].x *= l;
    x[t].y *= l;
  }
  __syncthreads();
  fft_dif(x, N1, logFB, w, true);
  for (int t = threadIdx.x; t < (N1 << logFB); t += blockDim.x) {
    int n1 = t & (N1 - 1), f = t >> logN1;
    wrow[(int64_t)(k2_0 + f) * N1 + n1] = x[(bitrev(n1, logN1) << logFB) + f];
  }
}

// C: for each n1 in a group of FA: conjugate twiddle, inverse FFT over k2,
//    real part of x[n1 + N1 n2] cropped to the mode length.
template <typename IO, typename R>
__global__ void k_four_c(const typename Cplx<R>::type* __restrict__ work, IO* __restrict__ out, ModeGeom mg, int N,
                         int N1, int N2, int logN2, int logFA, const typename Cplx<R>::type* __restrict__ tw) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const int FA = 1 << logFA;
  C* w = x + ((size_t)N2 << logFA);   // [N2 / 2] twiddles
  load_twiddles(w, N2, tw, N);
  const int n1_0 = blockIdx.x * FA;
  const int64_t fb = blockIdx.y;
  const int64_t col = fb / mg.nfib, fid = fb - col * mg.nfib;
  const C* wsrc = work + fb * (int64_t)N;
  for (int t = threadIdx.x; t < (N2 << logFA); t += blockDim.x) {
    int f = t & (FA - 1), k2 = t >> logFA;
    int n1 = n1_0 + f;
    C w = tw[((int64_t)n1 * k2) & (N - 1)];
    w.y = -w.y;
    x[t] = cmul(wsrc[(int64_t)k2 * N1 + n1], w);
  }
  __syncthreads();
  fft_dif(x, N2, logFA, w, true);
  for (int t = threadIdx.x; t < (N2 << logFA); t += blockDim.x) {
    int f = t & (FA - 1), n2 = t >> logFA;
    int64_t idx = (int64_t)(n1_0 + f) + (int64_t)N1 * n2;
    if (idx < mg.g) out[mg.offset(col, fid, idx)] = (IO)x[(bitrev(n2, logN2) << logFA) + f].x;
  }
}

// ----- short modes: dense double-float product ------------------------------
// out[f, i] = sum_j c[|i - j|] x[f, j] for TF fibres per CTA (every output i
// of them, so a product in place is safe): the fibres' inputs, the column of
// T (float pairs) and the outputs in shared memory; thread t takes the outputs
// i = i0 + t % 64 (i0 = 0, 64, ...) of TF / 4 fibres.  Products and sums in
// double-float (two FP32 words, ~2^-46 relative per operation): the FP32
// pipes run this several times faster than an FP64 FFT of the same mode.
__device__ __forceinline__ void df_mac(float& s, float& t, float ch, float cl, float xh, float xl) {
  const float p = ch * xh;
  float e = fmaf(ch, xh, -p);
  e = fmaf(ch, xl, e);
  e = fmaf(cl, xh, e);
  const float s2 = s + p;
  const float bb = s2 - s;
  t += ((s - (s2 - bb)) + (p - bb)) + e;
  s = s2;
}

template <typename IO, int TF>
__global__ void __launch_bounds__(256) k_toep_dense(const IO* __restrict__ in, IO* __restrict__ out, ModeGeom mg,
                                                    int64_t total_fib, const float2* __restrict__ col) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = (int)mg.g;
  float2* cs = reinterpret_cast<float2*>(smem_raw);   // [g]
  float2* xs = cs + g;                                 // [TF][g] inputs
  float2* ys = xs + (size_t)TF * g;                    // [TF][g] outputs
  const int64_t fib0 = (int64_t)blockIdx.x * TF;
  for (int r = threadIdx.x; r < g; r += blockDim.x) cs[r] = col[r];
  // inputs: i fastest along a unit-stride mode, the fibre fastest otherwise
  const bool unit = mg.stride == 1;
  for (int t = threadIdx.x; t < TF * g; t += blockDim.x) {
    const int f = unit ? t / g : t % TF;
    const int i = unit ? t % g : t / TF;
    const int64_t fb = fib0 + f;
    double v = 0.0;
    if (fb < total_fib) {
      const int64_t c = fb / mg.nfib, fid = fb - c * mg.nfib;
      v = (double)in[mg.offset(c, fid, i)];
    }
    const float h = (float)v;
    xs[f * g + i] = make_float2(h, (float)(v - (double)h));
  }
  __syncthreads();
  constexpr int NF = TF / 4;
  const int fq = threadIdx.x >> 6;   // 4 groups of NF fibres
  for (int i0 = 0; i0 < g; i0 += 64) {
    const int i = i0 + (threadIdx.x & 63);
    if (i >= g) continue;
    float s[NF], t[NF];
#pragma unroll
    for (int u = 0; u < NF; ++u) s[u] = t[u] = 0.f;
    for (int j = 0; j < g; ++j) {
      const float2 c = cs[i > j ? i - j : j - i];
#pragma unroll
      for (int u = 0; u < NF; ++u) {
        const float2 x = xs[(fq * NF + u) * g + j];
        df_mac(s[u], t[u], c.x, c.y, x.x, x.y);
      }
    }
#pragma unroll
    for (int u = 0; u < NF; ++u) ys[(fq * NF + u) * g + i] = make_float2(s[u], t[u]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TF * g; t += blockDim.x) {
    const int f = unit ? t / g : t % TF;
    const int i = unit ? t % g : t / TF;
    const int64_t fb = fib0 + f;
    if (fb < total_fib) {
      const int64_t c = fb / mg.nfib, fid = fb - c * mg.nfib;
      const float2 v = ys[f * g + i];
      out[mg.offset(c, fid, i)] = (IO)((double)v.x + (double)v.y);
    }
  }
}

template <typename IO, int TF>
love_status toep_dense_launch(const FftPlan& p, const IO* in, IO* out, ModeGeom mg, int64_t total, bool deriv,
                              cudaStream_t s) {
  const size_t sm = sizeof(float2) * (size_t)p.g * (1 + 2 * TF);
  LOVE_TRY(allow_smem(k_toep_dense<IO, TF>, sm));
  LOVE_COUNT_LAUNCH();
  k_toep_dense<IO, TF><<<(unsigned)((total + TF - 1) / TF), 256, sm, s>>>(
      in, out, mg, total, (const float2*)(deriv ? p.coldl2 : p.col2));
  return cuda_check(cudaGetLastError());
}

// ----- plan set-up kernels ---------------------------------------------------
__global__ void k_twiddles(double2* tw_d, float2* tw_f, int64_t N) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)N, &s, &c);
  tw_d[j] = make_double2(c, s);
  tw_f[j] = make_float2((float)c, (float)s);
}
// embedded circulant column of T_e (or dT_e/dl), times `scale`
__global__ void k_embed_column(double2* out, int64_t N, int64_t g, double h, double ls, double scale, int deriv) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  int64_t r = j < g ? j : (N - j < g ? N - j : -1);
  double v = 0.0;
  if (r >= 0) {
    double d = (double)r * h;
    v = scale * exp(-(d * d) / (2.0 * ls * ls));
    if (deriv) v *= d * d / (ls * ls * ls);
  }
  out[j] = make_double2(v, 0.0);
}
__global__ void k_lambda_store(const double2* X, int64_t N, double* lam_d, float* lam_f) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double v = X[j].x / (double)N;
  lam_d[j] = v;
  lam_f[j] = (float)v;
}

inline int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

constexpr int SMALL_MAX_N = 4096;

// FFTs per CTA in the four-step kernels: at most `cap` complex values per CTA
// and at most 16 transforms
// Transforms per CTA in the four-step kernels: at most `cap` complex values
// per CTA and at most 16 transforms, but few enough that the launch has
// >= 2 CTAs per SM (FP64 throughput per SM is low on this part, so the
// transforms must be spread over the whole GPU).  `count` = transforms in the launch.
inline int four_logF(int L, int cap, int64_t count) {
  int64_t want = count / (2 * (int64_t)num_sms());
  int F = (int)std::max<int64_t>(1, std::min<int64_t>({16, (int64_t)(cap / L), want}));
  int l = 0;
  while ((2 << l) <= F) ++l;
  return l;
}


template <typename R>
int small_logF(int N, int64_t total) {
  // total complex elements per CTA: 4096 (FP32, 32 KB) / 2048 (FP64, 32 KB),
  // and at least 2 CTAs per SM when there are enough fibres
  int cap = sizeof(R) == 4 ? 4096 : 2048;
  int64_t want = std::max<int64_t>(1, total / (2 * (int64_t)num_sms()));
  int F = (int)std::max<int64_t>(1, std::min<int64_t>(cap / N, want));
  int l = 0;
  while ((2 << l) <= F) ++l;
  return l;
}

// One mode of K_UU applied to FP32 or FP64 data.  The transform runs in R =
// FP64 (twiddles and lambda in FP64): K_UU is m-sized, so this costs little,
// and it keeps the Toeplitz product accurate to the rounding of its inputs and
// outputs (an FP32 transform of length N carries ~log2(N) 2^-24).
template <typename IO, typename R>
love_status toeplitz_mode(const FftPlan& p, const IO* in, IO* out, ModeGeom mg, int ncol, void* work,
                          bool deriv, cudaStream_t s) {
  using C = typename Cplx<R>::type;
  if (p.col2 != nullptr && p.g <= TOEP_DENSE_MAX) {
    // 16 fibres per CTA while that still gives two CTAs per SM, else 4
    const int64_t total = mg.nfib * ncol;
    if (total >= 16 * 2 * (int64_t)num_sms()) return toep_dense_launch<IO, 16>(p, in, out, mg, total, deriv, s);
    return toep_dense_launch<IO, 4>(p, in, out, mg, total, deriv, s);
  }
  const bool dbl = sizeof(R) == 8;
  const C* tw = (const C*)(dbl ? p.tw_d : p.tw_f);
  const R* lam = (const R*)(deriv ? (dbl ? p.lamdl_d : p.lamdl_f) : (dbl ? p.lam_d : p.lam_f));
  const int N = (int)p.N;
  const int64_t total = mg.nfib * ncol;
  if (p.N2 == 1) {
    int logF = small_logF<R>(N, total);
    int F = 1 << logF;
    size_t sm = ((size_t)N * F + N / 2) * sizeof(C);
    int threads = std::min(512, std::max(64, (N * F) / 4));
    int64_t blocks = (total + F - 1) / F;
    LOVE_TRY(allow_smem(k_toep_small<IO, R>, sm));
    LOVE_COUNT_LAUNCH(); k_toep_small<IO, R><<<(unsigned)blocks, threads, sm, s>>>(in, out, mg, total, N, ilog2(N), logF, tw, lam);
    return cuda_check(cudaGetLastError());
  }
  const int N1 = p.N1, N2 = p.N2;
  C* wk = (C*)work;
  const int cap = 2048;
  int logFA = four_logF(N2, cap, (int64_t)N1 * total);
  int FA = 1 << logFA;
  int logFB = four_logF(N1, cap, (int64_t)N2 * total);
  int FB = 1 << logFB;
  dim3 ga(N1 / FA, (unsigned)total), gb(N2 / FB, (unsigned)total);
  size_t sma = ((size_t)N2 * FA + N2 / 2) * sizeof(C), smb = ((size_t)N1 * FB + N1 / 2) * sizeof(C);
  LOVE_TRY(allow_smem(k_four_a<IO, R>, sma));
  LOVE_TRY(allow_smem(k_four_b<R>, smb));
  LOVE_TRY(allow_smem(k_four_c<IO, R>, sma));
  LOVE_COUNT_LAUNCH(); k_four_a<IO, R><<<ga, 256, sma, s>>>(in, wk, mg, N, N1, N2, ilog2(N2), logFA, tw);
  LOVE_COUNT_LAUNCH(); k_four_b<R><<<gb, 256, smb, s>>>(wk, N, N1, N2, ilog2(N1), logFB, tw, lam, nullptr);
  LOVE_COUNT_LAUNCH(); k_four_c<IO, R><<<ga, 256, sma, s>>>(wk, out, mg, N, N1, N2, ilog2(N2), logFA, tw);
  return cuda_check(cudaGetLastError());
}

// forward FFT (FP64) of `src` (N complex, N <= 4096) into `dst`: one CTA runs
// the DIT transform of k_four_b with N1 = N, N2 = 1 in forward-only mode.
love_status fft_forward_small_f64(const FftPlan& p, const double2* src, double2* dst, double2* work,
                                  cudaStream_t s) {
  const int N = (int)p.N;
  cudaError_t e = cudaMemcpyAsync(work, src, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_check(e);
  size_t sm = ((size_t)N + N / 2) * sizeof(double2);
  LOVE_TRY(allow_smem(k_four_b<double>, sm));
  LOVE_COUNT_LAUNCH(); k_four_b<double><<<dim3(1, 1), 256, sm, s>>>(work, N, N, 1, ilog2(N), 0, (const double2*)p.tw_d, nullptr, dst);
  return cuda_check(cudaGetLastError());
}

__global__ void k_real_part(const double2* a, double* out, int64_t N) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < N) out[j] = a[j].x;
}

}  // namespace

love_status fft_plan_create(FftPlan& p, const GridHost& g, int e, const Allocator& al, cudaStream_t s,
                            bool dense) {
  p.g = g.g[e];
  int64_t N = 4;
  while (N < 2 * p.g - 1) N <<= 1;
  p.N = N;
  if (N <= SMALL_MAX_N) {
    p.N1 = (int)N;
    p.N2 = 1;
  } else {
    int l = ilog2(N);
    p.N1 = 1 << (l / 2);
    p.N2 = (int)(N >> (l / 2));
  }
  if (N > (int64_t(1) << 22)) return LOVE_ERR_UNSUPPORTED;
  p.tw_d = al.alloc(sizeof(double2) * N, s);
  p.tw_f = al.alloc(sizeof(float2) * N, s);
  p.lam_d = al.alloc(sizeof(double) * N, s);
  p.lam_f = al.alloc(sizeof(float) * N, s);
  p.lamdl_d = al.alloc(sizeof(double) * N, s);
  p.lamdl_f = al.alloc(sizeof(float) * N, s);
  double2* col = (double2*)al.alloc(sizeof(double2) * N, s);
  double2* X = (double2*)al.alloc(sizeof(double2) * N, s);
  double2* wk = (double2*)al.alloc(sizeof(double2) * N, s);
  double* re = (double*)al.alloc(sizeof(double) * N, s);
  if (!p.tw_d || !p.tw_f || !p.lam_d || !p.lam_f || !p.lamdl_d || !p.lamdl_f || !col || !X || !wk || !re)
    return LOVE_ERR_OOM;
  int nb = ceil_div(N, 256);
  LOVE_COUNT_LAUNCH(); k_twiddles<<<nb, 256, 0, s>>>((double2*)p.tw_d, (float2*)p.tw_f, N);
  for (int deriv = 0; deriv < 2; ++deriv) {
    double scale = (e == 0 || g.additive) ? g.sf : 1.0;   // s_f in every block of an additive K_UU
    LOVE_COUNT_LAUNCH(); k_embed_column<<<nb, 256, 0, s>>>(col, N, p.g, g.h[e], g.ls[e], scale, deriv);
    if (p.N2 == 1) {
      LOVE_TRY(fft_forward_small_f64(p, col, X, wk, s));
    } else {
      // four-step forward with a real input: A (reads real parts) then B (forward only)
      LOVE_COUNT_LAUNCH(); k_real_part<<<nb, 256, 0, s>>>(col, re, N);
      ModeGeom mg{N, 1, 1, N};
      int logFA = four_logF(p.N2, 2048, p.N1);
      int logFB = four_logF(p.N1, 2048, p.N2);
      dim3 ga(p.N1 >> logFA, 1), gb(p.N2 >> logFB, 1);
      LOVE_COUNT_LAUNCH(); k_four_a<double, double><<<ga, 256, ((size_t)p.N2 * (1 << logFA) + p.N2 / 2) * sizeof(double2), s>>>(
          re, wk, mg, (int)N, p.N1, p.N2, ilog2(p.N2), logFA, (const double2*)p.tw_d);
      LOVE_COUNT_LAUNCH(); k_four_b<double><<<gb, 256, ((size_t)p.N1 * (1 << logFB) + p.N1 / 2) * sizeof(double2), s>>>(
          wk, (int)N, p.N1, p.N2, ilog2(p.N1), logFB, (const double2*)p.tw_d, nullptr, X);
    }
    LOVE_COUNT_LAUNCH(); k_lambda_store<<<nb, 256, 0, s>>>(X, N, (double*)(deriv ? p.lamdl_d : p.lam_d),
                                      (float*)(deriv ? p.lamdl_f : p.lam_f));
  }
  LOVE_TRY(cuda_check(cudaGetLastError()));
  if (dense && p.g <= TOEP_DENSE_MAX) {
    // first columns of T_e and dT_e/dl for the dense product, as float pairs
    const double scale = (e == 0 || g.additive) ? g.sf : 1.0;
    std::vector<float2> hc((size_t)p.g), hd((size_t)p.g);
    for (int64_t r = 0; r < p.g; ++r) {
      const double d = (double)r * g.h[e];
      const double v = scale * std::exp(-(d * d) / (2.0 * g.ls[e] * g.ls[e]));
      const double vd = v * d * d / (g.ls[e] * g.ls[e] * g.ls[e]);
      const float vh = (float)v, dh = (float)vd;
      hc[(size_t)r] = make_float2(vh, (float)(v - (double)vh));
      hd[(size_t)r] = make_float2(dh, (float)(vd - (double)dh));
    }
    p.col2 = al.alloc(sizeof(float2) * p.g, s);
    p.coldl2 = al.alloc(sizeof(float2) * p.g, s);
    if (!p.col2 || !p.coldl2) return LOVE_ERR_OOM;
    LOVE_TRY(cuda_check(cudaMemcpyAsync(p.col2, hc.data(), sizeof(float2) * p.g, cudaMemcpyHostToDevice, s)));
    LOVE_TRY(cuda_check(cudaMemcpyAsync(p.coldl2, hd.data(), sizeof(float2) * p.g, cudaMemcpyHostToDevice, s)));
    LOVE_TRY(cuda_check(cudaStreamSynchronize(s)));   // the host columns go out of scope
  }
  al.free(col, sizeof(double2) * N, s);
  al.free(X, sizeof(double2) * N, s);
  al.free(wk, sizeof(double2) * N, s);
  al.free(re, sizeof(double) * N, s);
  return LOVE_OK;
}

void fft_plan_destroy(FftPlan& p, const Allocator& al, cudaStream_t s) {
  al.free(p.tw_d, sizeof(double2) * p.N, s);
  al.free(p.tw_f, sizeof(float2) * p.N, s);
  al.free(p.lam_d, sizeof(double) * p.N, s);
  al.free(p.lam_f, sizeof(float) * p.N, s);
  al.free(p.lamdl_d, sizeof(double) * p.N, s);
  al.free(p.lamdl_f, sizeof(float) * p.N, s);
  if (p.col2) al.free(p.col2, sizeof(float2) * p.g, s);
  if (p.coldl2) al.free(p.coldl2, sizeof(float2) * p.g, s);
  p = FftPlan{};
}

size_t fft_work_bytes(const GridHost& g, const FftPlan* plans, int ncol, bool dbl) {
  size_t best = 0;
  for (int e = 0; e < g.dim; ++e) {
    if (plans[e].N2 == 1) continue;
    (void)dbl;  // the transforms always run in FP64
    const size_t fibres = g.additive ? 1 : (size_t)(g.m / g.g[e]);
    size_t b = (size_t)plans[e].N * fibres * (size_t)ncol * 16;
    best = std::max(best, b);
  }
  return best;
}

template <typename T>
love_status kuu_apply(const GridHost& g, const FftPlan* plans, const T* v, T* out, int ncol, int64_t ldc,
                      void* work, int deriv_dim, cudaStream_t s) {
  if (g.additive) {
    // block-diagonal K_UU: one Toeplitz product per 1-D block
    for (int e = 0; e < g.dim; ++e) {
      ModeGeom mg{g.g[e], 1, 1, ldc};
      LOVE_TRY((toeplitz_mode<T, double>(plans[e], v + g.off[e], out + g.off[e], mg, ncol, work, e == deriv_dim, s)));
    }
    return LOVE_OK;
  }
  const T* src = v;
  for (int e = 0; e < g.dim; ++e) {
    ModeGeom mg{g.g[e], g.stride[e], g.m / g.g[e], ldc};
    LOVE_TRY((toeplitz_mode<T, double>(plans[e], src, out, mg, ncol, work, e == deriv_dim, s)));
    src = out;
  }
  return LOVE_OK;
}

template love_status kuu_apply<float>(const GridHost&, const FftPlan*, const float*, float*, int, int64_t, void*, int,
                                      cudaStream_t);
template love_status kuu_apply<double>(const GridHost&, const FftPlan*, const double*, double*, int, int64_t, void*,
                                       int, cudaStream_t);

}  // namespace love
