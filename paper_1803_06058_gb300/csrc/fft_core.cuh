// fft_core.cuh -- radix-2 FFT passes on shared-memory arrays, shared by the
// K_UU products (k_fft.cu) and the persistent grid-space CG (k_lanczos.cu).
#pragma once

#include "love_internal.cuh"

namespace love {
namespace fftcore {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

__device__ __forceinline__ int bitrev(int i, int logL) { return (int)(__brev((unsigned)i) >> (32 - logL)); }

// twiddles of one transform length L, staged in shared memory: w[j] = W_L^j
// (j < L/2) taken from the master table W_N^j; a CTA loads them once and
// every butterfly stage reads them from shared memory
template <typename C>
__device__ __forceinline__ void load_twiddles(C* w, int L, const C* __restrict__ tw, int N) {
  const int step = N / L;
  for (int j = threadIdx.x; j < (L >> 1); j += blockDim.x) w[j] = tw[(int64_t)j * step];
}

// F interleaved arrays x[i * F + f] of length L; decimation in time on
// bit-reversed input, natural-order output.  w: shared twiddles W_L^j.
template <typename C>
__device__ void fft_dit(C* x, int L, int logF, const C* w, bool inverse) {
  const int F = 1 << logF;
  const int work = (L >> 1) << logF;
  for (int half = 1; half < L; half <<= 1) {
    const int tws = L / (2 * half);
    for (int t = threadIdx.x; t < work; t += blockDim.x) {
      int f = t & (F - 1), b = t >> logF;
      int j = b & (half - 1);
      int i1 = ((b - j) << 1) + j, i2 = i1 + half;
      C wv = w[j * tws];
      if (inverse) wv.y = -wv.y;
      C a = x[(i1 << logF) + f];
      C c = cmul(x[(i2 << logF) + f], wv);
      x[(i1 << logF) + f] = cadd(a, c);
      x[(i2 << logF) + f] = csub(a, c);
    }
    __syncthreads();
  }
}
// decimation in frequency: natural-order input, bit-reversed output
template <typename C>
__device__ void fft_dif(C* x, int L, int logF, const C* w, bool inverse) {
  const int F = 1 << logF;
  const int work = (L >> 1) << logF;
  for (int half = L >> 1; half >= 1; half >>= 1) {
    const int tws = L / (2 * half);
    for (int t = threadIdx.x; t < work; t += blockDim.x) {
      int f = t & (F - 1), b = t >> logF;
      int j = b & (half - 1);
      int i1 = ((b - j) << 1) + j, i2 = i1 + half;
      C wv = w[j * tws];
      if (inverse) wv.y = -wv.y;
      C a = x[(i1 << logF) + f];
      C c = x[(i2 << logF) + f];
      x[(i1 << logF) + f] = cadd(a, c);
      x[(i2 << logF) + f] = cmul(csub(a, c), wv);
    }
    __syncthreads();
  }
}

// ---- double-float complex transforms --------------------------------------
// A complex value as four floats {re.hi, re.lo, im.hi, im.lo} (~48-bit
// mantissas, error-free transformations): the same radix-2 passes as above on
// the FP32 pipes, for parts whose FP64 rate is a small fraction of FP32.
struct dfc {
  float rh, rl, ih, il;
};
// a + b (Dekker: TwoSum of the high parts, the low parts added, renormalised)
__device__ __forceinline__ void dfs_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float s = ah + bh;
  const float bb = s - ah;
  const float e = (ah - (s - bb)) + (bh - bb) + al + bl;
  sh = s + e;
  sl = e - (sh - s);
}
// a * b - c * d, every product error-free in its high part
__device__ __forceinline__ void dfs_mulsub(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                           float dl, float& rh, float& rl) {
  const float p = ah * bh, pe = fmaf(ah, bh, -p);
  const float q = ch * dh, qe = fmaf(ch, dh, -q);
  const float s = p - q;
  const float bb = s - p;
  float e = (p - (s - bb)) + (-q - bb);
  e += (pe - qe) + (fmaf(ah, bl, al * bh) - fmaf(ch, dl, cl * dh));
  rh = s + e;
  rl = e - (rh - s);
}
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) {
  dfc r;
  dfs_add(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
  dfs_add(a.ih, a.il, b.ih, b.il, r.ih, r.il);
  return r;
}
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) {
  dfc r;
  dfs_add(a.rh, a.rl, -b.rh, -b.rl, r.rh, r.rl);
  dfs_add(a.ih, a.il, -b.ih, -b.il, r.ih, r.il);
  return r;
}
// a * w (w conjugated when conj)
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc w, bool conj) {
  const float wih = conj ? -w.ih : w.ih, wil = conj ? -w.il : w.il;
  dfc r;
  dfs_mulsub(a.rh, a.rl, w.rh, w.rl, a.ih, a.il, wih, wil, r.rh, r.rl);
  dfs_mulsub(a.rh, a.rl, wih, wil, -a.ih, -a.il, w.rh, w.rl, r.ih, r.il);
  return r;
}
__device__ __forceinline__ dfc dfc_from(double2 v) {
  dfc r;
  r.rh = (float)v.x;
  r.rl = (float)(v.x - (double)r.rh);
  r.ih = (float)v.y;
  r.il = (float)(v.y - (double)r.ih);
  return r;
}
// twiddles W_L^j (j < L/2) of the FP64 master table W_N^j, as df complex
__device__ __forceinline__ void load_twiddles_df(dfc* w, int L, const double2* __restrict__ tw, int N) {
  const int step = N / L;
  for (int j = threadIdx.x; j < (L >> 1); j += blockDim.x) w[j] = dfc_from(tw[(int64_t)j * step]);
}
// F interleaved arrays x[i * F + f] of length L: DIT on bit-reversed input,
// natural-order output (as fft_dit)
__device__ inline void fft_dit_df(dfc* x, int L, int logF, const dfc* w, bool inverse) {
  const int F = 1 << logF;
  const int work = (L >> 1) << logF;
  for (int half = 1; half < L; half <<= 1) {
    const int tws = L / (2 * half);
    for (int t = threadIdx.x; t < work; t += blockDim.x) {
      const int f = t & (F - 1), b = t >> logF;
      const int j = b & (half - 1);
      const int i1 = ((b - j) << 1) + j, i2 = i1 + half;
      const dfc a = x[(i1 << logF) + f];
      const dfc c = dfc_mul(x[(i2 << logF) + f], w[j * tws], inverse);
      x[(i1 << logF) + f] = dfc_add(a, c);
      x[(i2 << logF) + f] = dfc_sub(a, c);
    }
    __syncthreads();
  }
}
// DIF: natural-order input, bit-reversed output (as fft_dif)
__device__ inline void fft_dif_df(dfc* x, int L, int logF, const dfc* w, bool inverse) {
  const int F = 1 << logF;
  const int work = (L >> 1) << logF;
  for (int half = L >> 1; half >= 1; half >>= 1) {
    const int tws = L / (2 * half);
    for (int t = threadIdx.x; t < work; t += blockDim.x) {
      const int f = t & (F - 1), b = t >> logF;
      const int j = b & (half - 1);
      const int i1 = ((b - j) << 1) + j, i2 = i1 + half;
      const dfc a = x[(i1 << logF) + f];
      const dfc c = x[(i2 << logF) + f];
      x[(i1 << logF) + f] = dfc_add(a, c);
      x[(i2 << logF) + f] = dfc_mul(dfc_sub(a, c), w[j * tws], inverse);
    }
    __syncthreads();
  }
}

}  // namespace fftcore
}  // namespace love
