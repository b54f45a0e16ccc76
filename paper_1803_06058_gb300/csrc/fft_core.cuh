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


}  // namespace fftcore
}  // namespace love
