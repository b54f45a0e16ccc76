// k_mvm.cu -- the SKI product of a 1-D Lanczos step as ONE cooperative kernel:
//     y = W^T K_UU W q_j + s^2 q_j        (eq. ski; Algorithm 1's mvm_K_XX)
// and q_j normalised in place, for FP32 data on a 1-D grid (the product the
// multi-launch path forms with a cell-sorted scatter, three FP64 FFT launches
// and a gather).
//
// K_UU u is the circulant-embedding product of length N = N1 N2 in the
// four-step split of k_fft.cu (pass A: FFTs over n2 for each n1 with the
// twiddles W_N^{n1 k2}; pass B: FFTs over n1 for each k2, times lambda / N,
// inverse; pass C: conjugate twiddles, inverse FFTs over k2), here in
// double-float complex arithmetic (fft_core.cuh) on the FP32 pipes: this part
// runs FP64 at a small fraction of its FP32 rate, and ~48-bit mantissas keep
// the product far below the FP32 rounding of its result.
//
// CTA b owns the columns n1 in [b NB, (b+1) NB) of passes A and C and with them
// the grid nodes r = n1 + N1 n2 (r < m):
//   0  the CTA's contiguous range of nodes / cells [r0, r1): x and q_j of the
//      points of cells r0-2 .. r1 land in shared memory (bulk async copies);
//      u_r = scal_j sum_p w_p(r) q_p for r in [r0, r1), a warp per node over
//      the points of cells r-2 .. r+1 (double-float sums, fixed order), as df
//      pairs in global memory                                          | barrier
//   1  pass A on its nodes                                            | barrier
//   2  pass B on the rows k2 in [b FB, (b+1) FB)                      | barrier
//   3  pass C -> (K_UU u)_r for its nodes, rounded to FP32 in global | barrier
//   4  the points of cells [r0, r1) (still in shared memory), with (K_UU u) of
//      nodes r0-1 .. r1 staged: q_p <- scal_j q_p,
//      y_p = sum_r w_r(p) (K_UU u)_r + s^2 q_p  (FP32, as the gather kernel).
// HBM sees each point's x and q once and q, y written once per product.
// Nothing runs after a Lanczos breakdown (the done flag).  The barriers are
// bounded (love_internal.cuh); their counters persist across the steps of a
// run, the caller passing the count already completed (4 per product).
#include <algorithm>
#include <cmath>

#include "love_internal.cuh"
#include "fft_core.cuh"

namespace love {
namespace {
using namespace fftcore;

constexpr int MVM_THREADS = 512;
constexpr int MVM_WARPS = MVM_THREADS / 32;
// points of a CTA's cells (with a 2-cell halo) staged in shared memory: x and
// q_j, 96 KB; a CTA whose cells hold more reads them from global memory
constexpr int STAGE_CAP = 12288;

struct MvmArgs {
  GridDev g;
  int m;
  int64_t n, n_pad;
  const float* xs;          // cell-sorted training coordinates (n_pad)
  const int* cell_start;    // m + 1
  float* q;                 // q_j, unnormalised: scaled in place
  const double* scal;       // 1 / |q_j|
  const int* done;          // the Lanczos run has stopped
  float noise;
  float* y;                 // n_pad
  float* ku;                // m: K_UU u, FP32
  float2* u;                // m: W q_j as df pairs
  int N, N1, N2, logN1, logN2, logNB, logFB, NB, FB, R2;
  const float4* twdf;       // W_N^j as df complex (converted once per run)
  const float2* lamdf;      // spectrum / N as df pairs
  dfc* work;                // N df complex
  unsigned int gen0;        // barriers already completed on gs
  GridSync* gs;
  DevStatus* status;
};

// weight of a cell-sorted point at node r (the arithmetic of the scatter kernels)
__device__ __forceinline__ float node_weight_1d(float x, const GridDev& g, int node) {
  const float s = grid_coord(x, g, 0);
  int i = (int)floorf(s);
  if (i > g.g[0] - 3) i = g.g[0] - 3;
  const float f = s - (float)i;
  const int r = node - (i - 1);
  return keys_u(f + 1.f - (float)r);
}

__global__ void __launch_bounds__(MVM_THREADS, 1) k_ski_mvm_1d(const __grid_constant__ MvmArgs a) {
  if (*a.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NB = a.NB, R2 = a.R2, RL = NB * R2;
  const int n1_0 = b * NB;
  // shared memory: x [N / G], wA [N2 / 2], wB [N1 / 2] (df complex), then the
  // staged points xsm, qsm [STAGE_CAP], the node sums us [RL] (df pairs) and
  // the staged K_UU u [per + 3]
  dfc* x = reinterpret_cast<dfc*>(smem_raw);
  dfc* wA = x + a.N / G;
  dfc* wB = wA + a.N2 / 2;
  float* xsm = reinterpret_cast<float*>(wB + a.N1 / 2);
  float* qsm = xsm + STAGE_CAP;
  float2* us = reinterpret_cast<float2*>(qsm + STAGE_CAP);
  float* kus = reinterpret_cast<float*>(us + RL);
  int* css = reinterpret_cast<int*>(kus + ((a.m + G - 1) / G + 4));   // cell_start[r0 - 2 .. r1 + 2]
  __shared__ uint64_t bar;
  unsigned int gen = a.gen0;
  const double sc = *a.scal;
  // this CTA's nodes / cells [r0, r1) and the staged point range [P0a, P1a)
  const int per = (a.m + G - 1) / G;
  const int r0 = min(a.m, b * per), r1 = min(a.m, r0 + per);
  const int P0 = r0 < r1 ? a.cell_start[max(r0 - 2, 0)] : 0;
  const int P1 = r0 < r1 ? a.cell_start[min(r1 + 1, a.m - 1) + 1] : 0;
  const int P0a = P0 & ~3, P1a = (P1 + 3) & ~3;   // 16-byte boundaries (n_pad is a multiple of 256)
  const bool staged = r0 < r1 && P1a - P0a <= STAGE_CAP;
  if (staged && tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint32_t bytes = (uint32_t)(P1a - P0a) * 4u;
    mbar_arrive_expect_tx(&bar, 2u * bytes);
    for (uint32_t off = 0; off < bytes; off += 32768u) {
      const uint32_t len = min(32768u, bytes - off);
      bulk_g2s(xsm + off / 4, a.xs + P0a + off / 4, len, &bar);
      bulk_g2s(qsm + off / 4, a.q + P0a + off / 4, len, &bar);
    }
  }
  // the cell starts of this CTA's nodes' point ranges (cells r0 - 2 .. r1 + 1)
  const int cb = max(r0 - 2, 0);
  for (int i = tid; cb + i <= min(r1 + 2, a.m) && r0 < r1; i += MVM_THREADS) css[i] = a.cell_start[cb + i];
  {
    const int sa = a.N / a.N2, sb = a.N / a.N1;
    for (int j = tid; j < (a.N2 >> 1); j += MVM_THREADS) {
      const float4 v = __ldg(a.twdf + (int64_t)j * sa);
      wA[j] = dfc{v.x, v.y, v.z, v.w};
    }
    for (int j = tid; j < (a.N1 >> 1); j += MVM_THREADS) {
      const float4 v = __ldg(a.twdf + (int64_t)j * sb);
      wB[j] = dfc{v.x, v.y, v.z, v.w};
    }
  }
  __syncthreads();
  if (staged && !mbar_wait_bounded(&bar, 0)) {
    dev_flag(a.status, LOVE_ERR_TIMEOUT);
    return;   // the other CTAs' next barrier expires too
  }
  // point p's x and q (p a global point number): staged or from global memory
  const float* xsrc = staged ? xsm : a.xs;
  const float* qsrc = staged ? qsm : a.q;
  const int poff = staged ? P0a : 0;
  // ---- 0: u = scal_j W q_j on the nodes [r0, r1) (warp per node)
  {
    constexpr int U = 4;
    for (int r = r0 + warp; r < r1; r += MVM_WARPS) {
      DotAccF acc;
      acc.zero();
      const int lo = css[max(r - 2, 0) - cb], hi = css[min(r + 1, a.m - 1) + 1 - cb];
      for (int p0 = lo + lane; p0 < hi; p0 += 32 * U) {
        float xv[U], qv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int p = p0 + 32 * u;
          xv[u] = p < hi ? xsrc[p - poff] : 0.f;
          qv[u] = p < hi ? qsrc[p - poff] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (p0 + 32 * u < hi) acc.add_prod(node_weight_1d(xv[u], a.g, r), qv[u]);
      }
      warp_merge(acc);
      if (lane == 0) {
        const double v = acc.value() * sc;
        const float h = (float)v;
        __stcg(a.u + r, make_float2(h, (float)(v - (double)h)));
      }
    }
  }
  if (!grid_barrier(a.gs, gen, a.status)) return;
  // ---- 1: pass A on own nodes
  for (int lr = tid; lr < RL; lr += MVM_THREADS) {
    const int f = lr / R2, n2 = lr - f * R2;
    const int r = n1_0 + f + a.N1 * n2;
    us[lr] = r < a.m ? __ldcg(a.u + r) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int t = tid; t < (a.N2 << a.logNB); t += MVM_THREADS) {
    const int f = t & (NB - 1), n2 = t >> a.logNB;
    dfc c{0.f, 0.f, 0.f, 0.f};
    if (n2 < R2) {
      const float2 u = us[f * R2 + n2];
      c.rh = u.x;
      c.rl = u.y;
    }
    x[(bitrev(n2, a.logN2) << a.logNB) + f] = c;
  }
  __syncthreads();
  fft_dit_df(x, a.N2, a.logNB, wA, false);
  for (int t = tid; t < (a.N2 << a.logNB); t += MVM_THREADS) {
    const int f = t & (NB - 1), k2 = t >> a.logNB;
    const int n1 = n1_0 + f;
    const float4 tw = __ldg(a.twdf + (((int64_t)n1 * k2) & (a.N - 1)));
    const dfc v = dfc_mul(x[t], dfc{tw.x, tw.y, tw.z, tw.w}, false);
    __stcg(reinterpret_cast<float4*>(a.work) + (int64_t)k2 * a.N1 + n1, make_float4(v.rh, v.rl, v.ih, v.il));
  }
  if (!grid_barrier(a.gs, gen, a.status)) return;
  // ---- 2: pass B
  {
    const int FB = a.FB, logFB = a.logFB;
    const int k2_0 = b * FB;
    const float4* wk = reinterpret_cast<const float4*>(a.work);
    for (int t = tid; t < (a.N1 << logFB); t += MVM_THREADS) {
      const int n1 = t & (a.N1 - 1), f = t >> a.logN1;
      const float4 v = __ldcg(wk + (int64_t)(k2_0 + f) * a.N1 + n1);
      x[(bitrev(n1, a.logN1) << logFB) + f] = dfc{v.x, v.y, v.z, v.w};
    }
    __syncthreads();
    fft_dit_df(x, a.N1, logFB, wB, false);
    for (int t = tid; t < (a.N1 << logFB); t += MVM_THREADS) {
      const int f = t & (FB - 1), k1 = t >> logFB;
      const float2 lv = __ldg(a.lamdf + (k2_0 + f) + a.N2 * k1);
      const float lh = lv.x, ll = lv.y;
      dfc v = x[t];
      dfs_mulsub(v.rh, v.rl, lh, ll, 0.f, 0.f, 0.f, 0.f, v.rh, v.rl);
      dfs_mulsub(v.ih, v.il, lh, ll, 0.f, 0.f, 0.f, 0.f, v.ih, v.il);
      x[t] = v;
    }
    __syncthreads();
    fft_dif_df(x, a.N1, logFB, wB, true);
    float4* wo = reinterpret_cast<float4*>(a.work);
    for (int t = tid; t < (a.N1 << logFB); t += MVM_THREADS) {
      const int n1 = t & (a.N1 - 1), f = t >> a.logN1;
      const dfc v = x[(bitrev(n1, a.logN1) << logFB) + f];
      __stcg(wo + (int64_t)(k2_0 + f) * a.N1 + n1, make_float4(v.rh, v.rl, v.ih, v.il));
    }
  }
  if (!grid_barrier(a.gs, gen, a.status)) return;
  // ---- 3: pass C -> K_UU u on own nodes
  {
    const float4* wk = reinterpret_cast<const float4*>(a.work);
    for (int t = tid; t < (a.N2 << a.logNB); t += MVM_THREADS) {
      const int f = t & (NB - 1), k2 = t >> a.logNB;
      const int n1 = n1_0 + f;
      const float4 v = __ldcg(wk + (int64_t)k2 * a.N1 + n1);
      const float4 tw = __ldg(a.twdf + (((int64_t)n1 * k2) & (a.N - 1)));
      x[t] = dfc_mul(dfc{v.x, v.y, v.z, v.w}, dfc{tw.x, tw.y, tw.z, tw.w}, true);
    }
    __syncthreads();
    fft_dif_df(x, a.N2, a.logNB, wA, true);
    for (int lr = tid; lr < RL; lr += MVM_THREADS) {
      const int f = lr / R2, n2 = lr - f * R2;
      const int r = n1_0 + f + a.N1 * n2;
      if (r < a.m) {
        const dfc v = x[(bitrev(n2, a.logN2) << a.logNB) + f];
        __stcg(a.ku + r, (float)((double)v.rh + (double)v.rl));
      }
    }
  }
  if (!grid_barrier(a.gs, gen, a.status)) return;
  // ---- 4: y = W^T (K_UU u) + s^2 q_j, q_j normalised, for the points of cells
  // [r0, r1) (their stencils reach the nodes r0 - 1 .. r1 + 1, staged first)
  {
    const float scf = (float)sc;
    const int kb = max(r0 - 1, 0), ke = min(r1 + 1, a.m - 1);
    for (int r = kb + tid; r <= ke && r0 < r1; r += MVM_THREADS) kus[r - kb] = __ldcg(a.ku + r);
    __syncthreads();
    const int q0 = r0 < r1 ? css[r0 - cb] : 0, q1 = r0 < r1 ? css[r1 - cb] : 0;
    for (int p = q0 + tid; p < q1; p += MVM_THREADS) {
      const float qs = qsrc[p - poff] * scf;
      int base;
      float w[4];
      keys_weights(grid_coord(xsrc[p - poff], a.g, 0), a.g.g[0], base, w);
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc += w[k] * kus[base - 1 + k - kb];   // nodes kb .. ke
      a.q[p] = qs;
      a.y[p] = acc + a.noise * qs;
    }
    // rows past n (padding to n_pad) are zero
    for (int64_t p = a.n + (int64_t)b * MVM_THREADS + tid; p < a.n_pad; p += (int64_t)G * MVM_THREADS) {
      a.q[p] = 0.f;
      a.y[p] = 0.f;
    }
  }
}

// the FP64 twiddles and spectrum as df pairs (once per run)
__global__ void k_mvm_tables(const double2* __restrict__ tw, const double* __restrict__ lam, int N,
                             float4* __restrict__ twdf, float2* __restrict__ lamdf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const dfc w = dfc_from(tw[j]);
  twdf[j] = make_float4(w.rh, w.rl, w.ih, w.il);
  const double l = lam[j];
  const float lh = (float)l;
  lamdf[j] = make_float2(lh, (float)(l - (double)lh));
}

int ilog2_mvm(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

// work: N df complex | N df twiddles | N df spectrum | m df pairs (u) | m floats
// (K_UU u) | barrier counters
static size_t mvm_gs_offset(const love_ski* ski) {
  const size_t N = (size_t)ski->fft[0].N;
  return (sizeof(dfc) * N * 2 + sizeof(float2) * N + (sizeof(float) + sizeof(float2)) * (size_t)ski->grid.m + 255) &
         ~(size_t)255;
}
size_t ski_mvm_fused_work_bytes(const love_ski* ski) { return mvm_gs_offset(ski) + sizeof(GridSync); }

love_status ski_mvm_fused(love_ski* ski, float* qj, const double* scal, const int* done, float* y, void* work,
                          unsigned int gen0, cudaStream_t s) {
  const GridHost& gh = ski->grid;
  if (gh.dim != 1 || gh.additive || ski->dtype != LOVE_F32) return LOVE_ERR_UNSUPPORTED;
  const FftPlan& p = ski->fft[0];
  const int m = (int)gh.m, N = (int)p.N;
  if (N < 64 || !p.tw_d || !p.lam_d) return LOVE_ERR_UNSUPPORTED;
  static const int coop = [] {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, dev);
    return c;
  }();
  if (!coop) return LOVE_ERR_UNSUPPORTED;
  const int l = ilog2_mvm(N);
  const int N1 = 1 << (l / 2), N2 = N >> (l / 2);
  int G = N1;
  while (G > num_sms()) G >>= 1;
  const int NB = N1 / G, FB = N2 / G, R2 = (m + N1 - 1) / N1, RL = NB * R2;
  const int per = (m + G - 1) / G;
  const size_t smem = sizeof(dfc) * ((size_t)N / G + N2 / 2 + N1 / 2) + sizeof(float) * 2 * (size_t)STAGE_CAP +
                      sizeof(float2) * (size_t)RL + sizeof(float) * ((size_t)per + 4) + sizeof(int) * ((size_t)per + 8);
  const int limit = smem_limit(reinterpret_cast<const void*>(k_ski_mvm_1d));
  if (limit < 0) return LOVE_ERR_CUDA;
  if (smem > (size_t)limit) return LOVE_ERR_UNSUPPORTED;
  LOVE_TRY(allow_smem(k_ski_mvm_1d, smem));
  int per_sm = 0;
  LOVE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ski_mvm_1d, MVM_THREADS, smem));
  if (per_sm < 1 || (int64_t)per_sm * num_sms() < G) return LOVE_ERR_UNSUPPORTED;
  MvmArgs a{};
  a.g = gh.dev();
  a.m = m;
  a.n = ski->n;
  a.n_pad = ski->n_pad;
  a.xs = (const float*)ski->xs;
  a.cell_start = ski->cell_start;
  a.q = qj;
  a.scal = scal;
  a.done = done;
  a.noise = (float)gh.noise;
  a.y = y;
  char* w = (char*)work;
  a.work = (dfc*)w;
  a.twdf = (const float4*)(w + sizeof(dfc) * (size_t)N);
  a.lamdf = (const float2*)(w + sizeof(dfc) * 2 * (size_t)N);
  a.u = (float2*)(w + (sizeof(dfc) * 2 + sizeof(float2)) * (size_t)N);
  a.ku = (float*)(a.u + m);
  a.gs = (GridSync*)(w + mvm_gs_offset(ski));
  a.N = N;
  a.N1 = N1;
  a.N2 = N2;
  a.logN1 = ilog2_mvm(N1);
  a.logN2 = ilog2_mvm(N2);
  a.logNB = ilog2_mvm(NB);
  a.logFB = ilog2_mvm(FB);
  a.NB = NB;
  a.FB = FB;
  a.R2 = R2;
  a.gen0 = gen0;
  a.status = ski->status;
  void* args[] = {(void*)&a};
  LOVE_COUNT_LAUNCH();
  return cuda_check(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_ski_mvm_1d), dim3(G),
                                                dim3(MVM_THREADS), args, smem, s));
}

love_status fft_df_tables(const FftPlan& p, float4* twdf, float2* lamdf, cudaStream_t s) {
  const int N = (int)p.N;
  if (!p.tw_d || !p.lam_d) return LOVE_ERR_UNSUPPORTED;
  LOVE_COUNT_LAUNCH();
  k_mvm_tables<<<ceil_div(N, 256), 256, 0, s>>>((const double2*)p.tw_d, (const double*)p.lam_d, N, twdf, lamdf);
  LOVE_LAUNCH_CHECK();
  return LOVE_OK;
}

// the df tables and the barrier counters of a run's fused products (once per run)
love_status ski_mvm_fused_reset(const love_ski* ski, void* work, cudaStream_t s) {
  const FftPlan& p = ski->fft[0];
  const size_t N = (size_t)p.N;
  LOVE_TRY(fft_df_tables(p, (float4*)((char*)work + sizeof(dfc) * N), (float2*)((char*)work + sizeof(dfc) * 2 * N), s));
  return cuda_check(cudaMemsetAsync((char*)work + mvm_gs_offset(ski), 0, sizeof(GridSync), s));
}

}  // namespace love
