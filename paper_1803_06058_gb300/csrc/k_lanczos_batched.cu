// k_lanczos_batched.cu -- the n-space Lanczos runs (Sec. 2.2 with the full
// reorthogonalisation of Sec. 5) of many independent GPs on 1-D grids, as ONE
// launch per phase per step for all of them.
//
// A GP of the batch is a row of a descriptor table (BGp): its sorted points,
// grid, circulant tables, Lanczos basis Q, working vector y and device-side
// scalars.  Every phase walks a ragged list of chunks that never straddle two
// GPs, so one launch covers all GPs whatever their sizes:
//   scatter   u = W q_j            a chunk of grid nodes, a warp per node
//                                  (double-float sums of ~4 n/m points)
//   K_UU      ku = K_UU u          a CTA per GP: the circulant-embedding
//                                  product of length N by the real-input split
//                                  (one complex FFT of length N/2 each way),
//                                  double-float butterflies in shared memory
//   gather    y = W^T ku + s^2 q_j a chunk of points, q_j normalised in place
//   dot       c = Q_j^T y          chunks of R rows; partial rows per chunk,
//   update+dot y -= Q_j c; c' = Q_j^T y     merged per GP by the GP's last chunk
//   update+norm y -= Q_j c'; beta_j = |y|   (fixed order: bit-reproducible)
// The sweeps are the detection form of the single-GP run (the second
// Gram-Schmidt pass only where |c'| > eta |y'|), with the single-GP run's
// epilogue (alpha_j, the detection test, beta_j, breakdown) applied per GP.
// R, the rows of a sweep chunk, is picked by timing the dot sweep on the
// batch itself.  The caller captures the k steps into one CUDA graph.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lanczos_common.cuh"
#include "fft_core.cuh"

namespace love {
namespace {
using namespace fftcore;

// one GP of the batch (device copy)
struct BGp {
  GridDev g;
  const float* xs;          // cell-sorted points (n_pad)
  const int* cell_start;    // m + 1
  int64_t n, n_pad;
  float noise;
  int kcols;                // columns of Q (this GP's k)
  float* Q;                 // n_pad x kcols, column-major (ldq = n_pad)
  float* y;                 // n_pad
  float2* u;                // m double-float (W q_j)
  float* ku;                // m (K_UU W q_j)
  const float4* twdf;       // W_N^j, double-float complex
  const float2* lamdf;      // lambda_j / N, double-float
  int N, logM;              // circulant length N, log2(N / 2)
  LanczosState* st;
  DevStatus* status;
  double2* partial;         // [max(nsweep, npts)][kcols + 2]
  int nsweep;               // sweep chunks of this GP
  int npts;                 // point chunks of this GP
};
// a piece of one GP's rows (points or grid nodes): [r0, r1), local index within the GP
struct Chunk {
  int gp, local;
  int64_t r0, r1;
};

constexpr int BSC_T = 256;        // scatter CTA (8 warps, a warp per node)
constexpr int BSC_NODES = 64;     // nodes per scatter chunk
constexpr int BG_T = 256;         // gather / probe CTA
constexpr int BG_POINTS = 1024;   // points per gather chunk
constexpr int BK_T = 1024;        // K_UU CTA
constexpr int BK_MAXM = 8192;     // largest half-length N / 2 (shared memory: 192 KB)

__device__ __forceinline__ void load_gp(BGp& dst, const BGp* src) {
  // the descriptor into shared memory, word by word
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(BGp) / sizeof(int)); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

__global__ void k_bat_init(const BGp* __restrict__ gps, int B, double tau) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  LanczosState* st = gps[b].st;
  st->maxabs = 0.0;
  st->tau = tau;
  st->done = 0;
  st->k_eff = gps[b].kcols;
  st->kmax = gps[b].kcols;
  for (int i = 0; i <= MERGE_MAXG; ++i) st->counter[i] = st->counter2[i] = 0u;
  st->cg_done = 0;
  st->cg_iters = 0;
  st->skip = 0;
  st->n_skip = 0;
}

// u[node] = scal_j sum_p w_p(node) Q[p, j] over the cell-sorted points of the
// node's four cells (as the single-GP scatter), the sum kept as a float pair
__global__ void __launch_bounds__(BSC_T) k_bat_scatter(const BGp* __restrict__ gps, const Chunk* __restrict__ chunks,
                                                       int j) {
  __shared__ BGp G;
  const Chunk c = chunks[blockIdx.x];
  load_gp(G, gps + c.gp);
  if (G.st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* q = G.Q + (int64_t)j * G.n_pad;
  const df sc = df_from_double(G.st->scal[j]);
  for (int64_t node = c.r0 + warp; node < c.r1; node += BSC_T / 32) {
    int nd[1] = {(int)node};
    NodeRanges<1> rg;
    rg.build(G.g, nd, G.cell_start, lane);
    DotAccF acc;
    acc.zero();
    for (int f = lane; f < rg.total; f += 32) {
      const int p = rg.point(f);
      acc.add_prod(node_weight<float, 1>(G.xs + p, G.g, nd), q[p]);
    }
    warp_merge(acc);
    if (lane == 0) {
      const df v = df_mul(two_sum(acc.s, acc.c), sc);
      G.u[node] = make_float2(v.hi, v.lo);
    }
  }
}

__device__ __forceinline__ dfc dfc_half(dfc a) { return dfc{0.5f * a.rh, 0.5f * a.rl, 0.5f * a.ih, 0.5f * a.il}; }
__device__ __forceinline__ dfc dfc_conj(dfc a) { return dfc{a.rh, a.rl, -a.ih, -a.il}; }
__device__ __forceinline__ dfc dfc_times_i(dfc a) { return dfc{-a.ih, -a.il, a.rh, a.rl}; }   // i a
__device__ __forceinline__ dfc dfc_times_mi(dfc a) { return dfc{a.ih, a.il, -a.rh, -a.rl}; }  // -i a
__device__ __forceinline__ dfc dfc_rscale(dfc a, float2 l) {
  const df re = df_mul(df{a.rh, a.rl}, df{l.x, l.y}), im = df_mul(df{a.ih, a.il}, df{l.x, l.y});
  return dfc{re.hi, re.lo, im.hi, im.lo};
}
__device__ __forceinline__ dfc ld_tw(const float4* t, int k) {
  const float4 v = t[k];
  return dfc{v.x, v.y, v.z, v.w};
}

// Between the two half-length transforms: from Z = DFT_M(u_even + i u_odd)
// (M = N / 2), the spectrum of the real u is X_k = E_k + W^k O_k and
// X_{k+M} = E_k - W^k O_k with E_k = (Z_k + conj Z_{M-k}) / 2 and
// O_k = -i (Z_k - conj Z_{M-k}) / 2 (W = W_N).  Y = lambda/N . X, and
// C_k = (Y_k + Y_{k+M}) + i conj(W^k) (Y_k - Y_{k+M}) is the half-length
// spectrum whose inverse transform is y_{2n} + i y_{2n+1}.
__device__ __forceinline__ dfc kuu_pack(int k, int M, dfc Zk, dfc Zmk, const float4* twdf, const float2* lamdf) {
  const dfc E = dfc_half(dfc_add(Zk, dfc_conj(Zmk)));
  const dfc O = dfc_half(dfc_times_mi(dfc_sub(Zk, dfc_conj(Zmk))));
  const dfc W = ld_tw(twdf, k);
  const dfc WO = dfc_mul(O, W, false);
  const dfc Y0 = dfc_rscale(dfc_add(E, WO), lamdf[k]);
  const dfc Y1 = dfc_rscale(dfc_sub(E, WO), lamdf[k + M]);
  return dfc_add(dfc_add(Y0, Y1), dfc_times_i(dfc_mul(dfc_sub(Y0, Y1), W, true)));
}

// ku = K_UU u (probe: u = 1), one CTA per GP
__global__ void __launch_bounds__(BK_T, 1) k_bat_kuu(const BGp* __restrict__ gps, int probe) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ BGp G;
  load_gp(G, gps + blockIdx.x);
  if (G.st->done) return;
  const int M = G.N >> 1, logM = G.logM, m = G.g.m;
  dfc* z = reinterpret_cast<dfc*>(smem_raw);
  dfc* w = z + M;
  {   // twiddles W_M^j = W_N^{2j}, j < M / 2
    for (int jj = threadIdx.x; jj < (M >> 1); jj += blockDim.x) w[jj] = ld_tw(G.twdf, 2 * jj);
  }
  for (int n = threadIdx.x; n < M; n += blockDim.x) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    if (2 * n < m) a = probe ? make_float2(1.f, 0.f) : G.u[2 * n];
    if (2 * n + 1 < m) b = probe ? make_float2(1.f, 0.f) : G.u[2 * n + 1];
    z[bitrev(n, logM)] = dfc{a.x, a.y, b.x, b.y};
  }
  __syncthreads();
  fft_dit_df(z, M, 0, w, false);
  for (int k = threadIdx.x; k <= (M >> 1); k += blockDim.x) {
    const int mk = (M - k) & (M - 1);
    const dfc Zk = z[k], Zmk = z[mk];
    const dfc Ck = kuu_pack(k, M, Zk, Zmk, G.twdf, G.lamdf);
    if (mk != k) z[mk] = kuu_pack(mk, M, Zmk, Zk, G.twdf, G.lamdf);
    z[k] = Ck;
  }
  __syncthreads();
  fft_dif_df(z, M, 0, w, true);
  for (int n = threadIdx.x; n < M; n += blockDim.x) {
    const dfc o = z[bitrev(n, logM)];
    if (2 * n < m) G.ku[2 * n] = o.rh + o.rl;
    if (2 * n + 1 < m) G.ku[2 * n + 1] = o.ih + o.il;
  }
}

// y = W^T ku + s^2 q_j with q_j normalised in place (zero past n)
__global__ void __launch_bounds__(BG_T) k_bat_gather(const BGp* __restrict__ gps, const Chunk* __restrict__ chunks,
                                                     int j) {
  __shared__ BGp G;
  const Chunk c = chunks[blockIdx.x];
  load_gp(G, gps + c.gp);
  if (G.st->done) return;
  const float scal = (float)G.st->scal[j];
  float* qj = G.Q + (int64_t)j * G.n_pad;
  for (int64_t p = c.r0 + threadIdx.x; p < c.r1; p += BG_T) {
    float q = 0.f, r = 0.f;
    if (p < G.n) {
      q = qj[p] * scal;
      Stencil<float, 1> stc;
      stc.compute(G.xs + p, G.g);
      r = stc.apply(G.ku, G.g) + G.noise * q;
    }
    qj[p] = q;
    G.y[p] = r;
  }
}

// probe b = (1/m) W^T K_UU 1 into Q[:, 0]; scal[0] = 1 / |b| (merged per GP)
__global__ void __launch_bounds__(BG_T) k_bat_probe(const BGp* __restrict__ gps, const Chunk* __restrict__ chunks) {
  __shared__ BGp G;
  __shared__ DotAccF red[32];
  const Chunk c = chunks[blockIdx.x];
  load_gp(G, gps + c.gp);
  const float inv_m = 1.f / (float)G.g.m;
  DotAccF a;
  a.zero();
  for (int64_t p = c.r0 + threadIdx.x; p < c.r1; p += BG_T) {
    float b = 0.f;
    if (p < G.n) {
      Stencil<float, 1> stc;
      stc.compute(G.xs + p, G.g);
      b = stc.apply(G.ku, G.g) * inv_m;
    }
    G.Q[p] = b;
    a.add_prod(b, b);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(G.partial + c.local, a);
  LanczosState* st = G.st;
  const bool last = last_cta_reduce<DotAccF>(G.partial, 1, 1, &st->norm2, st->counter, nullptr, G.npts, c.local);
  if (last && threadIdx.x == 0) st->scal[0] = 1.0 / sqrt(st->norm2);
}

// the members the shared sweep epilogue reads
struct BSweepArgs {
  LanczosState* st;
  DevStatus* status;
  double2* partial;
  double* gram;
  double eta2;
  int j, kcols, detect;
};

// One sweep over a chunk of one GP's rows, 64 rows at a time: rows 2l, 2l + 1
// of the columns w, w + 8, ... in the registers of warp w, lane l (as the
// single-GP register sweep); the dots accumulate over the chunk's blocks.
template <int MODE, int KPW>
__global__ void __launch_bounds__(TILE_T) k_bat_sweep(const BGp* __restrict__ gps, const Chunk* __restrict__ chunks,
                                                      int j, int detect, double eta2, DevStatus* status_override) {
  using Acc = DotAccF;
  constexpr int BR = 64;
  __shared__ BGp G;
  __shared__ Acc red[NWARP];
  __shared__ float hp[NWARP][BR];
  __shared__ float ys[BR];
  __shared__ float cf[LOVE_MAX_K + 8];
  __shared__ double2 wsum[8 * 32];   // epilogue scratch: 512 doubles >= (j + 1) + blockDim.x
  const Chunk c = chunks[blockIdx.x];
  load_gp(G, gps + c.gp);
  LanczosState* st = G.st;
  if (st->done || (MODE == MODE_UPDATE_NORM && detect && st->skip)) return;
  const int ncols = j + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
    const double* cc = MODE == MODE_UPDATE_DOT ? st->coef : st->coef2;
    for (int i = tid; i < ncols; i += TILE_T) cf[i] = (float)cc[i];
  }
  // detection: y' sits in the slot of q_{j+1}, where the second pass works
  float* yv_src = (MODE == MODE_UPDATE_NORM && detect && j + 1 < G.kcols) ? G.Q + (int64_t)(j + 1) * G.n_pad : G.y;
  float* ynext = j + 1 < G.kcols ? G.Q + (int64_t)(j + 1) * G.n_pad : G.y;
  Acc acc[KPW];
#pragma unroll
  for (int s2 = 0; s2 < KPW; ++s2) acc[s2].zero();
  Acc nacc;
  nacc.zero();
  const int r0 = 2 * lane;
  for (int64_t row0 = c.r0; row0 < c.r1; row0 += BR) {
    float q[KPW][2];
#pragma unroll
    for (int s2 = 0; s2 < KPW; ++s2) {
      const int i = warp + NWARP * s2;
      if (i < ncols) {
        const float2 v = *reinterpret_cast<const float2*>(G.Q + (int64_t)i * G.n_pad + row0 + r0);
        q[s2][0] = v.x;
        q[s2][1] = v.y;
      } else {
        q[s2][0] = 0.f;
        q[s2][1] = 0.f;
      }
    }
    if (tid < BR) ys[tid] = yv_src[row0 + tid];
    __syncthreads();
    if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
      float ps[2] = {0.f, 0.f};
#pragma unroll
      for (int s2 = 0; s2 < KPW; ++s2) {
        const int i = warp + NWARP * s2;
        if (i < ncols) {
          ps[0] = fmaf(q[s2][0], cf[i], ps[0]);
          ps[1] = fmaf(q[s2][1], cf[i], ps[1]);
        }
      }
      hp[warp][r0] = ps[0];
      hp[warp][r0 + 1] = ps[1];
      __syncthreads();
      if (tid < BR) {
        float sum = hp[0][tid];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) sum += hp[w][tid];
        const float yv = ys[tid] - sum;
        const int64_t p = row0 + tid;
        if (MODE == MODE_UPDATE_DOT) {
          if (detect) {
            ynext[p] = yv;
            nacc.add_prod(yv, yv);
          } else {
            G.y[p] = yv;
          }
          ys[tid] = yv;
        } else {
          ynext[p] = yv;
          nacc.add_prod(yv, yv);
        }
      }
      if (MODE == MODE_UPDATE_DOT) __syncthreads();
    }
    if (MODE != MODE_UPDATE_NORM) {
      const float y0 = ys[r0], y1 = ys[r0 + 1];
#pragma unroll
      for (int s2 = 0; s2 < KPW; ++s2) {
        const int i = warp + NWARP * s2;
        if (i < ncols) acc[s2].add(fmaf(q[s2][1], y1, q[s2][0] * y0));
      }
    }
    __syncthreads();
  }
  BSweepArgs a;
  a.st = st;
  a.status = status_override ? status_override : G.status;
  a.partial = G.partial;
  a.gram = nullptr;
  a.eta2 = eta2;
  a.j = j;
  a.kcols = G.kcols;
  a.detect = detect;
  sweep_epilogue<float, MODE, KPW>(a, acc, nacc, red, wsum, G.nsweep, c.local);
}

int ilog2b(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

template <int MODE>
love_status bat_sweep(const BGp* gps, const Chunk* ch, int nch, int j, int detect, double eta2, DevStatus* ovr,
                      cudaStream_t s) {
  const int ncols = j + 1;
#define LOVE_BSWEEP(KPW)                                                                        \
  if (ncols <= NWARP * KPW) {                                                                   \
    LOVE_COUNT_LAUNCH();                                                                        \
    k_bat_sweep<MODE, KPW><<<nch, TILE_T, 0, s>>>(gps, ch, j, detect, eta2, ovr);               \
    return cuda_check(cudaGetLastError());                                                      \
  }
  LOVE_BSWEEP(1)
  LOVE_BSWEEP(2)
  LOVE_BSWEEP(4)
  LOVE_BSWEEP(8)
  LOVE_BSWEEP(16)
  LOVE_BSWEEP(32)
#undef LOVE_BSWEEP
  return LOVE_ERR_UNSUPPORTED;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

love_status lanczos_batched(int B, love_ski* const* skis, const int* kcols, float* const* Q, double tau, double eta,
                            int rows, cudaStream_t s, BatchedLanczos* out) {
  if (B < 1 || !skis || !kcols || !Q || !out) return LOVE_ERR_ARG;
  int kmax = 0;
  for (int b = 0; b < B; ++b) {
    const love_ski* k = skis[b];
    if (!k || k->dtype != LOVE_F32 || k->grid.dim != 1 || k->grid.additive) return LOVE_ERR_UNSUPPORTED;
    const FftPlan& p = k->fft[0];
    if (!p.tw_d || !p.lam_d || p.N < 4 || (p.N >> 1) > BK_MAXM || k->n_pad % 128) return LOVE_ERR_UNSUPPORTED;
    if (kcols[b] < 1 || kcols[b] > LOVE_MAX_K) return LOVE_ERR_ARG;
    kmax = std::max(kmax, kcols[b]);
  }
  const bool detect = eta > 0.0;
  // ---- chunk lists
  std::vector<Chunk> nodes, pts;
  std::vector<int> npts(B);
  for (int b = 0; b < B; ++b) {
    const int64_t m = skis[b]->grid.m, np = skis[b]->n_pad;
    int l = 0;
    for (int64_t r = 0; r < m; r += BSC_NODES) nodes.push_back(Chunk{b, l++, r, std::min<int64_t>(m, r + BSC_NODES)});
    l = 0;
    for (int64_t r = 0; r < np; r += BG_POINTS) pts.push_back(Chunk{b, l++, r, std::min<int64_t>(np, r + BG_POINTS)});
    npts[b] = l;
  }
  auto sweep_list = [&](int R, std::vector<Chunk>& v, std::vector<int>& cnt) {
    v.clear();
    cnt.assign(B, 0);
    for (int b = 0; b < B; ++b) {
      const int64_t np = skis[b]->n_pad;
      int l = 0;
      for (int64_t r = 0; r < np; r += R) v.push_back(Chunk{b, l++, r, std::min<int64_t>(np, r + R)});
      cnt[b] = l;
    }
  };
  const int cand[] = {256, 512, 1024, 2048};
  int max_rows_chunks = 0;   // partial rows a GP can need: the most chunks of any candidate list
  for (int b = 0; b < B; ++b)
    max_rows_chunks = std::max<int>(max_rows_chunks, (int)std::max<int64_t>(npts[b], ceil_div(skis[b]->n_pad, 256)));
  // ---- one work area: descriptors | chunk lists (nodes, points, sweeps) | per GP:
  // state, y, u, ku, df tables, partial table | scratch state + status for tuning
  const size_t sweep_cap = [&] {
    size_t c = 0;
    for (int b = 0; b < B; ++b) c += (size_t)ceil_div(skis[b]->n_pad, 256);
    return c;
  }();
  size_t off = 0;
  const size_t o_gp = off;
  off = align256(off + sizeof(BGp) * B);
  const size_t o_nodes = off;
  off = align256(off + sizeof(Chunk) * nodes.size());
  const size_t o_pts = off;
  off = align256(off + sizeof(Chunk) * pts.size());
  const size_t o_sw = off;
  off = align256(off + sizeof(Chunk) * sweep_cap);
  std::vector<size_t> o_st(B), o_y(B), o_u(B), o_ku(B), o_tw(B), o_lam(B), o_part(B);
  for (int b = 0; b < B; ++b) {
    const love_ski* k = skis[b];
    const size_t m = (size_t)k->grid.m, N = (size_t)k->fft[0].N;
    o_st[b] = off;
    off = align256(off + sizeof(LanczosState));
    o_y[b] = off;
    off = align256(off + sizeof(float) * (size_t)k->n_pad);
    o_u[b] = off;
    off = align256(off + sizeof(float2) * m);
    o_ku[b] = off;
    off = align256(off + sizeof(float) * m);
    o_tw[b] = off;
    off = align256(off + sizeof(float4) * N);
    o_lam[b] = off;
    off = align256(off + sizeof(float2) * N);
    o_part[b] = off;
    off = align256(off + sizeof(double2) * (size_t)max_rows_chunks * (kcols[b] + 2));
  }
  const size_t o_tst = off;
  off = align256(off + sizeof(LanczosState) * B);
  const size_t o_tstat = off;
  off = align256(off + sizeof(DevStatus));
  const Allocator& al = skis[0]->alloc;
  DevBuf wb(al, s);
  if (!wb.get(off)) return LOVE_ERR_OOM;
  char* w = (char*)wb.p;
  std::vector<BGp> gh(B);
  for (int b = 0; b < B; ++b) {
    love_ski* k = skis[b];
    BGp& g = gh[b];
    g.g = k->grid.dev();
    g.xs = (const float*)k->xs;
    g.cell_start = k->cell_start;
    g.n = k->n;
    g.n_pad = k->n_pad;
    g.noise = (float)k->grid.noise;
    g.kcols = kcols[b];
    g.Q = Q[b];
    g.y = (float*)(w + o_y[b]);
    g.u = (float2*)(w + o_u[b]);
    g.ku = (float*)(w + o_ku[b]);
    g.twdf = (const float4*)(w + o_tw[b]);
    g.lamdf = (const float2*)(w + o_lam[b]);
    g.N = (int)k->fft[0].N;
    g.logM = ilog2b(g.N >> 1);
    g.st = (LanczosState*)(w + o_st[b]);
    g.status = k->status;
    g.partial = (double2*)(w + o_part[b]);
    g.npts = npts[b];
    LOVE_TRY(fft_df_tables(k->fft[0], (float4*)(w + o_tw[b]), (float2*)(w + o_lam[b]), s));
  }
  BGp* gps = (BGp*)(w + o_gp);
  Chunk* d_nodes = (Chunk*)(w + o_nodes);
  Chunk* d_pts = (Chunk*)(w + o_pts);
  Chunk* d_sw = (Chunk*)(w + o_sw);
  LOVE_CUDA(cudaMemcpyAsync(d_nodes, nodes.data(), sizeof(Chunk) * nodes.size(), cudaMemcpyHostToDevice, s));
  LOVE_CUDA(cudaMemcpyAsync(d_pts, pts.data(), sizeof(Chunk) * pts.size(), cudaMemcpyHostToDevice, s));
  int maxM = 0;
  for (int b = 0; b < B; ++b) maxM = std::max(maxM, gh[b].N >> 1);
  const size_t kuu_smem = sizeof(dfc) * ((size_t)maxM + maxM / 2);
  LOVE_TRY(allow_smem(k_bat_kuu, kuu_smem));
  const double eta2 = eta * eta;

  // ---- the sweep chunk size: given, or the fastest dot sweep at mid-run on this batch
  std::vector<Chunk> sw;
  std::vector<int> nsw;
  int R = rows;
  out->tune_ms.clear();
  if (R <= 0) {
    // scratch states and status: the timed sweeps read whatever Q holds
    std::vector<BGp> gt = gh;
    for (int b = 0; b < B; ++b) gt[b].st = (LanczosState*)(w + o_tst) + b;
    LOVE_CUDA(cudaMemsetAsync(w + o_tst, 0, sizeof(LanczosState) * B + 256, s));
    // at the middle of the run, and within every GP's columns (the sweep reads
    // columns 0..jt of each Q, zeroed here)
    int kmin = kmax;
    for (int b = 0; b < B; ++b) kmin = std::min(kmin, kcols[b]);
    const int jt = std::max(0, std::min(kmin - 1, kmax / 2));
    for (int b = 0; b < B; ++b)
      LOVE_CUDA(cudaMemsetAsync(Q[b], 0, sizeof(float) * (size_t)skis[b]->n_pad * kcols[b], s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LOVE_CUDA(cudaEventCreate(&e0));
    LOVE_CUDA(cudaEventCreate(&e1));
    float best = 0.f;
    love_status rc = LOVE_OK;
    for (int ci = 0; ci < 4 && rc == LOVE_OK; ++ci) {
      const int Rc = cand[ci];
      sweep_list(Rc, sw, nsw);
      for (int b = 0; b < B; ++b) gt[b].nsweep = nsw[b];
      rc = cuda_check(cudaMemcpyAsync(gps, gt.data(), sizeof(BGp) * B, cudaMemcpyHostToDevice, s));
      if (rc == LOVE_OK) rc = cuda_check(cudaMemcpyAsync(d_sw, sw.data(), sizeof(Chunk) * sw.size(), cudaMemcpyHostToDevice, s));
      if (rc == LOVE_OK) rc = bat_sweep<MODE_DOT>(gps, d_sw, (int)sw.size(), jt, detect, eta2, (DevStatus*)(w + o_tstat), s);
      if (rc == LOVE_OK) rc = cuda_check(cudaEventRecord(e0, s));
      for (int r = 0; r < 2 && rc == LOVE_OK; ++r)
        rc = bat_sweep<MODE_DOT>(gps, d_sw, (int)sw.size(), jt, detect, eta2, (DevStatus*)(w + o_tstat), s);
      if (rc == LOVE_OK) rc = cuda_check(cudaEventRecord(e1, s));
      if (rc == LOVE_OK) rc = cuda_check(cudaEventSynchronize(e1));
      float ms = 0.f;
      if (rc == LOVE_OK) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1));
      out->tune_ms.push_back(ms / 2);
      if (rc == LOVE_OK && (R <= 0 || ms < best)) {
        best = ms;
        R = Rc;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LOVE_TRY(rc);
  }
  if (R % 64 || R < 64) return LOVE_ERR_ARG;
  sweep_list(R, sw, nsw);
  if (sw.size() > sweep_cap) return LOVE_ERR_ARG;   // R below the smallest candidate
  for (int b = 0; b < B; ++b) gh[b].nsweep = nsw[b];
  out->rows = R;
  LOVE_CUDA(cudaMemcpyAsync(gps, gh.data(), sizeof(BGp) * B, cudaMemcpyHostToDevice, s));
  LOVE_CUDA(cudaMemcpyAsync(d_sw, sw.data(), sizeof(Chunk) * sw.size(), cudaMemcpyHostToDevice, s));
  const int nsw_tot = (int)sw.size();

  // ---- probe, then the k steps captured into one graph
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  LOVE_CUDA(cudaEventCreate(&t0));
  LOVE_CUDA(cudaEventCreate(&t1));
  struct EvFree {
    cudaEvent_t a, b;
    ~EvFree() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev_free{t0, t1};
  LOVE_CUDA(cudaEventRecord(t0, s));
  LOVE_COUNT_LAUNCH();
  k_bat_init<<<ceil_div(B, 128), 128, 0, s>>>(gps, B, tau);
  LOVE_LAUNCH_CHECK();
  LOVE_COUNT_LAUNCH();
  k_bat_kuu<<<B, BK_T, kuu_smem, s>>>(gps, 1);
  LOVE_LAUNCH_CHECK();
  LOVE_COUNT_LAUNCH();
  k_bat_probe<<<(int)pts.size(), BG_T, 0, s>>>(gps, d_pts);
  LOVE_LAUNCH_CHECK();
  auto steps = [&]() -> love_status {
    for (int j = 0; j < kmax; ++j) {
      LOVE_COUNT_LAUNCH();
      k_bat_scatter<<<(int)nodes.size(), BSC_T, 0, s>>>(gps, d_nodes, j);
      LOVE_LAUNCH_CHECK();
      LOVE_COUNT_LAUNCH();
      k_bat_kuu<<<B, BK_T, kuu_smem, s>>>(gps, 0);
      LOVE_LAUNCH_CHECK();
      LOVE_COUNT_LAUNCH();
      k_bat_gather<<<(int)pts.size(), BG_T, 0, s>>>(gps, d_pts, j);
      LOVE_LAUNCH_CHECK();
      LOVE_TRY(bat_sweep<MODE_DOT>(gps, d_sw, nsw_tot, j, detect, eta2, nullptr, s));
      LOVE_TRY(bat_sweep<MODE_UPDATE_DOT>(gps, d_sw, nsw_tot, j, detect, eta2, nullptr, s));
      LOVE_TRY(bat_sweep<MODE_UPDATE_NORM>(gps, d_sw, nsw_tot, j, detect, eta2, nullptr, s));
    }
    return LOVE_OK;
  };
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  LOVE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const love_status crc = steps();
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (crc != LOVE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return crc;
  }
  love_status rc = cuda_check(ce);
  if (rc == LOVE_OK) rc = cuda_check(cudaGraphInstantiate(&gexec, graph, 0));
  if (rc == LOVE_OK) rc = cuda_check(cudaGraphLaunch(gexec, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaEventRecord(t1, s));
  // ---- per-GP results
  std::vector<LanczosState> sth(B);
  for (int b = 0; b < B && rc == LOVE_OK; ++b)
    rc = cuda_check(cudaMemcpyAsync(&sth[b], gh[b].st, sizeof(LanczosState), cudaMemcpyDeviceToHost, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  LOVE_TRY(rc);
  LOVE_CUDA(cudaEventElapsedTime(&out->ms, t0, t1));
  out->gp.resize(B);
  for (int b = 0; b < B; ++b) {
    BatchedLanczos::Gp& o = out->gp[b];
    const int k = kcols[b];
    o.alpha.assign(sth[b].alpha, sth[b].alpha + k);
    o.beta.assign(sth[b].beta, sth[b].beta + k);
    o.k_eff = sth[b].k_eff;
    o.skipped = sth[b].n_skip;
  }
  return LOVE_OK;
}

}  // namespace love
