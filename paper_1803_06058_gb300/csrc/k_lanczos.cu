// k_lanczos.cu -- the n-space Lanczos run with full reorthogonalisation and
// the LOVE cache build (the mean solves are in k_cg.cu, the sampler's run in
// k_sampler.cu, the shared scatter / gather / merge pieces in lanczos_common.cuh).
//
// Lanczos (Sec. 2.2) on K^ = W^T K_UU W + s^2 I with full reorthogonalisation
// (Sec. 5) by classical Gram-Schmidt applied twice to the raw product:
//   y = K^ q_j ;  c = Q_j^T y ;  y -= Q_j c ;  c' = Q_j^T y ;  y -= Q_j c'
//   alpha_j = c_j ;  beta_j = |y| ;  q_{j+1} = y / beta_j
// (in exact arithmetic c holds the three-term coefficients alpha_j, beta_{j-1}
// and zeros, so pass 1 is the Lanczos recurrence plus reorthogonalisation).
//
// One step is six launches, all stream-ordered with every scalar kept on the
// device (graph-capturable, no host synchronisation):
//   scatter     u = W q_j           warp per grid node, gather over the
//                                   cell-sorted training points (deterministic)
//   K_UU        u = K_UU u          FFT Toeplitz / Kronecker (k_fft.cu)
//   gather      y = W^T u + s^2 q_j (q_j normalised in place)
//   dot         c = Q_j^T y
//   update+dot  y -= Q_j c;  c' = Q_j^T y
//   update+norm y -= Q_j c';  beta = |y|;  q_{j+1} = y (scaled on next use)
// The last three stream row tiles of [Q_j | y] (128 rows x (j + 1) columns
// of Q, plus y) through a 2- to 8-stage shared-memory ring filled by TMA
// (2-D tensor boxes of Q, a 1-D bulk copy of y; completion on an mbarrier),
// two CTAs per SM, so Q_j is read three times per step and nothing else of
// the step touches HBM.  Dot products accumulate in double-float per thread
// and per CTA, and CTA partials are combined by the last CTA to finish, in a
// fixed order (deterministic, no floating-point atomics).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "lanczos_common.cuh"

namespace love {

namespace {

// out[:, c] = W Q[:, c] on a 3-D grid: the block scheme of k_scatter3_block
// for many columns.  The halo points' cells and fractional coordinates are
// staged once; the columns pass through shared memory SC3M_CH at a time, and
// each thread evaluates a point's weight once per chunk for all its columns.
constexpr int SC3M_CH = 4;
template <typename T>
constexpr size_t sc3m_smem() {
  return SC3_OFF_PV + (size_t)SC3_CAP * SC3M_CH * sizeof(T) + (size_t)SC3_CAP * 3 * sizeof(float) + (size_t)SC3_CAP * 4;
}

template <typename T>
__global__ void __launch_bounds__(512) k_scatter3_multi_block(GridDev g, const T* __restrict__ xs,
                                                              const int* __restrict__ cell_start,
                                                              const T* __restrict__ Q, int64_t ldq, int ncol,
                                                              T* __restrict__ out, int64_t ldo) {
  using Acc = typename AccOf<T>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int* run_off = reinterpret_cast<int*>(smem_raw);
  int (*cs_loc)[SC3_HC + 1] = reinterpret_cast<int (*)[SC3_HC + 1]>(smem_raw + SC3_OFF_CS);
  int* run_g = reinterpret_cast<int*>(smem_raw + SC3_OFF_RG);
  T* pv = reinterpret_cast<T*>(smem_raw + SC3_OFF_PV);   // [SC3M_CH][SC3_CAP]
  float (*pf)[3] = reinterpret_cast<float (*)[3]>(smem_raw + SC3_OFF_PV + (size_t)SC3_CAP * SC3M_CH * sizeof(T));
  unsigned char (*pc)[4] = reinterpret_cast<unsigned char (*)[4]>(
      smem_raw + SC3_OFF_PV + (size_t)SC3_CAP * SC3M_CH * sizeof(T) + SC3_CAP * 3 * sizeof(float));
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int N[3] = {(int)blockIdx.z * SC3_NB, (int)blockIdx.y * SC3_NB, (int)blockIdx.x * SC3_NB};
  int c_lo[3], c_hi[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    c_lo[e] = max(N[e] - 2, 0);
    c_hi[e] = min(N[e] + SC3_NB, g.g[e] - 1);
  }
  const int h0 = c_hi[0] - c_lo[0] + 1, h1 = c_hi[1] - c_lo[1] + 1, h2 = c_hi[2] - c_lo[2] + 1;
  if (t < SC3_RUNS) {
    const int a = t / SC3_HC, b = t % SC3_HC;
    int len = 0, gs = 0;
    if (a < h0 && b < h1) {
      const int64_t base = (int64_t)(c_lo[0] + a) * g.stride[0] + (int64_t)(c_lo[1] + b) * g.stride[1];
      gs = cell_start[base + c_lo[2]];
      for (int z = 0; z <= h2; ++z) cs_loc[t][z] = cell_start[base + c_lo[2] + z] - gs;
      len = cs_loc[t][h2];
    }
    run_g[t] = gs;
    run_off[t + 1] = len;
  }
  if (t == 0) run_off[0] = 0;
  __syncthreads();
  if (t == 0)
    for (int r = 0; r < SC3_RUNS; ++r) run_off[r + 1] += run_off[r];
  __syncthreads();
  const int P = run_off[SC3_RUNS];
  const bool staged = P <= SC3_CAP;
  if (staged) {
    for (int r = w; r < SC3_RUNS; r += 16) {
      const int len = run_off[r + 1] - run_off[r];
      for (int q = lane; q < len; q += 32) {
        const int p = run_g[r] + q, slot = run_off[r] + q;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const T sc = grid_coord(xs[(int64_t)p * 3 + e], g, e);
          int i = (int)floor(sc);
          if (i > g.g[e] - 3) i = g.g[e] - 3;
          pf[slot][e] = (float)(sc - T(i));
          pc[slot][e] = (unsigned char)(i - c_lo[e]);
        }
      }
    }
  }
  const int nd[3] = {N[0] + t / 64, N[1] + (t / 8) % 8, N[2] + t % 8};
  const bool live = nd[0] < g.g[0] && nd[1] < g.g[1] && nd[2] < g.g[2];
  const int zlo = max(nd[2] - 2, c_lo[2]) - c_lo[2], zhi = min(nd[2] + 1, c_hi[2]) - c_lo[2];
  for (int c0 = 0; c0 < ncol; c0 += SC3M_CH) {
    __syncthreads();   // the previous chunk's values are no longer read
    if (staged) {
      for (int r = w; r < SC3_RUNS; r += 16) {
        const int len = run_off[r + 1] - run_off[r];
        for (int q = lane; q < len; q += 32) {
          const int p = run_g[r] + q, slot = run_off[r] + q;
#pragma unroll
          for (int c = 0; c < SC3M_CH; ++c)
            pv[c * SC3_CAP + slot] = c0 + c < ncol ? Q[(int64_t)(c0 + c) * ldq + p] : T(0);
        }
      }
    }
    __syncthreads();
    if (!live) continue;
    Acc acc[SC3M_CH];
#pragma unroll
    for (int c = 0; c < SC3M_CH; ++c) acc[c].zero();
    for (int dx = 0; dx < 4; ++dx) {
      const int a = nd[0] - 2 + dx - c_lo[0];
      if (a < 0 || a >= h0) continue;
      for (int dy = 0; dy < 4; ++dy) {
        const int b = nd[1] - 2 + dy - c_lo[1];
        if (b < 0 || b >= h1 || zlo > zhi) continue;
        const int r = a * SC3_HC + b;
        const int q0 = cs_loc[r][zlo], q1 = cs_loc[r][zhi + 1];
        for (int q = q0; q < q1; ++q) {
          if (staged) {
            const int slot = run_off[r] + q;
            float wt = 1.f;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
              const int rr = nd[e] - ((int)pc[slot][e] + c_lo[e] - 1);
              wt *= keys_u(pf[slot][e] + 1.f - (float)rr);
            }
#pragma unroll
            for (int c = 0; c < SC3M_CH; ++c) acc[c].add_prod((T)wt, pv[c * SC3_CAP + slot]);
          } else {
            const int p = run_g[r] + q;
            const T wt = node_weight<T, 3>(xs + (int64_t)p * 3, g, nd);
#pragma unroll
            for (int c = 0; c < SC3M_CH; ++c)
              if (c0 + c < ncol) acc[c].add_prod(wt, Q[(int64_t)(c0 + c) * ldq + p]);
          }
        }
      }
    }
    const int64_t node = (int64_t)nd[0] * g.stride[0] + (int64_t)nd[1] * g.stride[1] + nd[2];
#pragma unroll
    for (int c = 0; c < SC3M_CH; ++c)
      if (c0 + c < ncol) out[(int64_t)(c0 + c) * ldo + node] = (T)acc[c].value();
  }
}

// out[:, c] = W Q[:, c] for ncol columns (chunks of CH columns per pass),
// double-float accumulation as in k_scatter
template <typename T, int D, int CH>
__global__ void k_scatter_multi(GridDev g, const T* __restrict__ xs, const int* __restrict__ cell_start,
                                const T* __restrict__ Q, int64_t ldq, int ncol, T* __restrict__ out, int64_t ldo,
                                const int32_t* __restrict__ map) {
  using Acc = typename AccOf<T>::type;
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t node = wg; node < g.m; node += nw) {
    int nd[D];
    node_index<D>(node, g, nd);
    NodeRanges<D> rg;
    rg.build(g, nd, cell_start, lane);
    for (int c0 = 0; c0 < ncol; c0 += CH) {
      Acc acc[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) acc[c].zero();
      for (int f = lane; f < rg.total; f += 32) {
        int p = rg.point(f);
        const int pq = map ? map[p] : p;
        T w = node_weight<T, D>(xs + (int64_t)p * D, g, nd);
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (c0 + c < ncol) acc[c].add_prod(w, Q[(int64_t)(c0 + c) * ldq + pq]);
      }
      double val = 0.0;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        warp_merge(acc[c]);
        if (lane == c) val = acc[c].value();
      }
      if (lane < CH && c0 + lane < ncol) out[(int64_t)(c0 + lane) * ldo + node] = (T)val;
    }
  }
}

// out[:, c] = W Q[:, c] on a 1-D grid (FP32), a CTA of SMQ_T threads per
// SMQ_NB grid nodes, thread c summing column c.  The points of the nodes'
// cells (sorted order) pass through shared memory SMQ_PT at a time -- Q's
// columns read once, coalesced along the points and transposed, the next
// tile's values prefetched into registers -- with each point's stencil (first
// node, 4 Keys weights) computed once.  The points arrive by cell, and a node
// n takes points from cells n - 2 .. n + 1 only, so a thread keeps the four
// nodes of the current cell's stencil in registers (Dot2 pairs, as
// k_scatter_multi) and retires the lowest one when the walk moves past its
// last cell: every sum is taken in point order.  The warp-per-node form read
// every value of Q once per node of its stencil.
constexpr int SMQ_NB = 32, SMQ_PT = 64, SMQ_T = 128, SMQ_COLS_MAX = 128;
constexpr size_t smq_smem(int ncol) {
  return sizeof(float) * (size_t)SMQ_PT * (ncol + 1) + sizeof(float4) * SMQ_PT + sizeof(int) * SMQ_PT +
         sizeof(float) * (size_t)SMQ_NB * (ncol + 1);
}
__global__ void __launch_bounds__(SMQ_T) k_scatter_multi_1d(GridDev g, const float* __restrict__ xs,
                                                            const int* __restrict__ cell_start,
                                                            const float* __restrict__ Q, int64_t ldq, int ncol,
                                                            float* __restrict__ out, int64_t ldo) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* qs = reinterpret_cast<float*>(smem_raw);                         // [SMQ_PT][ncol + 1]
  float4* pw = reinterpret_cast<float4*>(qs + (size_t)SMQ_PT * (ncol + 1));
  int* pbase = reinterpret_cast<int*>(pw + SMQ_PT);
  float* os = reinterpret_cast<float*>(pbase + SMQ_PT);                  // [SMQ_NB][ncol + 1]
  const int tid = threadIdx.x, c = tid;
  const int n0 = blockIdx.x * SMQ_NB, n1 = min(n0 + SMQ_NB, g.m);
  const int clo = max(n0 - 2, 0), chi = min(n1, g.g[0] - 1);
  const int p_begin = cell_start[clo], p_end = cell_start[chi + 1];
  // the window: nodes lo .. lo + 3 (the stencil of cell lo + 1)
  DotAccF w0, w1, w2, w3;
  w0.zero();
  w1.zero();
  w2.zero();
  w3.zero();
  int lo = clo - 1;
  auto retire = [&]() {   // node lo is complete: store it, slide the window by one node
    const int nd = lo - n0;
    if (nd >= 0 && nd < n1 - n0 && c < ncol) os[nd * (ncol + 1) + c] = (float)w0.value();
    w0 = w1;
    w1 = w2;
    w2 = w3;
    w3.zero();
    ++lo;
  };
  constexpr int PRE = SMQ_COLS_MAX * SMQ_PT / SMQ_T;
  float pre[PRE];
  auto load_tile = [&](int p0) {
    const int np = min(SMQ_PT, p_end - p0);
#pragma unroll
    for (int e = 0; e < PRE; ++e) {
      const int i = tid + SMQ_T * e, cc = i / SMQ_PT, pp = i - cc * SMQ_PT;
      pre[e] = (cc < ncol && pp < np) ? Q[(int64_t)cc * ldq + p0 + pp] : 0.f;
    }
  };
  if (p_begin < p_end) load_tile(p_begin);
  for (int p0 = p_begin; p0 < p_end; p0 += SMQ_PT) {
    const int np = min(SMQ_PT, p_end - p0);
    __syncthreads();   // the previous tile is consumed
#pragma unroll
    for (int e = 0; e < PRE; ++e) {
      const int i = tid + SMQ_T * e, cc = i / SMQ_PT, pp = i - cc * SMQ_PT;
      if (cc < ncol) qs[pp * (ncol + 1) + cc] = pre[e];
    }
    if (tid < SMQ_PT) {
      int base = 0;
      float w[4] = {0.f, 0.f, 0.f, 0.f};
      if (tid < np) keys_weights(grid_coord(xs[p0 + tid], g, 0), g.g[0], base, w);
      pbase[tid] = base - 1;   // the stencil's first node (nondecreasing along the sorted points)
      pw[tid] = make_float4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    if (p0 + SMQ_PT < p_end) load_tile(p0 + SMQ_PT);
    for (int pp = 0; pp < np; ++pp) {
      const int b = pbase[pp];
      while (lo < b) retire();
      const float q = c < ncol ? qs[pp * (ncol + 1) + c] : 0.f;
      const float4 w4 = pw[pp];
      w0.add_prod(w4.x, q);
      w1.add_prod(w4.y, q);
      w2.add_prod(w4.z, q);
      w3.add_prod(w4.w, q);
    }
  }
  while (lo < n1) retire();
  __syncthreads();
  for (int i = tid; i < SMQ_NB * ncol; i += SMQ_T) {
    const int cc = i / SMQ_NB, nd = i - cc * SMQ_NB;
    if (n0 + nd < n1) out[(int64_t)cc * ldo + n0 + nd] = os[nd * (ncol + 1) + cc];
  }
}

// ---------------------------------------------------------------------------
// Lanczos tile kernels

// 2-D tiled bulk tensor copy (TMA) of a box of Q into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst_smem, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst_smem)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}


// 4 consecutive rows of one column in shared memory (one 16-byte access for
// float, two for double)
template <typename T> struct Row4;
template <> struct Row4<float> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  static __device__ __forceinline__ void store(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Row4<double> {
  static __device__ __forceinline__ void load(const double* p, double* v) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// One reorthogonalisation sweep over the row tiles of [Q_j | y].  Per tile,
// TILE_R rows of columns 0..j of Q (2-D TMA boxes of bc columns) and of y (a
// 1-D bulk copy) land in one stage of a shared-memory ring, so every step
// below reads shared memory only:
//   DOT          c = Q_j^T y                       (alpha_j = c_j)
//   UPDATE_DOT   y -= Q_j c;   c' = Q_j^T y
//   UPDATE_NORM  y -= Q_j c';  beta_j = |y|;  q_{j+1} = y (scaled on next use)
// With `detect`, UPDATE_DOT also writes y' = y - Q_j c to the slot of q_{j+1}
// and sums |y'|^2; its last CTA then measures what is left of y' in span(Q_j)
// and, when |c'| <= eta |y'|, finishes the step itself (beta_j = |y'|) so the
// UPDATE_NORM launch returns at once: the second pass runs only where the
// first one left a detectable component (a DGKS-type test on the measured
// c' instead of a norm-drop bound).
// Both the update and the dots give warp w the columns w, w + 8, ... and lane
// l the rows 4l .. 4l + 3 (16-byte shared-memory accesses); the update's eight
// per-warp partial sums of a row are added in a fixed order.
template <typename T, int MODE, int KPW>
__global__ void __launch_bounds__(TILE_T, 2) k_lanczos_tile(const __grid_constant__ TileArgs<T> a) {
  using Acc = typename AccOf<T>::type;
  static_assert(TILE_R == 128 && TILE_T == 256, "row-quad mapping assumes 128 rows, 8 warps");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  LanczosState* st = a.st;
  const int j = a.j;
  const int ncols = j + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t stage_elems = (size_t)(a.kpad + 1) * TILE_R;               // Q columns, then y
  T* ring = reinterpret_cast<T*>(smem_raw);                                // [stages][kpad + 1][TILE_R]
  T* cf = ring + (size_t)a.stages * stage_elems;                           // [kcols] (16-byte padded)
  T* hp = cf + ((a.kcols + 3) & ~3);                                       // [NWARP][TILE_R]
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(hp + NWARP * TILE_R) + 15) & ~uintptr_t(15));  // [stages]
  __shared__ Acc red[NWARP];

  const int64_t ntiles = a.n_pad / TILE_R;
  if (tid == 0) {
    for (int s = 0; s < a.stages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int nbox = (ncols + a.bc - 1) / a.bc;
  const uint32_t col_bytes = TILE_R * (uint32_t)sizeof(T);
  const uint32_t tx = col_bytes * (uint32_t)(nbox * a.bc + 1);
  // thread 0 fills a stage: 2-D TMA boxes of Q (bc columns x 128 rows; per
  // column 1-D bulk copies issued from a whole warp measured 1.4-1.5x slower)
  // and a 1-D bulk copy of y, completing on the stage's mbarrier
  // consecutive sweeps walk the tiles in opposite orders, so each one starts
  // on the tiles the previous one left in L2
  auto phys = [&](int64_t t) { return a.reverse ? ntiles - 1 - t : t; };
  auto issue = [&](int64_t t, int s) {
    const int64_t tile = phys(t);
    mbar_arrive_expect_tx(&bar[s], tx);
    T* dst = ring + (size_t)s * stage_elems;
    for (int b = 0; b < nbox; ++b)
      tma_load_2d(dst + (size_t)b * a.bc * TILE_R, &a.qmap, (int)(tile * TILE_R), b * a.bc, &bar[s]);
    bulk_g2s(dst + (size_t)a.kpad * TILE_R, a.y + tile * TILE_R, col_bytes, &bar[s]);
  };
  auto fill = [&]() {
    if (tid == 0) {
      for (int s = 0; s < a.stages; ++s) {
        int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
        if (t < ntiles) issue(t, s);
      }
    }
  };
  // Launched as a programmatic dependent of the previous sweep, the kernel may
  // start while that sweep's last CTA still merges.  The update + dot sweep
  // reads only what the sweep before it read (Q_j and y), so its ring fills
  // before the wait; everything else waits for the previous grid first.
  constexpr bool early = MODE == MODE_UPDATE_DOT;
  if (early) fill();
  grid_dep_wait();
  if (st->done || (MODE == MODE_UPDATE_NORM && a.detect && st->skip)) {
    if (early && tid == 0)   // let the copies already issued land before the shared memory is released
      for (int s = 0; s < a.stages; ++s)
        if (blockIdx.x + (int64_t)s * gridDim.x < ntiles) mbar_wait_bounded(&bar[s], 0u);
    return;
  }
  if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
    const double* c = MODE == MODE_UPDATE_DOT ? st->coef : st->coef2;
    for (int i = tid; i < ncols; i += TILE_T) cf[i] = (T)c[i];
  }
  if (!early) fill();

  Acc acc[KPW];
#pragma unroll
  for (int s = 0; s < KPW; ++s) acc[s].zero();
  Acc nacc;
  nacc.zero();
  const int r0 = 4 * lane;   // this lane's rows r0 .. r0 + 3

  int it = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int64_t tile = phys(t);
    const int s = it % a.stages;
    const uint32_t parity = (uint32_t)((it / a.stages) & 1);
    bool ok = mbar_wait_bounded(&bar[s], parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) dev_flag(a.status, LOVE_ERR_TIMEOUT);
      st->done = 1;
      return;
    }
    T* Qt = ring + (size_t)s * stage_elems;
    T* yt = Qt + (size_t)a.kpad * TILE_R;
    // ---- update: y -= Q_j c
    if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
      T ps[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
      for (int i = warp; i < ncols; i += NWARP) {
        T q[4];
        Row4<T>::load(Qt + (size_t)i * TILE_R + r0, q);
        const T ci = cf[i];
#pragma unroll
        for (int r = 0; r < 4; ++r) ps[r] = fma(q[r], ci, ps[r]);
      }
      Row4<T>::store(hp + warp * TILE_R + r0, ps);
      __syncthreads();
      if (tid < TILE_R) {
        T sum = hp[tid];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) sum += hp[w * TILE_R + tid];
        const T yv = yt[tid] - sum;
        const int64_t p = tile * TILE_R + tid;
        if (MODE == MODE_UPDATE_DOT) {
          if (a.detect) {
            if (j + 1 < a.kcols)
              a.Q[(int64_t)(j + 1) * a.ldq + p] = yv;
            else
              a.y[p] = yv;
            nacc.add_prod(yv, yv);
          } else {
            a.y[p] = yv;
          }
          yt[tid] = yv;
          fence_proxy_async();
        } else {
          if (j + 1 < a.kcols)
            a.Q[(int64_t)(j + 1) * a.ldq + p] = yv;
          else
            a.y[p] = yv;
          nacc.add_prod(yv, yv);
        }
      }
      if (MODE == MODE_UPDATE_DOT) __syncthreads();
    }
    // ---- column dots: c_i += q_i . y over this tile
    if (MODE != MODE_UPDATE_NORM) {
      T yr[4];
      Row4<T>::load(yt + r0, yr);
#pragma unroll
      for (int s2 = 0; s2 < KPW; ++s2) {
        const int i = warp + NWARP * s2;
        if (i < ncols) {
          // a partial over this lane's 4 rows, folded into the double-float
          // sum: the partials are ~sqrt(4 / n) of the total, so their
          // rounding stays far below the final rounding
          T q[4];
          Row4<T>::load(Qt + (size_t)i * TILE_R + r0, q);
          T part = q[0] * yr[0];
          part = fma(q[1], yr[1], part);
          part = fma(q[2], yr[2], part);
          part = fma(q[3], yr[3], part);
          acc[s2].add(part);
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      int64_t nt = t + (int64_t)a.stages * gridDim.x;
      if (nt < ntiles) {
        fence_proxy_async();
        issue(nt, s);
      }
    }
  }

  // the next sweep may launch now: it waits for this grid before it reads
  // what the merge below writes
  grid_dep_launch();
  // every issued stage has been consumed: the ring is free for the merge
  sweep_epilogue<T, MODE, KPW>(a, acc, nacc, red, reinterpret_cast<double2*>(smem_raw), (int)gridDim.x,
                              (int)blockIdx.x);
}

// The same three sweeps for short vectors (fewer row tiles than two per SM:
// grid-sized Krylov bases, small training sets).  A CTA owns SMALL_R = 64 rows
// and reads its rows of Q_j once, straight into registers (warp w: the columns
// w, w + 8, ...; lane l: rows 2l, 2l + 1), so every load of the sweep is in
// flight at once; y passes through shared memory between the update and the
// dots.  Partials, merge and scalar work are those of the tiled sweep.
constexpr int SMALL_R = 64;

template <typename T> struct Pair;
template <> struct Pair<float> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
};
template <> struct Pair<double> {
  static __device__ __forceinline__ void load(const double* p, double* v) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
};

template <typename T, int MODE, int KPW>
__global__ void __launch_bounds__(TILE_T) k_lanczos_small(const __grid_constant__ TileArgs<T> a) {
  using Acc = typename AccOf<T>::type;
  static_assert(SMALL_R == 64 && TILE_T == 256, "pair mapping assumes 64 rows, 8 warps");
  __shared__ Acc red[NWARP];
  __shared__ T hp[NWARP][SMALL_R];
  __shared__ T ys[SMALL_R];
  __shared__ T cf[LOVE_MAX_K + 8];
  __shared__ double2 wsum[8 * 32];   // epilogue scratch: 512 doubles >= (j + 1) + blockDim.x
  LanczosState* st = a.st;
  if (st->done || (MODE == MODE_UPDATE_NORM && a.detect && st->skip)) return;
  const int j = a.j;
  const int ncols = j + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
    const double* c = MODE == MODE_UPDATE_DOT ? st->coef : st->coef2;
    for (int i = tid; i < ncols; i += TILE_T) cf[i] = (T)c[i];
  }
  const int64_t row0 = (int64_t)blockIdx.x * SMALL_R;
  const int r0 = 2 * lane;
  T q[KPW][2];
#pragma unroll
  for (int s2 = 0; s2 < KPW; ++s2) {
    const int i = warp + NWARP * s2;
    if (i < ncols) {
      Pair<T>::load(a.Q + (int64_t)i * a.ldq + row0 + r0, q[s2]);
    } else {
      q[s2][0] = T(0);
      q[s2][1] = T(0);
    }
  }
  if (tid < SMALL_R) ys[tid] = a.y[row0 + tid];
  __syncthreads();
  Acc acc[KPW];
#pragma unroll
  for (int s2 = 0; s2 < KPW; ++s2) acc[s2].zero();
  Acc nacc;
  nacc.zero();
  // ---- update: y -= Q_j c
  if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
    T ps[2] = {T(0), T(0)};
#pragma unroll
    for (int s2 = 0; s2 < KPW; ++s2) {
      const int i = warp + NWARP * s2;
      if (i < ncols) {
        const T ci = cf[i];
        ps[0] = fma(q[s2][0], ci, ps[0]);
        ps[1] = fma(q[s2][1], ci, ps[1]);
      }
    }
    hp[warp][r0] = ps[0];
    hp[warp][r0 + 1] = ps[1];
    __syncthreads();
    if (tid < SMALL_R) {
      T sum = hp[0][tid];
#pragma unroll
      for (int w = 1; w < NWARP; ++w) sum += hp[w][tid];
      const T yv = ys[tid] - sum;
      const int64_t p = row0 + tid;
      if (MODE == MODE_UPDATE_DOT) {
        if (a.detect) {
          if (j + 1 < a.kcols)
            a.Q[(int64_t)(j + 1) * a.ldq + p] = yv;
          else
            a.y[p] = yv;
          nacc.add_prod(yv, yv);
        } else {
          a.y[p] = yv;
        }
        ys[tid] = yv;
      } else {
        if (j + 1 < a.kcols)
          a.Q[(int64_t)(j + 1) * a.ldq + p] = yv;
        else
          a.y[p] = yv;
        nacc.add_prod(yv, yv);
      }
    }
    if (MODE == MODE_UPDATE_DOT) __syncthreads();
  }
  // ---- column dots: c_i += q_i . y over this CTA's rows
  if (MODE != MODE_UPDATE_NORM) {
    const T y0 = ys[r0], y1 = ys[r0 + 1];
#pragma unroll
    for (int s2 = 0; s2 < KPW; ++s2) {
      const int i = warp + NWARP * s2;
      if (i < ncols) acc[s2].add(fma(q[s2][1], y1, q[s2][0] * y0));
    }
  }
  sweep_epilogue<T, MODE, KPW>(a, acc, nacc, red, wsum, (int)gridDim.x, (int)blockIdx.x);
}

// Lanczos product y = W^T u + s^2 q_j (u = K_UU W q_j), normalising q_j in
// place: Q[:, j] *= scal_j.  Rows past n are zero.  No-op after breakdown.
template <typename T, int D>
__global__ void k_lanczos_gather(GridDev g, const T* __restrict__ xs, int64_t n, int64_t n_pad,
                                 const T* __restrict__ u, T noise, T* __restrict__ qj, T* __restrict__ y,
                                 const LanczosState* st, int j) {
  if (st->done) return;
  const T scal = (T)st->scal[j];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad;
       p += (int64_t)gridDim.x * blockDim.x) {
    T q = T(0), r = T(0);
    if (p < n) {
      q = qj[p] * scal;
      Stencil<T, D> stc;
      stc.compute(xs + p * D, g);
      r = stc.apply(u, g) + noise * q;
    }
    qj[p] = q;
    y[p] = r;
  }
}

// probe b = (1/m) W^T K_UU 1 into Q[:, 0]; scal[0] = 1/|b|
template <typename T, int D>
__global__ void k_probe(GridDev g, const T* __restrict__ xs, int64_t n, int64_t n_pad, const T* __restrict__ u1,
                        T* __restrict__ q0, double2* partial, LanczosState* st) {
  using Acc = typename AccOf<T>::type;
  __shared__ Acc red[32];
  Acc a;
  a.zero();
  T inv_m = T(1) / T(g.m);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    T b = T(0);
    if (p < n) {
      Stencil<T, D> stc;
      stc.compute(xs + p * D, g);
      b = stc.apply(u1, g) * inv_m;
    }
    q0[p] = b;
    a.add_prod(b, b);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<Acc>(partial, 1, 1, &st->norm2, st->counter);
  if (last && threadIdx.x == 0) st->scal[0] = 1.0 / sqrt(st->norm2);
}

// ---------------------------------------------------------------------------
// tridiagonal Cholesky T = L L^T (one thread, FP64): l_11 = sqrt(alpha_1),
// e_j = beta_j / l_jj, l_{j+1,j+1} = sqrt(alpha_{j+1} - e_j^2)
__global__ void k_tridiag_chol(const double* alpha, const double* beta, const int* k_eff_ptr, int k_fixed,
                               double* d, double* e, DevStatus* status, int* ok) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = k_eff_ptr ? *k_eff_ptr : k_fixed;
  double piv = alpha[0];
  *ok = 1;
  for (int j = 0; j < k; ++j) {
    if (j > 0) {
      e[j - 1] = beta[j - 1] / d[j - 1];
      piv = alpha[j] - e[j - 1] * e[j - 1];
    }
    if (!(piv > 0.0)) {
      dev_flag(status, LOVE_ERR_NOT_PD);
      *ok = 0;
      for (int q = j; q < k; ++q) d[q] = 1.0;
      return;
    }
    d[j] = sqrt(piv);
  }
}

// X L^T = A row-wise (A, X: m x k column-major, lda), i.e. L x^T = a^T per row:
// x_0 = a_0 / d_0 ; x_c = (a_c - e_{c-1} x_{c-1}) / d_c   (FP64 scalars)
template <typename T>
__global__ void k_lt_solve(const T* __restrict__ A, int64_t lda, int64_t m, int k, const double* __restrict__ d,
                           const double* __restrict__ e, T* __restrict__ X, int64_t ldx) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double prev = 0.0;
  for (int c = 0; c < k; ++c) {
    double v = (double)A[(int64_t)c * lda + r];
    if (c > 0) v -= e[c - 1] * prev;
    prev = v / d[c];
    X[(int64_t)c * ldx + r] = (T)prev;
  }
}

// pack the predict cache: row r = [Rt[r, 0..k) | a[r] | 0 pad] in cache dtype
template <typename T, typename OutT>
__global__ void k_pack_rows(const T* __restrict__ Rt, int64_t ldr, int64_t m, int k, const double* __restrict__ a,
                            OutT* __restrict__ out, int ld) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * ld) return;
  int64_t r = idx / ld;
  int c = (int)(idx - r * ld);
  double v = 0.0;
  if (c < k) v = (double)Rt[(int64_t)c * ldr + r];
  else if (c == k && a) v = (double)a[r];
  if constexpr (std::is_same<OutT, __nv_bfloat16>::value) out[idx] = __double2bfloat16(v);
  else out[idx] = (OutT)v;
}

template <typename T>
__global__ void k_permute_in(const T* __restrict__ v, const int32_t* __restrict__ perm, int64_t n, int64_t n_pad,
                             T* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pad) return;
  out[p] = p < n ? v[perm[p]] : T(0);
}
template <typename T>
__global__ void k_permute_out(const T* __restrict__ v, const int32_t* __restrict__ perm, int64_t n,
                              T* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[perm[p]] = v[p];
}

// Ring geometry per launch: a stage holds the j + 1 live columns (rounded up
// to the box width) plus the y column.  Two CTAs per SM whenever each can
// keep at least two stages (one computes while the other waits on its ring),
// with as many stages as fit (up to 8); otherwise one CTA with as many stages
// as fit the SM's shared memory.
inline size_t tile_smem(int stages, int kpad, int kcols, size_t elem) {
  return (size_t)stages * (kpad + 1) * TILE_R * elem + (size_t)((kcols + 3) & ~3) * elem +
         (size_t)NWARP * TILE_R * elem + 16 + 8 * (size_t)stages;
}
struct TileGeom {
  int stages, ctas;
};
inline TileGeom tile_geom(int kpad, int kcols, size_t elem) {
  // per-CTA dynamic limit: 227 KB opt-in less ~1 KB for the kernel's static
  // shared memory; per SM: 228 KB, with 1 KB reserved per CTA plus the static part
  const size_t cta_cap = 231424, sm_cap = 233472, reserved = 2048;
  for (int ctas = 2; ctas >= 1; --ctas)
    for (int st = 8; st >= (ctas == 2 ? 2 : 1); --st) {
      const size_t b = tile_smem(st, kpad, kcols, elem);
      if (b <= cta_cap && (size_t)ctas * (b + reserved) <= sm_cap) return TileGeom{st, ctas};
    }
  return TileGeom{0, 1};
}

template <typename T>
love_status make_qmap(T* Q, int64_t ldq, int kcols, int bc, CUtensorMap* out);

// a launch that may begin before the previous one on the stream has finished
// (programmatic stream serialisation: the kernel orders its own reads)
template <typename K, typename A>
love_status launch_dependent(K kern, int grid, int threads, size_t smem, cudaStream_t s, const A& arg) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cuda_check(cudaLaunchKernelEx(&cfg, kern, arg));
}

template <typename T, int MODE>
love_status tile_run(TileArgs<T> a, cudaStream_t s) {
  const int ncols = a.j + 1;
  if (a.n_pad / TILE_R < (int64_t)TILE_CTAS_PER_SM * num_sms()) {
    // short vectors: one 64-row block per CTA, no staging ring
    const unsigned grid = (unsigned)(a.n_pad / SMALL_R);
#define LOVE_SMALL_CASE(KPW)                                                   \
    if (ncols <= NWARP * KPW) {                                                \
      LOVE_COUNT_LAUNCH(); k_lanczos_small<T, MODE, KPW><<<grid, TILE_T, 0, s>>>(a); \
      return cuda_check(cudaGetLastError());                                   \
    }
    LOVE_SMALL_CASE(1)
    LOVE_SMALL_CASE(2)
    LOVE_SMALL_CASE(4)
    LOVE_SMALL_CASE(8)
    LOVE_SMALL_CASE(16)
    LOVE_SMALL_CASE(32)
#undef LOVE_SMALL_CASE
    return LOVE_ERR_UNSUPPORTED;
  }
  a.kpad = (ncols + a.bc - 1) / a.bc * a.bc;
  a.reverse = MODE == MODE_UPDATE_DOT;   // dot forward, update + dot back, update + norm forward
  const TileGeom tg = tile_geom(a.kpad, a.kcols, sizeof(T));
  if (tg.stages == 0) return LOVE_ERR_UNSUPPORTED;
  a.stages = tg.stages;
  // the tensor map spans the live columns only (at least one box wide): box
  // columns past its extent read as zeros without touching memory
  LOVE_TRY(make_qmap<T>(a.Q, a.ldq, std::min(std::max(ncols, a.bc), a.kcols), a.bc, &a.qmap));
  const size_t smem = tile_smem(a.stages, a.kpad, a.kcols, sizeof(T));
  const int64_t ntiles = a.n_pad / TILE_R;
#define LOVE_TILE_CASE(KPW)                                                                    \
  if (ncols <= NWARP * KPW) {                                                                  \
    auto kern = k_lanczos_tile<T, MODE, KPW>;                                                  \
    LOVE_TRY(allow_smem(kern, smem));                                                          \
    int per_sm = 0;                                                                            \
    LOVE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TILE_T, smem));     \
    per_sm = std::min(std::max(per_sm, 1), tg.ctas);                                           \
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * num_sms());              \
    LOVE_COUNT_LAUNCH();                                                                       \
    return launch_dependent(kern, grid, TILE_T, smem, s, a);                                   \
  }
  LOVE_TILE_CASE(1)
  LOVE_TILE_CASE(2)
  LOVE_TILE_CASE(4)
  LOVE_TILE_CASE(8)
  LOVE_TILE_CASE(16)
  LOVE_TILE_CASE(32)
#undef LOVE_TILE_CASE
  return LOVE_ERR_UNSUPPORTED;
}

template <typename T>
love_status lanczos_gather_any(love_ski* ski, const T* u, T* qj, T* y, const LanczosState* st, int j,
                               cudaStream_t s) {
  const GridDev g = ski->grid.dev();
  const int blocks = (int)std::min<int64_t>(ceil_div(ski->n_pad, 256), (int64_t)num_sms() * 8);
  const T* xs = (const T*)ski->xs;
  const T nz = (T)ski->grid.noise;
  switch (g.dim) {
    case 1: LOVE_COUNT_LAUNCH(); k_lanczos_gather<T, 1><<<blocks, 256, 0, s>>>(g, xs, ski->n, ski->n_pad, u, nz, qj, y, st, j); break;
    case 2: LOVE_COUNT_LAUNCH(); k_lanczos_gather<T, 2><<<blocks, 256, 0, s>>>(g, xs, ski->n, ski->n_pad, u, nz, qj, y, st, j); break;
    default: LOVE_COUNT_LAUNCH(); k_lanczos_gather<T, 3><<<blocks, 256, 0, s>>>(g, xs, ski->n, ski->n_pad, u, nz, qj, y, st, j);
  }
  return cuda_check(cudaGetLastError());
}

template <typename T>
love_status make_qmap(T* Q, int64_t ldq, int kcols, int bc, CUtensorMap* out) {
  // resolved once (thread-safe static initialisation: the mean solve's host
  // thread builds tensor maps beside the caller's)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e =
        cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
    return e == cudaSuccess && q == cudaDriverEntryPointSuccess ? (PFN_cuTensorMapEncodeTiled_v12000)f : nullptr;
  }();
  if (!encode) return LOVE_ERR_UNSUPPORTED;
  cuuint64_t dims[2] = {(cuuint64_t)ldq, (cuuint64_t)kcols};
  cuuint64_t strides[1] = {(cuuint64_t)ldq * sizeof(T)};
  cuuint32_t box[2] = {(cuuint32_t)TILE_R, (cuuint32_t)bc};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(out, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                      (void*)Q, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LOVE_OK : LOVE_ERR_CUDA;
}


}  // namespace

template <typename T, int MODE>
love_status reorth_sweep(TileArgs<T> a, cudaStream_t s) {
  return tile_run<T, MODE>(a, s);
}
template love_status reorth_sweep<float, MODE_DOT>(TileArgs<float>, cudaStream_t);
template love_status reorth_sweep<float, MODE_UPDATE_DOT>(TileArgs<float>, cudaStream_t);
template love_status reorth_sweep<float, MODE_UPDATE_NORM>(TileArgs<float>, cudaStream_t);
template love_status reorth_sweep<double, MODE_DOT>(TileArgs<double>, cudaStream_t);
template love_status reorth_sweep<double, MODE_UPDATE_DOT>(TileArgs<double>, cudaStream_t);
template love_status reorth_sweep<double, MODE_UPDATE_NORM>(TileArgs<double>, cudaStream_t);


int smem_limit(const void* kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> limits;
  std::lock_guard<std::mutex> lock(mu);
  auto it = limits.find(kernel);
  if (it != limits.end()) return it->second;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return -1;
  const int l = std::max(optin - (int)fa.sharedSizeBytes, 48 * 1024);
  limits.emplace(kernel, l);
  return l;
}

int num_sms() {
  static const int cached = [] {   // thread-safe static initialisation
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return cached;
}

// ---------------------------------------------------------------------------
template <typename T>
love_status ski_mvm_sorted(love_ski* ski, const T* v, T* out, void* work, cudaStream_t s) {
  const GridHost& gh = ski->grid;
  T* u = (T*)work;
  T* u2 = u + gh.m;
  void* fftw = (void*)(u2 + gh.m);
  LOVE_TRY(scatter_any<T>(ski, v, nullptr, T(1), u, s));
  LOVE_TRY(kuu_apply<T>(gh, ski->fft, u, u2, 1, gh.m, fftw, -1, s));
  return gather_any<T>(ski, u2, T(1), (T)gh.noise, v, out, s);
}

template <typename T>
love_status lanczos_run(love_ski* ski, int k, double tau, double eta, T* Q, int64_t ldq, double* alpha_h,
                        double* beta_h, int* k_eff, int* skipped, cudaStream_t s, float* reorth_ms, bool lowsync) {
  const GridHost& gh = ski->grid;
  const int dim = gh.dim;
  if (k < 1 || k > LOVE_MAX_K) return LOVE_ERR_ARG;
  const int bc = box_cols(sizeof(T));
  if (ski->n_pad % TILE_R) return LOVE_ERR_ARG;
  const int max_grid = std::max(TILE_CTAS_PER_SM * num_sms(), 1024);
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), u(ski->alloc, s), y(ski->alloc, s), fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, sizeof(T) == 8);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * (size_t)max_grid * (k + 1)) ||
      !u.get(sizeof(T) * gh.m * 2) || !y.get(sizeof(T) * ski->n_pad) || !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  T* u1 = u.as<T>();
  T* u2 = u1 + gh.m;
  const GridDev g = gh.dev();
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, k, tau);
  // probe: b = (1/m) W^T K_UU 1
  LOVE_COUNT_LAUNCH(); k_fill<T><<<ceil_div(gh.m, 256), 256, 0, s>>>(u1, gh.m, T(1));
  LOVE_TRY(kuu_apply<T>(gh, ski->fft, u1, u2, 1, gh.m, fw.p, -1, s));
  {
    int pb = std::min(1024, ceil_div(ski->n_pad, 256));
    switch (dim) {
      case 1: LOVE_COUNT_LAUNCH(); k_probe<T, 1><<<pb, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, ski->n_pad, u2, Q, part.as<double2>(), st); break;
      case 2: LOVE_COUNT_LAUNCH(); k_probe<T, 2><<<pb, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, ski->n_pad, u2, Q, part.as<double2>(), st); break;
      default: LOVE_COUNT_LAUNCH(); k_probe<T, 3><<<pb, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, ski->n_pad, u2, Q, part.as<double2>(), st);
    }
    LOVE_LAUNCH_CHECK();
  }
  TileArgs<T> ta{};
  ta.n_pad = ski->n_pad;
  ta.kcols = k;
  ta.bc = bc;
  ta.Q = Q;
  ta.ldq = ldq;
  ta.y = y.as<T>();
  ta.partial = part.as<double2>();
  ta.st = st;
  ta.status = ski->status;
  ta.detect = eta > 0.0;
  ta.eta2 = eta * eta;
  DevBuf gb(ski->alloc, s);
  if (lowsync) {
    // G = Q^T Q, starting from |q_0|^2 = 1
    if (!ta.detect || !gb.get(sizeof(double) * (size_t)k * k)) return LOVE_ERR_OOM;
    LOVE_CUDA(cudaMemsetAsync(gb.p, 0, sizeof(double) * (size_t)k * k, s));
    const double one = 1.0;
    LOVE_CUDA(cudaMemcpyAsync(gb.p, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    ta.gram = gb.as<double>();
  }
  // optional CUDA events around each step's sweeps (reorth_ms)
  std::vector<cudaEvent_t> rev;
  struct EvFree {
    std::vector<cudaEvent_t>& v;
    ~EvFree() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
  } rev_free{rev};
  if (reorth_ms) {
    rev.resize(2 * (size_t)k, nullptr);
    for (auto& e : rev) LOVE_CUDA(cudaEventCreate(&e));
  }
  // 1-D grids with FP32 data: the whole product in one cooperative kernel (k_mvm.cu)
  DevBuf fz(ski->alloc, s);
  bool fused = sizeof(T) == 4 && dim == 1 && !gh.additive && fz.get(ski_mvm_fused_work_bytes(ski));
  if (fused) {
    const love_status fr = ski_mvm_fused_reset(ski, fz.p, s);
    if (fr == LOVE_ERR_UNSUPPORTED) fused = false;
    else LOVE_TRY(fr);
  }
  unsigned int fgen = 0;
  for (int j = 0; j < k; ++j) {
    if (fused) {
      const love_status fr = ski_mvm_fused(ski, reinterpret_cast<float*>(Q + (int64_t)j * ldq), st->scal + j,
                                           &st->done, reinterpret_cast<float*>(y.as<T>()), fz.p, fgen, s);
      if (fr == LOVE_ERR_UNSUPPORTED && j == 0) fused = false;
      else LOVE_TRY(fr);
      fgen += 4;
    }
    if (!fused) {
      // u = W q_j (q_j stored unnormalised, scaled by scal[j])
      LOVE_TRY(scatter_any<T>(ski, Q + (int64_t)j * ldq, st->scal + j, T(1), u1, s));
      LOVE_TRY(kuu_apply<T>(gh, ski->fft, u1, u2, 1, gh.m, fw.p, -1, s));
      // y = W^T u + s^2 q_j (q_j normalised in place)
      LOVE_TRY(lanczos_gather_any<T>(ski, u2, Q + (int64_t)j * ldq, y.as<T>(), st, j, s));
    }
    ta.j = j;
    ta.y = y.as<T>();
    if (reorth_ms) LOVE_CUDA(cudaEventRecord(rev[2 * (size_t)j], s));
    LOVE_TRY(tile_run<T, MODE_DOT>(ta, s));
    LOVE_TRY(tile_run<T, MODE_UPDATE_DOT>(ta, s));
    // detection mode: y' sits in the slot of q_{j+1}; the second pass works
    // in place there (and returns at once when the step was finished)
    if (ta.detect && j + 1 < k) ta.y = Q + (int64_t)(j + 1) * ldq;
    LOVE_TRY(tile_run<T, MODE_UPDATE_NORM>(ta, s));
    if (reorth_ms) LOVE_CUDA(cudaEventRecord(rev[2 * (size_t)j + 1], s));
  }
  int keff = 0, nskip = 0;
  LOVE_CUDA(cudaMemcpyAsync(&nskip, &st->n_skip, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaMemcpyAsync(&keff, &st->k_eff, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaMemcpyAsync(alpha_h, st->alpha, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaMemcpyAsync(beta_h, st->beta, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  *k_eff = keff;
  if (skipped) *skipped = nskip;
  if (reorth_ms) {
    float tot = 0.f;
    for (int j = 0; j < k; ++j) {
      float ms = 0.f;
      LOVE_CUDA(cudaEventElapsedTime(&ms, rev[2 * (size_t)j], rev[2 * (size_t)j + 1]));
      tot += ms;
    }
    *reorth_ms = tot;
  }
  return LOVE_OK;
}

template <typename T>
love_status scatter_multi(love_ski* ski, const T* Q, int64_t ldq, int ncol, T* out, int64_t ldo, cudaStream_t s) {
  GridDev g = ski->grid.dev();
  if (g.additive) {
    for (int e = 0; e < g.dim; ++e) {
      const GridDev ge = component_dev(ski->grid, e);
      int blocks = (int)std::min<int64_t>(((int64_t)ge.m * 32 + 255) / 256, (int64_t)num_sms() * 16);
      LOVE_COUNT_LAUNCH();
      k_scatter_multi<T, 1, 16><<<blocks, 256, 0, s>>>(ge, (const T*)ski->xs1[e], ski->cs1[e], Q, ldq, ncol,
                                                      out + ski->grid.off[e], ldo, ski->map1[e]);
    }
    return cuda_check(cudaGetLastError());
  }
  int blocks = (int)std::min<int64_t>((g.m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  if (sizeof(T) == 4 && g.dim == 1 && ncol <= SMQ_COLS_MAX) {
    const size_t sm = smq_smem(ncol);
    LOVE_TRY(allow_smem(k_scatter_multi_1d, sm));
    LOVE_COUNT_LAUNCH();
    k_scatter_multi_1d<<<(unsigned)ceil_div(g.m, SMQ_NB), SMQ_T, sm, s>>>(
        g, (const float*)ski->xs, ski->cell_start, (const float*)Q, ldq, ncol, (float*)out, ldo);
    return cuda_check(cudaGetLastError());
  }
  switch (g.dim) {
    case 1: LOVE_COUNT_LAUNCH(); k_scatter_multi<T, 1, 16><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Q, ldq, ncol, out, ldo, nullptr); break;
    case 2: LOVE_COUNT_LAUNCH(); k_scatter_multi<T, 2, 16><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Q, ldq, ncol, out, ldo, nullptr); break;
    default:
      if (sizeof(T) == 4) {
        dim3 grid((unsigned)ceil_div(g.g[2], SC3_NB), (unsigned)ceil_div(g.g[1], SC3_NB), (unsigned)ceil_div(g.g[0], SC3_NB));
        constexpr size_t sm = sc3m_smem<T>();
        LOVE_TRY(allow_smem(k_scatter3_multi_block<T>, sm));
        LOVE_COUNT_LAUNCH();
        k_scatter3_multi_block<T><<<grid, 512, sm, s>>>(g, (const T*)ski->xs, ski->cell_start, Q, ldq, ncol, out, ldo);
      } else {
        LOVE_COUNT_LAUNCH(); k_scatter_multi<T, 3, 8><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Q, ldq, ncol, out, ldo, nullptr);
      }
  }
  return cuda_check(cudaGetLastError());
}

// cache build: Rt = K_UU W Q L^{-T}; a = K_UU W z; packed rows [Rt | a | 0]
template <typename T>
love_status build_cache(love_ski* ski, love_cache* c, const T* Q, int64_t ldq, const double* zmean, cudaStream_t s,
                        T* keep_rt, const double* amean) {
  const GridHost& gh = ski->grid;
  const int64_t m = gh.m;
  const int k = c->k_eff;
  DevBuf P0(ski->alloc, s), R0(ski->alloc, s), Rt(ski->alloc, s), av(ski->alloc, s), fw(ski->alloc, s),
      dd(ski->alloc, s), okb(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, std::max(k, 1), sizeof(T) == 8);
  if (!P0.get(sizeof(T) * m * k) || !R0.get(sizeof(T) * m * k) || (!keep_rt && !Rt.get(sizeof(T) * m * k)) ||
      !av.get(sizeof(double) * m * 2) || !fw.get(std::max<size_t>(fwb, 16)) || !dd.get(sizeof(double) * 2 * (k + 1)) ||
      !okb.get(sizeof(int)))
    return LOVE_ERR_OOM;
  // T = L L^T on the device
  T* RT = keep_rt ? keep_rt : Rt.as<T>();  // Rt = K_UU W Q L^{-T}, m x k column-major
  double* dptr = dd.as<double>();
  double* eptr = dptr + (k + 1);
  {
    DevBuf ab(ski->alloc, s);
    if (!ab.get(sizeof(double) * 2 * (k + 1))) return LOVE_ERR_OOM;
    LOVE_CUDA(cudaMemcpyAsync(ab.as<double>(), c->alpha, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    if (k > 1)
      LOVE_CUDA(cudaMemcpyAsync(ab.as<double>() + (k + 1), c->beta, sizeof(double) * (k - 1), cudaMemcpyHostToDevice, s));
    LOVE_COUNT_LAUNCH(); k_tridiag_chol<<<1, 32, 0, s>>>(ab.as<double>(), ab.as<double>() + (k + 1), nullptr, k, dptr, eptr, c->status,
                                    okb.as<int>());
    LOVE_LAUNCH_CHECK();
    int ok = 0;
    LOVE_CUDA(cudaMemcpyAsync(&ok, okb.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (!ok) return LOVE_ERR_NOT_PD;
  }
  // P0 = W Q, R0 = K_UU P0
  LOVE_TRY(scatter_multi<T>(ski, Q, ldq, k, P0.as<T>(), m, s));
  LOVE_TRY(kuu_apply<T>(gh, ski->fft, P0.as<T>(), R0.as<T>(), k, m, fw.p, -1, s));
  int blocks = ceil_div(m, 256);
  LOVE_COUNT_LAUNCH(); k_lt_solve<T><<<blocks, 256, 0, s>>>(R0.as<T>(), m, m, k, dptr, eptr, RT, m);
  LOVE_LAUNCH_CHECK();
  const double* aptr = amean;
  if (zmean && !amean) {
    // a = K_UU W z (eq. pred_mean_ski) in FP64
    double* a1 = av.as<double>();
    size_t fwb2 = fft_work_bytes(gh, ski->fft, 1, true);
    DevBuf fw2(ski->alloc, s);
    if (!fw2.get(std::max<size_t>(fwb2, 16))) return LOVE_ERR_OOM;
    LOVE_TRY(scatter_any<T, double>(ski, zmean, nullptr, 1.0, a1, s));
    LOVE_TRY(kuu_apply<double>(gh, ski->fft, a1, a1 + m, 1, m, fw2.p, -1, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    aptr = a1 + m;
  }
  // packed predict cache
  const int64_t tot = m * c->ld;
  int pb = ceil_div(tot, 256);
  LOVE_COUNT_LAUNCH();
  if (c->cache_dtype == LOVE_BF16)
    k_pack_rows<T, __nv_bfloat16><<<pb, 256, 0, s>>>(RT, m, m, k, aptr, (__nv_bfloat16*)c->Rc, c->ld);
  else if (c->cache_dtype == LOVE_F64)
    k_pack_rows<T, double><<<pb, 256, 0, s>>>(RT, m, m, k, aptr, (double*)c->Rc, c->ld);
  else
    k_pack_rows<T, float><<<pb, 256, 0, s>>>(RT, m, m, k, aptr, (float*)c->Rc, c->ld);
  LOVE_LAUNCH_CHECK();
  // keep P = W Q L^{-T} (column-major, dtype) for gradients
  if (c->flags & LOVE_WANT_GRAD) {
    LOVE_COUNT_LAUNCH(); k_lt_solve<T><<<blocks, 256, 0, s>>>(P0.as<T>(), m, m, k, dptr, eptr, (T*)c->P, m);
    LOVE_LAUNCH_CHECK();
  }
  return cuda_check(cudaStreamSynchronize(s));
}

template love_status ski_mvm_sorted<float>(love_ski*, const float*, float*, void*, cudaStream_t);
template love_status ski_mvm_sorted<double>(love_ski*, const double*, double*, void*, cudaStream_t);
template love_status lanczos_run<float>(love_ski*, int, double, double, float*, int64_t, double*, double*, int*,
                                        int*, cudaStream_t, float*, bool);
template love_status lanczos_run<double>(love_ski*, int, double, double, double*, int64_t, double*, double*, int*,
                                         int*, cudaStream_t, float*, bool);
template love_status scatter_multi<float>(love_ski*, const float*, int64_t, int, float*, int64_t, cudaStream_t);
template love_status scatter_multi<double>(love_ski*, const double*, int64_t, int, double*, int64_t, cudaStream_t);
// mean column of the packed cache: Rc[r, k] = a[r] (cache dtype)
template <typename OutT>
__global__ void k_set_mean_col(const double* __restrict__ a, int64_t m, int k, OutT* __restrict__ out, int ld) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  if constexpr (std::is_same<OutT, __nv_bfloat16>::value) out[r * ld + k] = __double2bfloat16(a[r]);
  else out[r * ld + k] = (OutT)a[r];
}
love_status cache_set_mean(love_cache* c, const double* a, cudaStream_t s) {
  const int64_t m = c->grid.m;
  const int blocks = ceil_div(m, 256);
  LOVE_COUNT_LAUNCH();
  if (c->cache_dtype == LOVE_BF16)
    k_set_mean_col<__nv_bfloat16><<<blocks, 256, 0, s>>>(a, m, c->k_eff, (__nv_bfloat16*)c->Rc, c->ld);
  else if (c->cache_dtype == LOVE_F64)
    k_set_mean_col<double><<<blocks, 256, 0, s>>>(a, m, c->k_eff, (double*)c->Rc, c->ld);
  else
    k_set_mean_col<float><<<blocks, 256, 0, s>>>(a, m, c->k_eff, (float*)c->Rc, c->ld);
  return cuda_check(cudaGetLastError());
}

template love_status build_cache<float>(love_ski*, love_cache*, const float*, int64_t, const double*, cudaStream_t,
                                        float*, const double*);
template love_status build_cache<double>(love_ski*, love_cache*, const double*, int64_t, const double*,
                                         cudaStream_t, double*, const double*);

// permutation helpers used by the API (caller order <-> cell-sorted order)
template <typename T>
love_status permute_in(const T* v, const int32_t* perm, int64_t n, int64_t n_pad, T* out, cudaStream_t s) {
  LOVE_COUNT_LAUNCH(); k_permute_in<T><<<ceil_div(n_pad, 256), 256, 0, s>>>(v, perm, n, n_pad, out);
  return cuda_check(cudaGetLastError());
}
template <typename T>
love_status permute_out(const T* v, const int32_t* perm, int64_t n, T* out, cudaStream_t s) {
  LOVE_COUNT_LAUNCH(); k_permute_out<T><<<ceil_div(n, 256), 256, 0, s>>>(v, perm, n, out);
  return cuda_check(cudaGetLastError());
}
template love_status permute_in<float>(const float*, const int32_t*, int64_t, int64_t, float*, cudaStream_t);
template love_status permute_in<double>(const double*, const int32_t*, int64_t, int64_t, double*, cudaStream_t);
template love_status permute_out<float>(const float*, const int32_t*, int64_t, float*, cudaStream_t);
template love_status permute_out<double>(const double*, const int32_t*, int64_t, double*, cudaStream_t);
}  // namespace love
