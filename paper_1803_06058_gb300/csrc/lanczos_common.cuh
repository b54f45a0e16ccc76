// lanczos_common.cuh -- pieces shared by the n-space Lanczos run (k_lanczos.cu),
// the mean solves (k_cg.cu) and the sampler's multi-launch run (k_sampler.cu):
// the device-side Lanczos / CG scalars, the interpolation stencil and the
// scatter / gather kernels of W, the fixed-order merge of per-CTA partial sums,
// and the reorthogonalisation sweep interface.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda.h>

#include "love_internal.cuh"

namespace love {

constexpr int MERGE_GS = 20;     // partial rows per level-1 merge group and per batch of loads
constexpr int MERGE_MAXG = 64;   // level-1 merge groups (a group grows past MERGE_GS beyond 1280 CTAs)

// device-side Lanczos / CG scalars
struct LanczosState {
  double alpha[LOVE_MAX_K + 1];
  double beta[LOVE_MAX_K + 1];
  double scal[LOVE_MAX_K + 2];   // 1 / |q_j| of the stored (unnormalised) column j
  double coef[LOVE_MAX_K + 1];   // pass-1 coefficients c
  double coef2[LOVE_MAX_K + 1];  // pass-2 coefficients c'
  double maxabs;
  double tau;
  double norm2;
  int done;
  int k_eff;
  int kmax;
  unsigned counter[1 + MERGE_MAXG];    // merge counters of the Lanczos sweeps (all groups, then per group)
  int skip;        // detection mode: the second pass of this step is not needed
  int n_skip;      // second passes skipped so far
  // CG
  double rr, rr0, pap, cg_alpha, cg_beta, tol2;
  int cg_done, cg_iters;
  unsigned counter2[1 + MERGE_MAXG];   // merge counters of the CG reductions
};

// reorthogonalisation sweeps (k_lanczos.cu)
enum { MODE_DOT = 0, MODE_UPDATE_DOT = 1, MODE_UPDATE_NORM = 2 };

template <typename T>
struct TileArgs {
  CUtensorMap qmap;   // Q as a 2-D tensor {rows = ldq, cols = kcols}, box {TILE_R, bc}
  int bc;             // columns per TMA box
  int kpad;           // Q columns of one ring stage: j + 1 rounded up to bc
  int stages;         // ring depth
  int64_t n_pad;      // rows (a multiple of TILE_R)
  int j;
  int kcols;          // allocated columns of Q
  T* Q;
  int64_t ldq;
  T* y;               // [n_pad], 16-byte aligned
  double2* partial;   // [gridDim][kcols + 1]
  LanczosState* st;
  DevStatus* status;
  int detect;         // skip the second pass when |Q_j^T y'| <= eta |y'|
  double eta2;        // eta^2
  double* gram;       // low-synchronisation mode: Q^T Q (kcols x kcols, FP64), else nullptr
  int reverse;        // walk the row tiles from the last one (tiled sweeps)
};

// Q as a 2-D tensor for TMA: rows (inner, n_pad) x columns (kcols), box
// {TILE_R rows, bc columns}; columns past kcols read as zeros
inline int box_cols(size_t elem) { return elem == 4 ? 8 : 4; }
// one sweep over the row tiles of [Q_j | y] (DOT, UPDATE_DOT or UPDATE_NORM):
// the TMA-ring tile kernel, or the register kernel for short vectors
template <typename T, int MODE>
love_status reorth_sweep(TileArgs<T> a, cudaStream_t s);

namespace {

constexpr int TILE_R = 128;     // rows per reorthogonalisation tile
constexpr int TILE_T = 256;     // threads per tile CTA (two per row in the update)
constexpr int NWARP = TILE_T / 32;
constexpr int TILE_CTAS_PER_SM = 2;


template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = DotAccF; };
template <> struct AccOf<double> { using type = DotAccD; };

// A partial sum in a 16-byte slot of a partial table, stored exactly in its
// first 8 bytes: the two floats of a double-float sum, or the double
template <typename Acc> struct SlotOf;
template <> struct SlotOf<DotAccF> { using type = float2; };
template <> struct SlotOf<DotAccD> { using type = double; };
__device__ __forceinline__ void acc_store(double2* p, const DotAccF& a) {
  *reinterpret_cast<float2*>(p) = make_float2(a.s, a.c);
}
__device__ __forceinline__ void acc_store(double2* p, const DotAccD& a) { *reinterpret_cast<double*>(p) = a.s; }
__device__ __forceinline__ void acc_merge(DotAccF& a, float2 v) { a.merge(v.x, v.y); }
__device__ __forceinline__ void acc_merge(DotAccD& a, double v) { a.merge(v, 0.0); }

// ---------------------------------------------------------------------------
// per-point interpolation (4^D nonzeros)
template <typename T, int D>
struct Stencil {
  int base[D];
  T w[D][4];
  bool ok;
  __device__ __forceinline__ void compute(const T* xp, const GridDev& g) {
    ok = true;
#pragma unroll
    for (int e = 0; e < D; ++e) ok &= keys_weights(grid_coord(xp[e], g, e), g.g[e], base[e], w[e]);
  }
  // sum_r w_r u[node_r], weights in T, values and accumulation in V
  template <typename V>
  __device__ __forceinline__ V apply(const V* __restrict__ u, const GridDev& g) const {
    V acc = V(0);
    if (D > 1 && g.additive) {
      // stacked interpolation vector: 4 nonzeros per 1-D block
#pragma unroll
      for (int e = 0; e < D; ++e) {
        const V* p = u + g.off[e] + (base[e] - 1);
        V a = V(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) a += (V)w[e][r] * p[r];
        acc += a;
      }
      return acc;
    }
    if (D == 1) {
      const V* p = u + (base[0] - 1);
#pragma unroll
      for (int r = 0; r < 4; ++r) acc += (V)w[0][r] * p[r];
    } else if (D == 2) {
#pragma unroll
      for (int r0 = 0; r0 < 4; ++r0) {
        const V* p = u + (int64_t)(base[0] - 1 + r0) * g.stride[0] + (base[1] - 1);
        V a = V(0);
#pragma unroll
        for (int r1 = 0; r1 < 4; ++r1) a += (V)w[1][r1] * p[r1];
        acc += (V)w[0][r0] * a;
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < 4; ++r0) {
        V a0 = V(0);
#pragma unroll
        for (int r1 = 0; r1 < 4; ++r1) {
          const V* p = u + (int64_t)(base[0] - 1 + r0) * g.stride[0] + (int64_t)(base[1] - 1 + r1) * g.stride[1] +
                       (base[2] - 1);
          V a = V(0);
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) a += (V)w[2][r2] * p[r2];
          a0 += (V)w[1][r1] * a;
        }
        acc += (V)w[0][r0] * a0;
      }
    }
    return acc;
  }
};

// weight of a cell-sorted point at grid node nd[] (same arithmetic as keys_weights)
template <typename T, int D>
__device__ __forceinline__ T node_weight(const T* xp, const GridDev& g, const int* nd) {
  T w = T(1);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    T s = grid_coord(xp[e], g, e);
    int i = (int)floor(s);
    if (i > g.g[e] - 3) i = g.g[e] - 3;
    T f = s - T(i);
    int r = nd[e] - (i - 1);
    w *= keys_u(f + T(1) - T(r));
  }
  return w;
}

// ranges of sorted points whose stencil covers node nd[]: 4^(D-1) ranges, each
// 4 consecutive cells of the last dimension.  Lane l < NR computes range l.
template <int D>
struct NodeRanges {
  static constexpr int NR = D == 1 ? 1 : (D == 2 ? 4 : 16);
  int lo[NR];
  int ex[NR];  // exclusive prefix of lengths
  int total;
  __device__ __forceinline__ void build(const GridDev& g, const int* nd, const int* __restrict__ cell_start,
                                        int lane) {
    int mylo = 0, mylen = 0;
    if (lane < NR) {
      int64_t cbase = 0;
      bool ok = true;
      int rem = lane;
#pragma unroll
      for (int e = 0; e < D - 1; ++e) {
        int re = rem & 3;
        rem >>= 2;
        int c = nd[e] - re + 1;
        if (c < 0 || c >= g.g[e]) ok = false;
        cbase += (int64_t)c * g.stride[e];
      }
      int clo = max(nd[D - 1] - 2, 0), chi = min(nd[D - 1] + 1, g.g[D - 1] - 1);
      if (ok && clo <= chi) {
        mylo = cell_start[cbase + clo];
        mylen = cell_start[cbase + chi + 1] - mylo;
      }
    }
    int incl = mylen;
#pragma unroll
    for (int o = 1; o < NR; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int excl = incl - mylen;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      lo[q] = __shfl_sync(0xffffffffu, mylo, q);
      ex[q] = __shfl_sync(0xffffffffu, excl, q);
    }
    total = __shfl_sync(0xffffffffu, incl, NR - 1);
  }
  __device__ __forceinline__ int point(int f) const {
    int ri = 0;
#pragma unroll
    for (int q = 1; q < NR; ++q)
      if (ex[q] <= f) ri = q;
    return lo[ri] + (f - ex[ri]);
  }
};

template <int D>
__device__ __forceinline__ void node_index(int64_t node, const GridDev& g, int* nd) {
  int64_t r = node;
#pragma unroll
  for (int e = D - 1; e >= 0; --e) {
    nd[e] = (int)(r % g.g[e]);
    r /= g.g[e];
  }
}

// u[node] = scale * sum over sorted points of w_p(node) v[p]   (u = W v).
// A node collects ~4 n/m points in 1-D (400 on the n = 1e6, m = 1e4 grid), so
// the sum is accumulated in double-float (Dot2) and rounded once.
// map (additive composition): position of each sorted point in the order of v
template <typename T, int D, typename V = T>
__global__ void k_scatter(GridDev g, const T* __restrict__ xs, const int* __restrict__ cell_start,
                          const V* __restrict__ v, const double* __restrict__ scal, V scale, V* __restrict__ u,
                          const V* __restrict__ v2, const double* __restrict__ beta2, const int* __restrict__ skip,
                          const int32_t* __restrict__ map) {
  // with v2: scatters v + beta2 v2 (the CG direction r + beta p, formed on the fly)
  using Acc = typename AccOf<V>::type;
  if (skip && *skip) return;
  const V b2 = v2 ? (V)(*beta2) : V(0);
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double sc = (double)scale * (scal ? *scal : 1.0);
  for (int64_t node = wg; node < g.m; node += nw) {
    int nd[D];
    node_index<D>(node, g, nd);
    NodeRanges<D> rg;
    rg.build(g, nd, cell_start, lane);
    Acc acc;
    acc.zero();
    for (int f = lane; f < rg.total; f += 32) {
      int p = rg.point(f);
      const int pv = map ? map[p] : p;
      V val = v[pv];
      if (v2) val += b2 * v2[pv];
      acc.add_prod((V)node_weight<T, D>(xs + (int64_t)p * D, g, nd), val);
    }
    warp_merge(acc);
    if (lane == 0) u[node] = (V)(acc.value() * sc);
  }
}

// u = W v on a 3-D grid, a CTA per 8 x 8 x 8 block of nodes and a thread per
// node.  The points of the block's 11 x 11 x 11 halo cells (cells n - 2 ..
// n + 1 feed node n) are 121 contiguous runs of the cell-sorted order; they
// are staged once in shared memory as (cell, fractional coordinate, value),
// and each thread then sums over the points of its 64 cells in a fixed order
// (double-float), with the weights evaluated as in node_weight.  A block
// whose halo holds more than SC3_CAP points reads them from global memory.
constexpr int SC3_NB = 8, SC3_HC = SC3_NB + 3, SC3_RUNS = SC3_HC * SC3_HC, SC3_CAP = 4096;
// dynamic shared memory: run offsets, per-run cell starts, run starts, then the
// staged points (values, fractional coordinates, cells)
constexpr size_t SC3_OFF_CS = 512, SC3_OFF_RG = 6400, SC3_OFF_PV = 6912;
template <typename V>
constexpr size_t sc3_smem() {
  return SC3_OFF_PV + (size_t)SC3_CAP * sizeof(V) + (size_t)SC3_CAP * 3 * sizeof(float) + (size_t)SC3_CAP * 4;
}

template <typename T, typename V>
__global__ void __launch_bounds__(512) k_scatter3_block(GridDev g, const T* __restrict__ xs,
                                                        const int* __restrict__ cell_start, const V* __restrict__ v,
                                                        const double* __restrict__ scal, V scale, V* __restrict__ u,
                                                        const V* __restrict__ v2, const double* __restrict__ beta2,
                                                        const int* __restrict__ skip) {
  using Acc = typename AccOf<V>::type;
  static_assert((SC3_RUNS + 1) * 4 <= SC3_OFF_CS && SC3_OFF_CS + SC3_RUNS * (SC3_HC + 1) * 4 <= SC3_OFF_RG &&
                    SC3_OFF_RG + SC3_RUNS * 4 <= SC3_OFF_PV && SC3_OFF_PV % 16 == 0,
                "shared-memory layout");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int* run_off = reinterpret_cast<int*>(smem_raw);                                    // [SC3_RUNS + 1]
  int (*cs_loc)[SC3_HC + 1] = reinterpret_cast<int (*)[SC3_HC + 1]>(smem_raw + SC3_OFF_CS);  // cell starts
  int* run_g = reinterpret_cast<int*>(smem_raw + SC3_OFF_RG);                         // global run starts
  V* pv = reinterpret_cast<V*>(smem_raw + SC3_OFF_PV);                                // values
  float (*pf)[3] = reinterpret_cast<float (*)[3]>(smem_raw + SC3_OFF_PV + SC3_CAP * sizeof(V));  // fractions
  unsigned char (*pc)[4] = reinterpret_cast<unsigned char (*)[4]>(
      smem_raw + SC3_OFF_PV + SC3_CAP * sizeof(V) + SC3_CAP * 3 * sizeof(float));  // halo cells
  if (skip && *skip) return;
  const V b2 = v2 ? (V)(*beta2) : V(0);
  const int t = threadIdx.x;
  int N[3] = {(int)blockIdx.z * SC3_NB, (int)blockIdx.y * SC3_NB, (int)blockIdx.x * SC3_NB};
  int c_lo[3], c_hi[3];   // halo cells, clipped to the grid
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    c_lo[e] = max(N[e] - 2, 0);
    c_hi[e] = min(N[e] + SC3_NB, g.g[e] - 1);
  }
  const int h0 = c_hi[0] - c_lo[0] + 1, h1 = c_hi[1] - c_lo[1] + 1, h2 = c_hi[2] - c_lo[2] + 1;
  // runs along the last dimension: lengths, then an exclusive scan
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
    const int lane = t & 31, w = t >> 5;
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
        V val = v[p];
        if (v2) val += b2 * v2[p];
        pv[slot] = val;
      }
    }
  }
  __syncthreads();
  const int nd[3] = {N[0] + t / 64, N[1] + (t / 8) % 8, N[2] + t % 8};
  if (nd[0] >= g.g[0] || nd[1] >= g.g[1] || nd[2] >= g.g[2]) return;
  Acc acc;
  acc.zero();
  const int zlo = max(nd[2] - 2, c_lo[2]) - c_lo[2], zhi = min(nd[2] + 1, c_hi[2]) - c_lo[2];
  for (int dx = 0; dx < 4; ++dx) {
    const int a = nd[0] - 2 + dx - c_lo[0];
    if (a < 0 || a >= h0) continue;
    for (int dy = 0; dy < 4; ++dy) {
      const int b = nd[1] - 2 + dy - c_lo[1];
      if (b < 0 || b >= h1 || zlo > zhi) continue;
      const int r = a * SC3_HC + b;
      const int q0 = cs_loc[r][zlo], q1 = cs_loc[r][zhi + 1];
      for (int q = q0; q < q1; ++q) {
        V wv;
        if (staged) {
          const int slot = run_off[r] + q;
          float wt = 1.f;
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const int rr = nd[e] - ((int)pc[slot][e] + c_lo[e] - 1);
            wt *= keys_u(pf[slot][e] + 1.f - (float)rr);
          }
          wv = pv[slot];
          acc.add_prod((V)wt, wv);
        } else {
          const int p = run_g[r] + q;
          V val = v[p];
          if (v2) val += b2 * v2[p];
          acc.add_prod((V)node_weight<T, 3>(xs + (int64_t)p * 3, g, nd), val);
        }
      }
    }
  }
  const double sc = (double)scale * (scal ? *scal : 1.0);
  u[(int64_t)nd[0] * g.stride[0] + (int64_t)nd[1] * g.stride[1] + nd[2]] = (V)(acc.value() * sc);
}


// out[p] = a * sum_r w_r u[node_r] + b * v[p]   (p < n; 0 on padding rows)
template <typename T, int D>
__global__ void k_gather(GridDev g, const T* __restrict__ xs, int64_t n, int64_t n_pad, const T* __restrict__ u,
                         T a, T b, const T* __restrict__ v, T* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pad) return;
  T r = T(0);
  if (p < n) {
    Stencil<T, D> st;
    st.compute(xs + p * D, g);
    r = a * st.apply(u, g);
    if (v) r += b * v[p];
  }
  out[p] = r;
}

// ---------------------------------------------------------------------------
// block reduction of a DotAcc into partial[blockIdx.x]; then the merge of all
// CTA partials into result[0..ncols) (fixed order).
template <typename Acc>
__device__ __forceinline__ void block_merge(Acc& a, Acc* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  warp_merge(a);
  if (lane == 0) sm[w] = a;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    Acc b;
    b.zero();
    if (lane < nw) b = sm[lane];
    warp_merge(b);
    if (lane == 0) sm[0] = b;
  }
  __syncthreads();
  a = sm[0];
}

// The per-CTA partial rows (sums in columns 0..ncols) are merged in two levels
// so that no CTA walks the whole table through a chain of L2 round trips: the
// CTAs form groups of `gs` consecutive indices; the last CTA of a group to
// arrive merges the group's rows (in index order) into the group's first row;
// the last group to arrive merges those rows (in group order) into result.  A
// thread owns a column and keeps a batch of MERGE_GS row loads in flight, so a
// sum's merge order never depends on how many sums are merged beside it.
// counters: [0] the group count, [1 + g] group g's count; all are zero between
// launches (each is reset by the CTA that saw it complete).
template <typename Acc>
__device__ __forceinline__ Acc merge_column(const double2* p, int64_t rstride, int nrows) {
  using Slot = typename SlotOf<Acc>::type;
  Acc a;
  a.zero();
  for (int r0 = 0; r0 < nrows; r0 += MERGE_GS) {
    Slot v[MERGE_GS];
#pragma unroll
    for (int u = 0; u < MERGE_GS; ++u)
      if (r0 + u < nrows) v[u] = __ldcg(reinterpret_cast<const Slot*>(p + (int64_t)(r0 + u) * rstride));
#pragma unroll
    for (int u = 0; u < MERGE_GS; ++u)
      if (r0 + u < nrows) acc_merge(a, v[u]);
  }
  return a;
}

// Returns true in the one CTA that formed result (after the merge, with a copy
// in sh_result when given), so the caller can finish scalar work there.
// G partial rows (one per CTA, or per chunk of a batched launch); b: this CTA's row.
template <typename Acc>
__device__ bool last_cta_reduce(double2* partial, int stride, int ncols, double* result, unsigned* counters,
                                double* sh_result, int G, int b) {
  __shared__ int is_last;
  const int gs = max(MERGE_GS, (G + MERGE_MAXG - 1) / MERGE_MAXG);
  const int ng = (G + gs - 1) / gs;
  const int grp = b / gs;
  const int r0 = grp * gs, nr = min(gs, G - r0);
  const int tid = threadIdx.x, nthr = blockDim.x;
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&counters[1 + grp], 1u) == (unsigned)(nr - 1));
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double2* rows = partial + (int64_t)r0 * stride;
  for (int i = tid; i < ncols; i += nthr) acc_store(rows + i, merge_column<Acc>(rows + i, stride, nr));
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    counters[1 + grp] = 0u;
    is_last = (atomicAdd(&counters[0], 1u) == (unsigned)(ng - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  for (int i = tid; i < ncols; i += nthr) {
    const double v = merge_column<Acc>(partial + i, (int64_t)gs * stride, ng).value();
    result[i] = v;
    if (sh_result) sh_result[i] = v;
  }
  __syncthreads();
  if (tid == 0) counters[0] = 0u;
  return true;
}
template <typename Acc>
__device__ __forceinline__ bool last_cta_reduce(double2* partial, int stride, int ncols, double* result,
                                                unsigned* counters, double* sh_result = nullptr) {
  return last_cta_reduce<Acc>(partial, stride, ncols, result, counters, sh_result, (int)gridDim.x, (int)blockIdx.x);
}

template <typename T>
__global__ void k_fill(T* p, int64_t n, T v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_state_init(LanczosState* st, int kmax, double tau) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->maxabs = 0.0;
  st->tau = tau;
  st->done = 0;
  st->k_eff = kmax;
  st->kmax = kmax;
  for (int i = 0; i <= MERGE_MAXG; ++i) st->counter[i] = st->counter2[i] = 0u;
  st->cg_done = 0;
  st->cg_iters = 0;
  st->skip = 0;
  st->n_skip = 0;
}

// ---------------------------------------------------------------------------

// end of step j: beta_j = sqrt(norm2); stop at kmax, on NaN or on breakdown
// (beta_j <= tau max|alpha|), else the scale of the stored q_{j+1}
__device__ void finish_step(LanczosState* st, DevStatus* status, int j) {
  const double b = sqrt(st->norm2);
  st->beta[j] = b;
  if (!isfinite(b)) {
    dev_flag(status, LOVE_ERR_NAN);
    st->done = 1;
    st->k_eff = j;
  } else if (j + 1 >= st->kmax) {
    st->k_eff = st->kmax;
    st->done = 1;
  } else if (b <= st->tau * st->maxabs) {
    st->k_eff = j + 1;
    st->done = 1;
  } else {
    st->scal[j + 1] = 1.0 / b;
  }
}

// End of a sweep (both kernel shapes): per-CTA partials of the column dots
// (or of |y|^2), the last CTA's fixed-order merge, and the step's scalar work
// (alpha_j; the detection test; beta_j, breakdown and the next scale).
// A: TileArgs<T>, or any argument block with the members read here (st, j,
// kcols, partial, detect, eta2, gram, status).  G partial rows, b this CTA's.
template <typename T, int MODE, int KPW, typename A>
__device__ __forceinline__ void sweep_epilogue(const A& a, typename AccOf<T>::type (&acc)[KPW],
                                               typename AccOf<T>::type& nacc, typename AccOf<T>::type* red,
                                               double2* scratch, int G, int b) {
  using Acc = typename AccOf<T>::type;
  LanczosState* st = a.st;
  const int j = a.j;
  const int ncols = j + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- CTA partials
  const int pstride = a.kcols + 1;
  if (MODE == MODE_UPDATE_NORM) {
    block_merge(nacc, red);
    if (tid == 0) acc_store(a.partial + (int64_t)b * pstride, nacc);
  } else {
#pragma unroll
    for (int s2 = 0; s2 < KPW; ++s2) {
      const int i = warp + NWARP * s2;
      warp_merge(acc[s2]);
      if (lane == 0 && i < ncols) acc_store(a.partial + (int64_t)b * pstride + i, acc[s2]);
    }
    if (MODE == MODE_UPDATE_DOT && a.detect) {   // |y'|^2 in slot j + 1
      block_merge(nacc, red);
      if (tid == 0) acc_store(a.partial + (int64_t)b * pstride + ncols, nacc);
    }
  }
  double* result = MODE == MODE_UPDATE_NORM ? &st->norm2 : (MODE == MODE_UPDATE_DOT ? st->coef2 : st->coef);
  const int nres = MODE == MODE_UPDATE_NORM ? 1 : ncols + (MODE == MODE_UPDATE_DOT && a.detect ? 1 : 0);
  // scratch (shared memory, at least j + 1 + blockDim.x doubles): the merged
  // sums, then the pieces of the low-synchronisation product
  double* cm = reinterpret_cast<double*>(scratch);
  bool last = last_cta_reduce<Acc>(a.partial, pstride, nres, result, st->counter,
                                   MODE == MODE_UPDATE_NORM ? nullptr : cm, G, b);
  if (!last) return;
  if (MODE == MODE_DOT && a.gram != nullptr) {
    // low-synchronisation form: the second Gram-Schmidt pass folded into the
    // first through the Gram matrix G = Q_j^T Q_j, c <- c + (c - G c) (the
    // coefficients CGS2's second pass would find on y - Q_j c); alpha_j keeps
    // the first-pass c_j.  G is stored symmetric, so row i of G is read as
    // column i (coalesced across a warp); the threads split the l range of
    // every row into `parts` pieces (16 loads in flight each), then add the
    // pieces in a fixed order.
    const double* G = a.gram;
    double* pp = cm + ncols;   // [parts][ncols], parts * ncols <= blockDim.x
    const int parts = max(1, (int)blockDim.x / ncols);
    const int span = (ncols + parts - 1) / parts;
    for (int t = tid; t < parts * ncols; t += blockDim.x) {
      const int part = t / ncols, i = t - part * ncols;
      const int lb = part * span, le = min(ncols, lb + span);
      double v = 0.0;
      for (int l0 = lb; l0 < le; l0 += 16) {
        double gl[16];
#pragma unroll
        for (int u = 0; u < 16; ++u)
          gl[u] = l0 + u < le ? __ldcg(G + (int64_t)(l0 + u) * a.kcols + i) : 0.0;
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (l0 + u < le) v = fma(gl[u], cm[l0 + u], v);
      }
      pp[t] = v;
    }
    __syncthreads();
    for (int i = tid; i < ncols; i += blockDim.x) {
      double v = 0.0;
      for (int p = 0; p < parts; ++p) v += pp[p * ncols + i];
      st->coef[i] = 2.0 * cm[i] - v;
    }
    if (tid != 0) return;
    const double c1j = cm[j];
    st->alpha[j] = c1j;
    if (!isfinite(c1j)) {
      dev_flag(a.status, LOVE_ERR_NAN);
      st->done = 1;
      st->k_eff = j;
    }
    st->maxabs = fmax(st->maxabs, fabs(c1j));
    return;
  }
  if (MODE == MODE_UPDATE_DOT && a.detect) {
    // the detection test on the measured c' = Q_j^T y' (warp 0, fixed order)
    __shared__ int skip_sh;
    if (warp == 0) {
      double c2 = 0.0;
      for (int i = lane; i < ncols; i += 32) c2 = fma(cm[i], cm[i], c2);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
      if (lane == 0) skip_sh = c2 <= a.eta2 * cm[ncols];   // false for NaN: the second pass reports it
    }
    __syncthreads();
    const bool skip = skip_sh != 0;
    const double yn = cm[ncols];
    if (a.gram != nullptr && j + 1 < a.kcols) {
      // row and column j + 1 of G: the measured dots of q_{j+1} = y'/|y'| with
      // Q_j (zero when the second pass runs and removes them)
      double* G = a.gram;
      const int64_t ld = a.kcols;
      const double inv = skip && yn > 0.0 ? 1.0 / sqrt(yn) : 0.0;
      for (int i = tid; i < ncols; i += blockDim.x) {
        const double g = cm[i] * inv;
        G[(int64_t)(j + 1) * ld + i] = g;
        G[(int64_t)i * ld + (j + 1)] = g;
      }
      if (tid == 0) G[(int64_t)(j + 1) * ld + (j + 1)] = 1.0;
    }
    if (tid != 0) return;
    st->skip = skip;
    if (skip) {
      st->n_skip += 1;
      st->norm2 = yn;
      finish_step(st, a.status, j);
    }
    return;
  }
  if (tid != 0) return;
  if (MODE == MODE_DOT) {
    double al = cm[j];
    st->alpha[j] = al;
    if (!isfinite(al)) {
      dev_flag(a.status, LOVE_ERR_NAN);
      st->done = 1;
      st->k_eff = j;
    }
    st->maxabs = fmax(st->maxabs, fabs(al));
  } else if (MODE == MODE_UPDATE_NORM) {
    finish_step(st, a.status, j);
  }
}

struct DevBuf {
  const Allocator* al;
  cudaStream_t s;
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf(const Allocator& a, cudaStream_t st) : al(&a), s(st) {}
  bool get(size_t b) {
    bytes = b;
    p = scratch_alloc(*al, b, s);
    return p != nullptr || b == 0;
  }
  ~DevBuf() {
    if (p) scratch_free(*al, p, bytes, s);
  }
  template <typename X> X* as() const { return (X*)p; }
};

template <typename T, int D, typename V>
love_status scatter_launch(love_ski* ski, const V* v, const double* scal, V scale, V* u, cudaStream_t s,
                           const V* v2, const double* beta2, const int* skip) {
  GridDev g = ski->grid.dev();
  if (D == 3 && sizeof(T) == 4) {
    dim3 grid((unsigned)ceil_div(g.g[2], SC3_NB), (unsigned)ceil_div(g.g[1], SC3_NB), (unsigned)ceil_div(g.g[0], SC3_NB));
    constexpr size_t sm = sc3_smem<V>();
    LOVE_TRY(allow_smem(k_scatter3_block<T, V>, sm));
    LOVE_COUNT_LAUNCH();
    k_scatter3_block<T, V><<<grid, 512, sm, s>>>(g, (const T*)ski->xs, ski->cell_start, v, scal, scale, u, v2, beta2, skip);
    return cuda_check(cudaGetLastError());
  }
  int64_t warps = g.m;
  int blocks = (int)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)num_sms() * 16);
  LOVE_COUNT_LAUNCH(); k_scatter<T, D, V><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, v, scal, scale, u, v2, beta2, skip, nullptr);
  return cuda_check(cudaGetLastError());
}
// additive composition: block e of u = W_e v, over the points sorted in dimension e
template <typename T, typename V>
love_status scatter_additive(love_ski* ski, const V* v, const double* scal, V scale, V* u, cudaStream_t s,
                             const V* v2, const double* beta2, const int* skip) {
  for (int e = 0; e < ski->grid.dim; ++e) {
    const GridDev g = component_dev(ski->grid, e);
    int blocks = (int)std::min<int64_t>(((int64_t)g.m * 32 + 255) / 256, (int64_t)num_sms() * 16);
    LOVE_COUNT_LAUNCH();
    k_scatter<T, 1, V><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs1[e], ski->cs1[e], v, scal, scale,
                                               u + ski->grid.off[e], v2, beta2, skip, ski->map1[e]);
  }
  return cuda_check(cudaGetLastError());
}
// u = W v (or W (v + beta2 v2)) with coordinates of type T (the ski dtype) and values of type V
template <typename T, typename V = T>
love_status scatter_any(love_ski* ski, const V* v, const double* scal, V scale, V* u, cudaStream_t s,
                        const V* v2 = nullptr, const double* beta2 = nullptr, const int* skip = nullptr) {
  if (ski->grid.additive) return scatter_additive<T, V>(ski, v, scal, scale, u, s, v2, beta2, skip);
  switch (ski->grid.dim) {
    case 1: return scatter_launch<T, 1, V>(ski, v, scal, scale, u, s, v2, beta2, skip);
    case 2: return scatter_launch<T, 2, V>(ski, v, scal, scale, u, s, v2, beta2, skip);
    default: return scatter_launch<T, 3, V>(ski, v, scal, scale, u, s, v2, beta2, skip);
  }
}
template <typename T>
love_status gather_any(love_ski* ski, const T* u, T a, T b, const T* v, T* out, cudaStream_t s) {
  GridDev g = ski->grid.dev();
  int blocks = ceil_div(ski->n_pad, 256);
  switch (g.dim) {
    case 1: LOVE_COUNT_LAUNCH(); k_gather<T, 1><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, ski->n_pad, u, a, b, v, out); break;
    case 2: LOVE_COUNT_LAUNCH(); k_gather<T, 2><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, ski->n_pad, u, a, b, v, out); break;
    default: LOVE_COUNT_LAUNCH(); k_gather<T, 3><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, ski->n_pad, u, a, b, v, out);
  }
  return cuda_check(cudaGetLastError());
}


// a stored Krylov column scaled in place by *scal (no-op after breakdown)
template <typename QT>
__global__ void k_normalize_col(QT* __restrict__ q, int64_t n_pad, const double* __restrict__ scal,
                                const LanczosState* st) {
  if (st->done) return;
  const QT sc = (QT)*scal;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x)
    q[i] *= sc;
}

}  // namespace
}  // namespace love
