// k_lanczos.cu -- SKI matrix-vector products, Lanczos with full
// reorthogonalisation, CG, and the LOVE cache build.
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

namespace {

constexpr int GM_R = 40;        // GMRES restart length (Arnoldi steps per cycle)
constexpr int GM_CYCLES = 4;    // GMRES cycles before the mean solve falls back to plain CG
constexpr int TILE_R = 128;     // rows per reorthogonalisation tile
constexpr int TILE_T = 256;     // threads per tile CTA (two per row in the update)
constexpr int NWARP = TILE_T / 32;

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
template <typename Acc>
__device__ bool last_cta_reduce(double2* partial, int stride, int ncols, double* result, unsigned* counters,
                                double* sh_result = nullptr) {
  __shared__ int is_last;
  const int G = gridDim.x;
  const int gs = max(MERGE_GS, (G + MERGE_MAXG - 1) / MERGE_MAXG);
  const int ng = (G + gs - 1) / gs;
  const int grp = (int)blockIdx.x / gs;
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

// ---------------------------------------------------------------------------
// Lanczos tile kernels
enum { MODE_DOT = 0, MODE_UPDATE_DOT = 1, MODE_UPDATE_NORM = 2 };

// 2-D tiled bulk tensor copy (TMA) of a box of Q into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst_smem, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst_smem)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

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
template <typename T, int MODE, int KPW>
__device__ __forceinline__ void sweep_epilogue(const TileArgs<T>& a, typename AccOf<T>::type (&acc)[KPW],
                                               typename AccOf<T>::type& nacc, typename AccOf<T>::type* red,
                                               double2* scratch) {
  using Acc = typename AccOf<T>::type;
  LanczosState* st = a.st;
  const int j = a.j;
  const int ncols = j + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- CTA partials
  const int pstride = a.kcols + 1;
  if (MODE == MODE_UPDATE_NORM) {
    block_merge(nacc, red);
    if (tid == 0) acc_store(a.partial + (int64_t)blockIdx.x * pstride, nacc);
  } else {
#pragma unroll
    for (int s2 = 0; s2 < KPW; ++s2) {
      const int i = warp + NWARP * s2;
      warp_merge(acc[s2]);
      if (lane == 0 && i < ncols) acc_store(a.partial + (int64_t)blockIdx.x * pstride + i, acc[s2]);
    }
    if (MODE == MODE_UPDATE_DOT && a.detect) {   // |y'|^2 in slot j + 1
      block_merge(nacc, red);
      if (tid == 0) acc_store(a.partial + (int64_t)blockIdx.x * pstride + ncols, nacc);
    }
  }
  double* result = MODE == MODE_UPDATE_NORM ? &st->norm2 : (MODE == MODE_UPDATE_DOT ? st->coef2 : st->coef);
  const int nres = MODE == MODE_UPDATE_NORM ? 1 : ncols + (MODE == MODE_UPDATE_DOT && a.detect ? 1 : 0);
  // scratch (shared memory, at least j + 1 + blockDim.x doubles): the merged
  // sums, then the pieces of the low-synchronisation product
  double* cm = reinterpret_cast<double*>(scratch);
  bool last = last_cta_reduce<Acc>(a.partial, pstride, nres, result, st->counter,
                                   MODE == MODE_UPDATE_NORM ? nullptr : cm);
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
  if (st->done || (MODE == MODE_UPDATE_NORM && a.detect && st->skip)) return;
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

  if (MODE == MODE_UPDATE_DOT || MODE == MODE_UPDATE_NORM) {
    const double* c = MODE == MODE_UPDATE_DOT ? st->coef : st->coef2;
    for (int i = tid; i < ncols; i += TILE_T) cf[i] = (T)c[i];
  }
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
  if (tid == 0) {
    for (int s = 0; s < a.stages; ++s) {
      int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
      if (t < ntiles) issue(t, s);
    }
  }

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

  // every issued stage has been consumed: the ring is free for the merge
  sweep_epilogue<T, MODE, KPW>(a, acc, nacc, red, reinterpret_cast<double2*>(smem_raw));
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
  sweep_epilogue<T, MODE, KPW>(a, acc, nacc, red, wsum);
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
// CG (Sec. 2.1) for the mean cache: K^ z = y on the cell-sorted vectors.  The
// vectors and all reductions are FP64 whatever the coordinate type T (the
// interpolation weights stay in T, as in the Lanczos MVMs): an FP32 CG stalls
// on this ill-conditioned system (cond(K^) ~ 1e7 on the n = 1e6 workload).
// p = r + beta p (the new direction, written back); Ap = W^T u + s^2 p; pAp = p . Ap
// (u = K_UU W p was scattered from r + beta p on the fly)
template <typename T, int D>
__global__ void k_cg_gather_dot(GridDev g, const T* __restrict__ xs, int64_t n, int64_t n_pad,
                                const double* __restrict__ u, double noise, const double* __restrict__ r,
                                double* __restrict__ pv, double* __restrict__ Ap, double2* partial, LanczosState* st) {
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double be = st->cg_beta;
  DotAccD a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    const double pn = r[p] + be * pv[p];
    pv[p] = pn;
    double q = 0.0;
    if (p < n) {
      Stencil<T, D> stc;
      stc.compute(xs + p * D, g);
      q = stc.apply(u, g) + noise * pn;
    }
    Ap[p] = q;
    a.add_prod(pn, q);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->pap, st->counter2);
  if (last && threadIdx.x == 0) st->cg_alpha = st->rr / st->pap;
}
// x += a p ; r -= a Ap ; rr' = r.r
__global__ void k_cg_update(int64_t n_pad, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ pv, const double* __restrict__ Ap, double2* partial,
                            LanczosState* st, int max_iter, DevStatus* status) {
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double al = st->cg_alpha;
  DotAccD a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    x[p] += al * pv[p];
    double rv = r[p] - al * Ap[p];
    r[p] = rv;
    a.add_prod(rv, rv);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    double rrn = st->norm2;
    st->cg_beta = rrn / st->rr;
    st->rr = rrn;
    st->cg_iters += 1;
    if (!isfinite(rrn)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (rrn <= st->tol2 || st->cg_iters >= max_iter) {
      st->cg_done = 1;
    }
  }
}
template <typename T>
__global__ void k_cg_init(int64_t n_pad, const T* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
                          double* __restrict__ pv, double2* partial, LanczosState* st, double tol) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)b[p];
    x[p] = 0.0;
    r[p] = v;
    pv[p] = 0.0;  // first direction r + 0 p = r
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr = st->norm2;
    st->rr0 = st->norm2;
    st->tol2 = tol * tol * st->norm2;
    st->cg_iters = 0;
    st->cg_beta = 0.0;
    st->cg_done = st->norm2 == 0.0 ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// The same CG for the FP32 path in double-float: x, r, p, Ap are (hi, lo) float
// pairs (~48-bit), every operation runs on the FP32 pipes (GB300's FP64 rate
// is a small fraction of FP32), and K_UU still goes through the FP64 FFT on
// the m-sized grid vectors.
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ void acc_add_dfprod(DotAccF& acc, df a, df b) {
  acc.add_prod(a.hi, b.hi);
  acc.c += fmaf(a.hi, b.lo, a.lo * b.hi);
}

// u[node] = sum over sorted points of w_p(node) (r_p + beta p_p), FP64 result
template <int D>
__global__ void k_scatter_df(GridDev g, const float* __restrict__ xs, const int* __restrict__ cell_start,
                             const df* __restrict__ r, const df* __restrict__ pv, const LanczosState* st,
                             double* __restrict__ u) {
  if (st->cg_done) return;
  const df be = df_from_double(st->cg_beta);
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t node = wg; node < g.m; node += nw) {
    int nd[D];
    node_index<D>(node, g, nd);
    NodeRanges<D> rg;
    rg.build(g, nd, cell_start, lane);
    DotAccF acc;
    acc.zero();
    for (int f = lane; f < rg.total; f += 32) {
      int p = rg.point(f);
      df val = df_add(r[p], df_mul(be, pv[p]));
      float w = node_weight<float, D>(xs + (int64_t)p * D, g, nd);
      acc.add_prod(w, val.hi);
      acc.c += w * val.lo;
    }
    warp_merge(acc);
    if (lane == 0) u[node] = acc.value();
  }
}
__global__ void k_double_to_df(int64_t m, const double* __restrict__ a, df* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = df_from_double(a[i]);
}
// p = r + beta p (written back); Ap = W^T u + s^2 p; pAp = p . Ap
template <int D>
__global__ void k_cgdf_gather_dot(GridDev g, const float* __restrict__ xs, int64_t n, int64_t n_pad,
                                  const df* __restrict__ u, double noise, const df* __restrict__ r,
                                  df* __restrict__ pv, df* __restrict__ Ap, double2* partial, LanczosState* st) {
  __shared__ DotAccF red[32];
  if (st->cg_done) return;
  const df be = df_from_double(st->cg_beta);
  const df nz = df_from_double(noise);
  DotAccF a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    const df pn = df_add(r[p], df_mul(be, pv[p]));
    pv[p] = pn;
    df q = {0.f, 0.f};
    if (p < n) {
      Stencil<float, D> stc;
      stc.compute(xs + p * D, g);
      // sum over the 4^D stencil nodes of w * u (df)
      if (D == 1) {
#pragma unroll
        for (int r0 = 0; r0 < 4; ++r0) q = df_add(q, df_mul_f(u[stc.base[0] - 1 + r0], stc.w[0][r0]));
      } else if (D == 2) {
#pragma unroll
        for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
          for (int r1 = 0; r1 < 4; ++r1) {
            int64_t node = (int64_t)(stc.base[0] - 1 + r0) * g.stride[0] + (stc.base[1] - 1 + r1);
            q = df_add(q, df_mul_f(u[node], stc.w[0][r0] * stc.w[1][r1]));
          }
      } else {
#pragma unroll
        for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
          for (int r1 = 0; r1 < 4; ++r1)
#pragma unroll
            for (int r2 = 0; r2 < 4; ++r2) {
              int64_t node = (int64_t)(stc.base[0] - 1 + r0) * g.stride[0] +
                             (int64_t)(stc.base[1] - 1 + r1) * g.stride[1] + (stc.base[2] - 1 + r2);
              q = df_add(q, df_mul_f(u[node], stc.w[0][r0] * stc.w[1][r1] * stc.w[2][r2]));
            }
      }
      q = df_add(q, df_mul(nz, pn));
    }
    Ap[p] = q;
    acc_add_dfprod(a, pn, q);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccF>(partial, 1, 1, &st->pap, st->counter2);
  if (last && threadIdx.x == 0) st->cg_alpha = st->rr / st->pap;
}
// x += a p ; r -= a Ap ; rr' = r.r
__global__ void k_cgdf_update(int64_t n_pad, df* __restrict__ x, df* __restrict__ r, const df* __restrict__ pv,
                              const df* __restrict__ Ap, double2* partial, LanczosState* st, int max_iter,
                              DevStatus* status) {
  __shared__ DotAccF red[32];
  if (st->cg_done) return;
  const df al = df_from_double(st->cg_alpha);
  const df mal = df_neg(al);
  DotAccF a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    x[p] = df_add(x[p], df_mul(al, pv[p]));
    df rv = df_add(r[p], df_mul(mal, Ap[p]));
    r[p] = rv;
    acc_add_dfprod(a, rv, rv);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccF>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    double rrn = st->norm2;
    st->cg_beta = rrn / st->rr;
    st->rr = rrn;
    st->cg_iters += 1;
    if (!isfinite(rrn)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (rrn <= st->tol2 || st->cg_iters >= max_iter) {
      st->cg_done = 1;
    }
  }
}
__global__ void k_cgdf_init(int64_t n_pad, const float* __restrict__ b, df* __restrict__ x, df* __restrict__ r,
                            df* __restrict__ pv, double2* partial, LanczosState* st, double tol) {
  __shared__ DotAccF red[32];
  DotAccF a;
  a.zero();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    float v = b[p];
    x[p] = {0.f, 0.f};
    r[p] = {v, 0.f};
    pv[p] = {0.f, 0.f};
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccF>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr = st->norm2;
    st->rr0 = st->norm2;
    st->tol2 = tol * tol * st->norm2;
    st->cg_iters = 0;
    st->cg_beta = 0.0;
    st->cg_done = st->norm2 == 0.0 ? 1 : 0;
  }
}
__global__ void k_df_to_double(int64_t n, const df* __restrict__ a, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = df_to_double(a[i]);
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
__global__ void k_fill(T* p, int64_t n, T v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
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

// ---------------------------------------------------------------------------

struct DevBuf {
  const Allocator* al;
  cudaStream_t s;
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf(const Allocator& a, cudaStream_t st) : al(&a), s(st) {}
  bool get(size_t b) {
    bytes = b;
    p = al->alloc(b, s);
    return p != nullptr || b == 0;
  }
  ~DevBuf() {
    if (p) al->free(p, bytes, s);
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
constexpr int TILE_CTAS_PER_SM = 2;

template <typename T>
love_status make_qmap(T* Q, int64_t ldq, int kcols, int bc, CUtensorMap* out);

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
    LOVE_COUNT_LAUNCH(); kern<<<grid, TILE_T, smem, s>>>(a);                                   \
    return cuda_check(cudaGetLastError());                                                     \
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

// Q as a 2-D tensor for TMA: rows (inner, n_pad) x columns (kcols), box
// {TILE_R rows, bc columns}; columns past kcols read as zeros
inline int box_cols(size_t elem) { return elem == 4 ? 8 : 4; }
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

// FP32 ski: double-float CG; the solution is returned as FP64 in x
love_status cg_solve_df(love_ski* ski, const float* b, double* x, double tol, int max_iter, int* iters,
                        cudaStream_t s) {
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int64_t np = ski->n_pad;
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), xb(ski->alloc, s), r(ski->alloc, s), pv(ski->alloc, s),
      Ap(ski->alloc, s), u(ski->alloc, s), udf(ski->alloc, s), fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * 1024) || !xb.get(sizeof(df) * np) ||
      !r.get(sizeof(df) * np) || !pv.get(sizeof(df) * np) || !Ap.get(sizeof(df) * np) ||
      !u.get(sizeof(double) * gh.m * 2) || !udf.get(sizeof(df) * gh.m) || !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  double* u1 = u.as<double>();
  double* u2 = u1 + gh.m;
  const int blocks = std::min(1024, ceil_div(np, 256));
  const int sblocks = (int)std::min<int64_t>((g.m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, 1, 0.0);
  LOVE_COUNT_LAUNCH(); k_cgdf_init<<<blocks, 256, 0, s>>>(np, b, xb.as<df>(), r.as<df>(), pv.as<df>(), part.as<double2>(), st, tol);
  LOVE_LAUNCH_CHECK();
  int it = 0;
  const int chunk = 32;
  while (it < max_iter) {
    for (int c = 0; c < chunk && it < max_iter; ++c, ++it) {
      switch (g.dim) {
        case 1: LOVE_COUNT_LAUNCH(); k_scatter_df<1><<<sblocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->cell_start, r.as<df>(), pv.as<df>(), st, u1); break;
        case 2: LOVE_COUNT_LAUNCH(); k_scatter_df<2><<<sblocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->cell_start, r.as<df>(), pv.as<df>(), st, u1); break;
        default: LOVE_COUNT_LAUNCH(); k_scatter_df<3><<<sblocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->cell_start, r.as<df>(), pv.as<df>(), st, u1);
      }
      LOVE_TRY(kuu_apply<double>(gh, ski->fft, u1, u2, 1, gh.m, fw.p, -1, s));
      LOVE_COUNT_LAUNCH(); k_double_to_df<<<ceil_div(gh.m, 256), 256, 0, s>>>(gh.m, u2, udf.as<df>());
      switch (g.dim) {
        case 1: LOVE_COUNT_LAUNCH(); k_cgdf_gather_dot<1><<<blocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->n, np, udf.as<df>(), gh.noise, r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st); break;
        case 2: LOVE_COUNT_LAUNCH(); k_cgdf_gather_dot<2><<<blocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->n, np, udf.as<df>(), gh.noise, r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st); break;
        default: LOVE_COUNT_LAUNCH(); k_cgdf_gather_dot<3><<<blocks, 256, 0, s>>>(g, (const float*)ski->xs, ski->n, np, udf.as<df>(), gh.noise, r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st);
      }
      LOVE_COUNT_LAUNCH(); k_cgdf_update<<<blocks, 256, 0, s>>>(np, xb.as<df>(), r.as<df>(), pv.as<df>(), Ap.as<df>(), part.as<double2>(), st, max_iter, ski->status);
      LOVE_LAUNCH_CHECK();
    }
    int done = 0;
    LOVE_CUDA(cudaMemcpyAsync(&done, &st->cg_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (done) break;
  }
  LOVE_COUNT_LAUNCH(); k_df_to_double<<<ceil_div(np, 256), 256, 0, s>>>(np, xb.as<df>(), x);
  LOVE_LAUNCH_CHECK();
  int n_it = 0;
  LOVE_CUDA(cudaMemcpyAsync(&n_it, &st->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = n_it;
  return LOVE_OK;
}

template <typename T>
love_status cg_solve(love_ski* ski, const T* b, double* x, double tol, int max_iter, int* iters, cudaStream_t s) {
  // the double-float form scatters over the product grid only; an additive
  // grid takes the FP64-vector form below
  if (sizeof(T) == 4 && !ski->grid.additive) return cg_solve_df(ski, (const float*)b, x, tol, max_iter, iters, s);
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int64_t np = ski->n_pad;
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), r(ski->alloc, s), pv(ski->alloc, s), Ap(ski->alloc, s),
      u(ski->alloc, s), fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * 1024) || !r.get(sizeof(double) * np) ||
      !pv.get(sizeof(double) * np) || !Ap.get(sizeof(double) * np) || !u.get(sizeof(double) * gh.m * 2) ||
      !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  double* u1 = u.as<double>();
  double* u2 = u1 + gh.m;
  int blocks = std::min(1024, ceil_div(np, 256));
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, 1, 0.0);
  LOVE_COUNT_LAUNCH(); k_cg_init<T><<<blocks, 256, 0, s>>>(np, b, x, r.as<double>(), pv.as<double>(), part.as<double2>(), st, tol);
  LOVE_LAUNCH_CHECK();
  int it = 0;
  const int chunk = 32;
  while (it < max_iter) {
    for (int c = 0; c < chunk && it < max_iter; ++c, ++it) {
      LOVE_TRY(scatter_any<T, double>(ski, r.as<double>(), nullptr, 1.0, u1, s, pv.as<double>(), &st->cg_beta,
                                      &st->cg_done));
      LOVE_TRY(kuu_apply<double>(gh, ski->fft, u1, u2, 1, gh.m, fw.p, -1, s));
      switch (g.dim) {
        case 1: LOVE_COUNT_LAUNCH(); k_cg_gather_dot<T, 1><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, np, u2, gh.noise, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st); break;
        case 2: LOVE_COUNT_LAUNCH(); k_cg_gather_dot<T, 2><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, np, u2, gh.noise, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st); break;
        default: LOVE_COUNT_LAUNCH(); k_cg_gather_dot<T, 3><<<blocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->n, np, u2, gh.noise, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st);
      }
      LOVE_COUNT_LAUNCH(); k_cg_update<<<blocks, 256, 0, s>>>(np, x, r.as<double>(), pv.as<double>(), Ap.as<double>(), part.as<double2>(), st, max_iter,
                                           ski->status);
      LOVE_LAUNCH_CHECK();
    }
    int done = 0;
    LOVE_CUDA(cudaMemcpyAsync(&done, &st->cg_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (done) break;
  }
  int n_it = 0;
  LOVE_CUDA(cudaMemcpyAsync(&n_it, &st->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = n_it;
  return LOVE_OK;
}

// ---------------------------------------------------------------------------
// Mean cache on the grid (d <= 2).  W is m x n here (u = W v scatters points
// to nodes) and G = W W^T is the m x m Gram matrix of the interpolation
// weights, banded with 7^d diagonals.  The push-through identity
//   W (W^T K W + s^2 I)^-1 = (G K + s^2 I)^-1 W
// turns the mean weights a = K_UU W K^^-1 y (Sec. 3, predictive mean) into
//   a = K z,   A z = W y,   A = G K + s^2 I,
// an m-sized system.  A is self-adjoint and positive definite in the inner
// product <u, v>_K = u^T K v (K A = K G K + s^2 K), with eigenvalues >= s^2,
// so CG runs in that inner product: s = K r and q = K p are carried by
// recurrence, leaving one K product (FFT) per iteration and no n-sized work.
// Stopping rule: CG minimises E = <e, A e>_K over the Krylov space (e the
// error of z), and |W^T (a_i - a)|^2 = e^T K G K e <= E <= <r, r>_K / s^2, so
//   rho = r^T K r <= tol^2 s^2 |y|^2
// bounds the error of the fitted values at the training points by tol |y|,
// the same guarantee the rule |y - K^ x| <= tol |y| gives CG on K^ x = y
// (there W^T (a_i - a) = (K^ - s^2 I) K^^-1 r, a contraction of r).
namespace {

template <int D> struct Band { static constexpr int B = D == 1 ? 7 : 49; };

// G[o][node] = sum_p w_p(node) w_p(node + off(o)), offsets -3..3 per dimension;
// warp per node over the cell-sorted points, FP64 accumulation
template <typename T, int D>
__global__ void k_gram_band(GridDev g, const T* __restrict__ xs, const int* __restrict__ cell_start,
                            double* __restrict__ G) {
  constexpr int B = Band<D>::B;
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t node = wg; node < g.m; node += nw) {
    int nd[D];
    node_index<D>(node, g, nd);
    NodeRanges<D> rg;
    rg.build(g, nd, cell_start, lane);
    double acc[B];
#pragma unroll
    for (int o = 0; o < B; ++o) acc[o] = 0.0;
    for (int f = lane; f < rg.total; f += 32) {
      const int p = rg.point(f);
      T wd[D][7];
#pragma unroll
      for (int e = 0; e < D; ++e) {
        T sc = grid_coord(xs[(int64_t)p * D + e], g, e);
        int i = (int)floor(sc);
        if (i > g.g[e] - 3) i = g.g[e] - 3;
        T fr = sc - T(i);
#pragma unroll
        for (int o = 0; o < 7; ++o) wd[e][o] = keys_u(fr + T(1) - T(nd[e] + o - 3 - (i - 1)));
      }
      if constexpr (D == 1) {
#pragma unroll
        for (int o = 0; o < 7; ++o) acc[o] = fma((double)wd[0][3], (double)wd[0][o], acc[o]);
      } else {
        const T wu = wd[0][3] * wd[D - 1][3];
#pragma unroll
        for (int o0 = 0; o0 < 7; ++o0)
#pragma unroll
          for (int o1 = 0; o1 < 7; ++o1)
            acc[o0 * 7 + o1] = fma((double)wu, (double)(wd[0][o0] * wd[D - 1][o1]), acc[o0 * 7 + o1]);
      }
    }
#pragma unroll
    for (int o = 0; o < B; ++o) {
      double v = acc[o];
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
      if (lane == 0) G[(int64_t)o * g.m + node] = v;
    }
  }
}

// The new direction p = r + beta p', q = s + beta q' (q = K p) is formed on
// the fly (at the node and at its band neighbours, the same fma everywhere)
// and written to the other buffer of a pair; then t = G q + s^2 p (= A p) and
// pi = q . t (= <p, A p>_K).
template <int D>
__global__ void k_mcg_band(GridDev g, const double* __restrict__ G, const double* __restrict__ r,
                           const double* __restrict__ sv, const double* __restrict__ p_old,
                           const double* __restrict__ q_old, double* __restrict__ p_new, double* __restrict__ q_new,
                           double noise, double* __restrict__ t, double2* partial, LanczosState* st, int max_iter,
                           DevStatus* status) {
  constexpr int B = Band<D>::B;
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double be = st->cg_beta;
  DotAccD api;
  api.zero();
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.m;
       node += (int64_t)gridDim.x * blockDim.x) {
    int nd[D];
    node_index<D>(node, g, nd);
    double gq = 0.0;
#pragma unroll
    for (int o = 0; o < B; ++o) {
      const int o0 = D == 1 ? o : o / 7, o1 = o % 7;
      const int a0 = nd[0] + o0 - 3;
      const int a1 = D == 1 ? 0 : nd[D - 1] + o1 - 3;
      bool in = a0 >= 0 && a0 < g.g[0];
      if (D == 2) in = in && a1 >= 0 && a1 < g.g[1];
      if (in) {
        const int64_t nb = D == 1 ? a0 : (int64_t)a0 * g.stride[0] + a1;
        gq = fma(G[(int64_t)o * g.m + node], fma(be, q_old[nb], sv[nb]), gq);
      }
    }
    const double pn = fma(be, p_old[node], r[node]);
    const double qn = fma(be, q_old[node], sv[node]);
    p_new[node] = pn;
    q_new[node] = qn;
    const double tv = gq + noise * pn;
    t[node] = tv;
    api.add_prod(qn, tv);
  }
  block_merge(api, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, api);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->pap, st->counter2);
  if (last && threadIdx.x == 0) {
    const double pi = st->pap;
    if (!isfinite(pi)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (pi <= 0.0 || st->cg_iters >= max_iter) {
      st->cg_done = 1;
    } else {
      st->cg_alpha = st->rr / pi;
    }
  }
}

// w += a q;  r -= a t;  s -= a K t;  rho' = r . s
__global__ void k_mcg_update(int64_t m, double* __restrict__ w, double* __restrict__ r, double* __restrict__ sv,
                             const double* __restrict__ q, const double* __restrict__ t,
                             const double* __restrict__ Kt, double2* partial, LanczosState* st, DevStatus* status) {
  __shared__ DotAccD red[32];
  if (st->cg_done) return;
  const double al = st->cg_alpha;
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    w[i] = fma(al, q[i], w[i]);
    const double rv = fma(-al, t[i], r[i]);
    const double sn = fma(-al, Kt[i], sv[i]);
    r[i] = rv;
    sv[i] = sn;
    a.add_prod(rv, sn);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    const double rho = st->norm2;
    st->cg_beta = rho / st->rr;
    st->rr = rho;
    st->cg_iters += 1;
    if (!isfinite(rho)) {
      dev_flag(status, LOVE_ERR_NAN);
      st->cg_done = 1;
    } else if (rho <= st->tol2) {
      st->cg_done = 1;
    }
  }
}

// |y|^2 -> the stopping threshold tol^2 s^2 |y|^2
template <typename T>
__global__ void k_mcg_ynorm(int64_t n, const T* __restrict__ y, double* __restrict__ yd, double tol, double noise,
                            double2* partial, LanczosState* st) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)y[i];
    if (yd) yd[i] = v;
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr0 = st->norm2;
    st->tol2 = tol * tol * st->norm2 * noise;
    st->cg_iters = 0;
    st->cg_beta = 0.0;
    st->cg_done = st->norm2 == 0.0 ? 1 : 0;
  }
}

// r = b, s = K b, w = 0, p' = q' = 0 (so the first direction is p = r, q = s);
// rho = r . s
__global__ void k_mcg_start(int64_t m, const double* __restrict__ b, const double* __restrict__ Kb,
                            double* __restrict__ r, double* __restrict__ pv, double* __restrict__ sv,
                            double* __restrict__ q, double* __restrict__ w, double2* partial, LanczosState* st) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = b[i];
    pv[i] = 0.0;
    sv[i] = Kb[i];
    q[i] = 0.0;
    w[i] = 0.0;
    a.add_prod(b[i], Kb[i]);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter2);
  if (last && threadIdx.x == 0) {
    st->rr = st->norm2;
    if (!(st->norm2 > st->tol2)) st->cg_done = 1;
  }
}

// ---- preconditioned grid-space solve (1-D grids) ------------------------------
// M = B K + s^2 I, B the symmetric Toeplitz stencil of G = W W^T averaged over
// the interior nodes (7 diagonals).  B and K are both Toeplitz, so on the
// circulant embedding of length N, P = M^{-1} is approximated by the spectral
// multiplier 1 / (lambda_B lambda_K + s^2) applied to the zero-padded vector
// and cropped back to the grid.  P does not commute with K exactly (the crop),
// so it is used as a right preconditioner of GMRES rather than inside CG.

// bhat[d] = average over interior nodes of (G[node, node+d] + G[node, node-d]) / 2;
// bhat[4] = fraction of interior nodes whose G_ii is below a fifth of the
// average (empty stretches of the grid, where the stencil does not fit)
__global__ void k_pcg_stencil(const double* __restrict__ G, int64_t m, double* __restrict__ bhat) {
  __shared__ double red[4][256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t lo = 6, hi = m - 6;   // nodes whose 7-wide band sees the whole data range
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    acc[0] += G[3 * m + i];
#pragma unroll
    for (int d = 1; d < 4; ++d) acc[d] += 0.5 * (G[(int64_t)(3 + d) * m + i] + G[(int64_t)(3 - d) * m + i]);
  }
#pragma unroll
  for (int d = 0; d < 4; ++d) red[d][threadIdx.x] = acc[d];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int d = 0; d < 4; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + w];
    __syncthreads();
  }
  const double b0 = hi > lo ? red[0][0] / (double)(hi - lo) : 0.0;
  if (threadIdx.x < 4) bhat[threadIdx.x] = hi > lo ? red[threadIdx.x][0] / (double)(hi - lo) : 0.0;
  __syncthreads();
  double cnt = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) cnt += G[3 * m + i] < 0.2 * b0 ? 1.0 : 0.0;
  red[0][threadIdx.x] = cnt;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[0][threadIdx.x] += red[0][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) bhat[4] = hi > lo ? red[0][0] / (double)(hi - lo) : 1.0;
}

// symbol of P on the embedding (stored / N like the K_UU spectrum) and the
// largest eigenvalue of K's circulant embedding (>= the largest of K)
__global__ void k_pcg_symbol(const double* __restrict__ lamK, int64_t N, const double* __restrict__ bhat, double noise,
                             double* __restrict__ sym, unsigned long long* __restrict__ lk_bits) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double lb = bhat[0];
#pragma unroll
  for (int d = 1; d < 4; ++d) lb += 2.0 * bhat[d] * cospi(2.0 * (double)(d * j % N) / (double)N);
  const double lk = fmax((double)N * lamK[j], 0.0);
  sym[j] = 1.0 / ((fmax(lb, 0.0) * lk + noise) * (double)N);
  atomicMax(lk_bits, (unsigned long long)__double_as_longlong(lk));   // lk >= 0: bit order = value order
}

}  // namespace

bool mean_grid_cg_supported(const love_ski* ski) { return ski->grid.dim <= 2 && !ski->grid.additive; }

template <typename T>
love_status mean_grid_gmres(love_ski* ski, double tol, int max_iter, double* a, int* iters, bool* converged,
                            cudaStream_t s);

template <typename T>
love_status mean_grid_cg(love_ski* ski, double tol, int max_iter, double* a, int* iters, cudaStream_t s,
                         bool precond) {
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int dim = gh.dim;
  if (dim > 2) return LOVE_ERR_UNSUPPORTED;
  int pre_iters = 0;
  if (precond && dim == 1 && gh.g[0] >= 16) {
    // the averaged stencil fits G where the training points are spread over
    // the grid; where they are not (clusters, gaps) the GMRES setup declines
    // (more than 10 % of the interior nearly empty) or, should it stall, the
    // plain CG below takes over from zero after GM_CYCLES restarts
    bool conv = false;
    LOVE_TRY(mean_grid_gmres<T>(ski, tol, std::min(max_iter, GM_CYCLES * GM_R), a, &pre_iters, &conv, s));
    if (conv || pre_iters >= max_iter) {
      if (iters) *iters = pre_iters;
      return LOVE_OK;
    }
    max_iter -= pre_iters;
  }
  const int64_t m = gh.m, n = ski->n;
  const int B = dim == 1 ? 7 : 49;
  DevBuf stb(ski->alloc, s), part(ski->alloc, s), Gb(ski->alloc, s), vec(ski->alloc, s), yb(ski->alloc, s),
      fw(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  const bool conv = sizeof(T) != sizeof(double);
  if (!stb.get(sizeof(LanczosState)) || !part.get(sizeof(double2) * 2048) || !Gb.get(sizeof(double) * B * m) ||
      !vec.get(sizeof(double) * 9 * m) || (conv && !yb.get(sizeof(double) * std::max<int64_t>(n, 1))) ||
      !fw.get(std::max<size_t>(fwb, 16)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();
  double* v = vec.as<double>();
  double *b = v, *r = v + m, *sv = v + 2 * m, *t = v + 3 * m, *Kt = v + 4 * m;
  double* pbuf[2] = {v + 5 * m, v + 6 * m};  // directions p, q: double-buffered
  double* qbuf[2] = {v + 7 * m, v + 8 * m};
  double* w = a;  // a = K z accumulates in place
  double2* pp = part.as<double2>();
  const int sblocks = (int)std::min<int64_t>((m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  const int mblocks = (int)std::min<int64_t>(ceil_div(m, 256), 1024);
  const int nblocks = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), 1024);
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, 1, 0.0);
  // G = W W^T
  if (dim == 1) {
    LOVE_COUNT_LAUNCH(); k_gram_band<T, 1><<<sblocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Gb.as<double>());
  } else {
    LOVE_COUNT_LAUNCH(); k_gram_band<T, 2><<<sblocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Gb.as<double>());
  }
  // b = W y (FP64), |y|^2
  const double* yd = conv ? yb.as<double>() : (const double*)ski->ys;
  LOVE_COUNT_LAUNCH();
  k_mcg_ynorm<T><<<nblocks, 256, 0, s>>>(n, (const T*)ski->ys, conv ? yb.as<double>() : nullptr, tol, gh.noise, pp, st);
  LOVE_LAUNCH_CHECK();
  // K products in FP64 transforms: with FP32 transforms (error ~log2(N) 2^-24)
  // the K-inner product loses positivity on the high-frequency components and
  // the iteration stops early (mean errors ~6e-3 std(y) on the n = 1e6 workload)
  auto kmul = [&](const double* in, double* out) -> love_status {
    return kuu_apply<double>(gh, ski->fft, in, out, 1, m, fw.p, -1, s);
  };
  LOVE_TRY(scatter_any<T, double>(ski, yd, nullptr, 1.0, b, s));
  LOVE_TRY(kmul(b, Kt));
  LOVE_COUNT_LAUNCH(); k_mcg_start<<<mblocks, 256, 0, s>>>(m, b, Kt, r, pbuf[0], sv, qbuf[0], w, pp, st);
  LOVE_LAUNCH_CHECK();
  int it = 0;
  const int chunk = 64;
  while (it <= max_iter) {
    for (int c = 0; c < chunk && it <= max_iter; ++c, ++it) {
      const double *po = pbuf[it & 1], *qo = qbuf[it & 1];
      double *pn = pbuf[(it + 1) & 1], *qn = qbuf[(it + 1) & 1];
      if (dim == 1) {
        LOVE_COUNT_LAUNCH(); k_mcg_band<1><<<mblocks, 256, 0, s>>>(g, Gb.as<double>(), r, sv, po, qo, pn, qn, gh.noise, t, pp, st, max_iter, ski->status);
      } else {
        LOVE_COUNT_LAUNCH(); k_mcg_band<2><<<mblocks, 256, 0, s>>>(g, Gb.as<double>(), r, sv, po, qo, pn, qn, gh.noise, t, pp, st, max_iter, ski->status);
      }
      LOVE_TRY(kmul(t, Kt));
      LOVE_COUNT_LAUNCH(); k_mcg_update<<<mblocks, 256, 0, s>>>(m, w, r, sv, qn, t, Kt, pp, st, ski->status);
      LOVE_LAUNCH_CHECK();
    }
    int done = 0;
    LOVE_CUDA(cudaMemcpyAsync(&done, &st->cg_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (done) break;
  }
  int n_it = 0;
  LOVE_CUDA(cudaMemcpyAsync(&n_it, &st->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  LOVE_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = pre_iters + n_it;
  return LOVE_OK;
}
template love_status mean_grid_cg<float>(love_ski*, double, int, double*, int*, cudaStream_t, bool);
template love_status mean_grid_cg<double>(love_ski*, double, int, double*, int*, cudaStream_t, bool);

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
template love_status cg_solve<float>(love_ski*, const float*, double*, double, int, int*, cudaStream_t);
template love_status cg_solve<double>(love_ski*, const double*, double*, double, int, int*, cudaStream_t);
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

// ---------------------------------------------------------------------------
// Sampler Lanczos (Sec. 3.3, eq. lancapprox): k' steps on M = K_UU - Rt Rt^T,
// an m x m operator, in FP64 with the same CGS2 reorthogonalisation kernels.
// M's entries are differences of nearly equal numbers (K_UU ~ 1, posterior
// ~ 1e-7 on the 1-D n = 1e6 workload), so FP32 would lose them entirely.
// The probe (not given by the paper) is the Rademacher vector
// r_i = +1 if the low bit of SplitMix64 output i (seeded with `seed`) is 1, else -1.
namespace {

__device__ __forceinline__ uint64_t splitmix64_output(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename QT>
__global__ void k_rademacher(int64_t m, int64_t m_pad, uint64_t seed, QT* __restrict__ q0, LanczosState* st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m_pad) q0[i] = i < m ? ((splitmix64_output(seed, (uint64_t)i) & 1ull) ? QT(1) : QT(-1)) : QT(0);
  if (i == 0) st->scal[0] = 1.0 / sqrt((double)m);
}
template <typename QT>
__global__ void k_normalize_col(QT* __restrict__ q, int64_t n_pad, const double* __restrict__ scal,
                                const LanczosState* st) {
  if (st->done) return;
  const QT sc = (QT)*scal;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x)
    q[i] *= sc;
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
    LOVE_TRY(tile_run<double, MODE_DOT>(ta, s));
    LOVE_TRY(tile_run<double, MODE_UPDATE_DOT>(ta, s));
    LOVE_TRY(tile_run<double, MODE_UPDATE_NORM>(ta, s));
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

// ---------------------------------------------------------------------------
// Right-preconditioned GMRES for the grid-space mean system (1-D grids):
// A z = W y with A = G K_UU + s^2 I (G = W W^T banded), a = K_UU z; solved as
// A P u = W y, z = P u, with P the spectral approximation of (B K_UU + s^2 I)^{-1}.
// The Arnoldi basis V (m_pad x (R + 1), FP64) is orthogonalised by the same
// CGS2 tile kernels as the Lanczos runs; the Hessenberg columns go through
// Givens rotations on the device, so |g_{j+1}| is the Euclidean residual of
// the current iterate.  The solve stops when |g_{j+1}|^2 <= tol^2 s^2 |y|^2 /
// (2 lambda_max(K)), which implies the CG stopping rule r^T K r <= tol^2 s^2 |y|^2
// for the recursively updated residual (as the plain CG applies it); a cycle
// that ends without meeting it restarts from the recomputed residual b - A z.
namespace {

struct GmresState {
  double H[(GM_R + 1) * GM_R];   // rotated Hessenberg columns (upper triangle), ld GM_R + 1
  double cs[GM_R], sn[GM_R];
  double g[GM_R + 1];
  double y[GM_R];
  int ncols;
  int converged;
  double target2;
  unsigned long long lk_bits;   // largest eigenvalue of K's circulant embedding
};

__global__ void k_gm_target(GmresState* gm, const LanczosState* cg) {
  const double lk = __longlong_as_double((long long)gm->lk_bits);
  gm->target2 = 0.5 * cg->tol2 / fmax(lk, 1e-300);
}

// V[:, 0] = r (zero past m); g = (|r|, 0, ...); scal_0 = 1 / |r|
__global__ void k_gm_start(int64_t m, int64_t m_pad, const double* __restrict__ r, double* __restrict__ v0,
                           double2* partial, LanczosState* st, GmresState* gm, DevStatus* status) {
  __shared__ DotAccD red[32];
  DotAccD a;
  a.zero();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = i < m ? r[i] : 0.0;
    v0[i] = v;
    a.add_prod(v, v);
  }
  block_merge(a, red);
  if (threadIdx.x == 0) acc_store(partial + blockIdx.x, a);
  bool last = last_cta_reduce<DotAccD>(partial, 1, 1, &st->norm2, st->counter);
  if (last && threadIdx.x == 0) {
    const double b2 = st->norm2, b = sqrt(b2);
    gm->g[0] = b;
    for (int i = 1; i <= GM_R; ++i) gm->g[i] = 0.0;
    gm->ncols = 0;
    st->scal[0] = b > 0.0 ? 1.0 / b : 0.0;
    if (!isfinite(b2)) dev_flag(status, LOVE_ERR_NAN);
    if (!(b2 > gm->target2)) {
      st->done = 1;
      st->k_eff = 0;
      gm->converged = 1;
    }
  }
}

// y = G (K P v) + s^2 (P v) over the padded rows (zero past m)
__global__ void k_gm_band(int64_t m, int64_t m_pad, const double* __restrict__ G, const double* __restrict__ kv,
                          const double* __restrict__ pv, double noise, double* __restrict__ y,
                          const LanczosState* st) {
  if (st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (i < m) {
#pragma unroll
      for (int o = 0; o < 7; ++o) {
        const int64_t nb = i + o - 3;
        if (nb >= 0 && nb < m) acc = fma(G[(int64_t)o * m + i], kv[nb], acc);
      }
      acc = fma(noise, pv[i], acc);
    }
    y[i] = acc;
  }
}

// Hessenberg column j: h_ij = c_i + c'_i (the two Gram-Schmidt passes), h_{j+1,j}
// = beta_j; earlier rotations, then the rotation that zeroes h_{j+1,j}
__global__ void k_gm_givens(LanczosState* st, GmresState* gm, int j, DevStatus* status) {
  if (j >= st->k_eff || gm->ncols != j) return;
  double h[GM_R + 1];
  for (int i = 0; i <= j; ++i) h[i] = st->coef[i] + st->coef2[i];
  h[j + 1] = st->beta[j];
  for (int i = 0; i < j; ++i) {
    const double t = gm->cs[i] * h[i] + gm->sn[i] * h[i + 1];
    h[i + 1] = -gm->sn[i] * h[i] + gm->cs[i] * h[i + 1];
    h[i] = t;
  }
  const double r = hypot(h[j], h[j + 1]);
  const double c = r > 0.0 ? h[j] / r : 1.0, sn = r > 0.0 ? h[j + 1] / r : 0.0;
  gm->cs[j] = c;
  gm->sn[j] = sn;
  h[j] = r;
  gm->g[j + 1] = -sn * gm->g[j];
  gm->g[j] = c * gm->g[j];
  for (int i = 0; i <= j; ++i) gm->H[(int64_t)j * (GM_R + 1) + i] = h[i];
  gm->ncols = j + 1;
  if (!isfinite(gm->g[j + 1])) {
    dev_flag(status, LOVE_ERR_NAN);
    gm->converged = 1;   // nothing more to gain; the status reports it
    st->done = 1;
    st->k_eff = j;
    gm->ncols = j;
  } else if (gm->g[j + 1] * gm->g[j + 1] <= gm->target2) {
    st->done = 1;
    st->k_eff = j + 1;
    gm->converged = 1;
  }
}

// R y = g by back substitution (ncols columns)
__global__ void k_gm_solve(GmresState* gm) {
  const int kc = gm->ncols;
  for (int i = kc - 1; i >= 0; --i) {
    double v = gm->g[i];
    for (int l = i + 1; l < kc; ++l) v -= gm->H[(int64_t)l * (GM_R + 1) + i] * gm->y[l];
    const double d = gm->H[(int64_t)i * (GM_R + 1) + i];
    gm->y[i] = d != 0.0 ? v / d : 0.0;
  }
}

// u = V y
__global__ void k_gm_combine(int64_t m, const double* __restrict__ V, int64_t ldv, const GmresState* gm,
                             double* __restrict__ u) {
  const int kc = gm->ncols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < kc; ++c) acc = fma(V[(int64_t)c * ldv + i], gm->y[c], acc);
    u[i] = acc;
  }
}

__global__ void k_gm_add(int64_t m, double* __restrict__ z, const double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += d[i];
}

// r = b - (G K z + s^2 z)
__global__ void k_gm_resid(int64_t m, const double* __restrict__ G, const double* __restrict__ kz,
                           const double* __restrict__ z, const double* __restrict__ b, double noise,
                           double* __restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
      const int64_t nb = i + o - 3;
      if (nb >= 0 && nb < m) acc = fma(G[(int64_t)o * m + i], kz[nb], acc);
    }
    r[i] = b[i] - fma(noise, z[i], acc);
  }
}

}  // namespace

template <typename T>
love_status mean_grid_gmres(love_ski* ski, double tol, int max_iter, double* a, int* iters, bool* converged,
                            cudaStream_t s) {
  const GridHost& gh = ski->grid;
  const GridDev g = gh.dev();
  const int64_t m = gh.m, n = ski->n;
  const int64_t m_pad = (m + TILE_R - 1) / TILE_R * TILE_R;
  const FftPlan& kp = ski->fft[0];
  const int bc = box_cols(sizeof(double));
  const int max_grid = std::max(TILE_CTAS_PER_SM * num_sms(), 1024);
  DevBuf stb(ski->alloc, s), cgb(ski->alloc, s), gmb(ski->alloc, s), part(ski->alloc, s), Gb(ski->alloc, s),
      vec(ski->alloc, s), Vb(ski->alloc, s), yb(ski->alloc, s), fw(ski->alloc, s), symb(ski->alloc, s);
  size_t fwb = fft_work_bytes(gh, ski->fft, 1, true);
  const bool conv = sizeof(T) != sizeof(double);
  if (!stb.get(sizeof(LanczosState)) || !cgb.get(sizeof(LanczosState)) || !gmb.get(sizeof(GmresState)) ||
      !part.get(sizeof(double2) * (size_t)max_grid * (GM_R + 2)) || !Gb.get(sizeof(double) * 7 * m) ||
      !vec.get(sizeof(double) * (6 * m + m_pad)) || !Vb.get(sizeof(double) * m_pad * (GM_R + 1)) ||
      (conv && !yb.get(sizeof(double) * std::max<int64_t>(n, 1))) || !fw.get(std::max<size_t>(fwb, 16)) ||
      !symb.get(sizeof(double) * (kp.N + 8)))
    return LOVE_ERR_OOM;
  LanczosState* st = stb.as<LanczosState>();   // Arnoldi state (tile kernels)
  LanczosState* cg = cgb.as<LanczosState>();   // |y|^2 and the stopping threshold
  GmresState* gm = gmb.as<GmresState>();
  double* v = vec.as<double>();
  double *b = v, *r = v + m, *z = v + 2 * m, *pv = v + 3 * m, *kv = v + 4 * m, *u = v + 5 * m, *yv = v + 6 * m;
  double* V = Vb.as<double>();
  double* sym = symb.as<double>();
  double* bhat = sym + kp.N;
  double2* pp = part.as<double2>();
  const int sblocks = (int)std::min<int64_t>((m * 32 + 255) / 256, (int64_t)num_sms() * 16);
  const int mblocks = (int)std::min<int64_t>(ceil_div(m_pad, 256), 1024);
  const int nblocks = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), 1024);
  FftPlan pplan = kp;   // the same transform with the spectrum of P (never the dense form)
  pplan.lam_d = sym;
  pplan.col2 = pplan.coldl2 = nullptr;
  auto kmul = [&](const double* in, double* out) -> love_status {
    return kuu_apply<double>(gh, ski->fft, in, out, 1, m, fw.p, -1, s);
  };
  auto pmul = [&](const double* in, double* out) -> love_status {
    return kuu_apply<double>(gh, &pplan, in, out, 1, m, fw.p, -1, s);
  };
  LOVE_CUDA(cudaMemsetAsync(gm, 0, sizeof(GmresState), s));
  LOVE_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * m, s));
  LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(cg, 1, 0.0);
  LOVE_COUNT_LAUNCH(); k_gram_band<T, 1><<<sblocks, 256, 0, s>>>(g, (const T*)ski->xs, ski->cell_start, Gb.as<double>());
  LOVE_COUNT_LAUNCH(); k_pcg_stencil<<<1, 256, 0, s>>>(Gb.as<double>(), m, bhat);
  LOVE_LAUNCH_CHECK();
  {
    // more than 10 % of the interior nearly empty: leave the solve to the CG
    double empty = 1.0;
    LOVE_CUDA(cudaMemcpyAsync(&empty, bhat + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (!(empty <= 0.1)) {
      *iters = 0;
      return LOVE_OK;
    }
  }
  LOVE_COUNT_LAUNCH();
  k_pcg_symbol<<<ceil_div(kp.N, 256), 256, 0, s>>>((const double*)kp.lam_d, kp.N, bhat, gh.noise, sym, &gm->lk_bits);
  const double* yd = conv ? yb.as<double>() : (const double*)ski->ys;
  LOVE_COUNT_LAUNCH();
  k_mcg_ynorm<T><<<nblocks, 256, 0, s>>>(n, (const T*)ski->ys, conv ? yb.as<double>() : nullptr, tol, gh.noise, pp, cg);
  LOVE_COUNT_LAUNCH(); k_gm_target<<<1, 1, 0, s>>>(gm, cg);
  LOVE_LAUNCH_CHECK();
  LOVE_TRY(scatter_any<T, double>(ski, yd, nullptr, 1.0, b, s));
  LOVE_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  TileArgs<double> ta{};
  ta.n_pad = m_pad;
  ta.kcols = GM_R + 1;
  ta.bc = bc;
  ta.Q = V;
  ta.ldq = m_pad;
  ta.y = yv;
  ta.partial = pp;
  ta.st = st;
  ta.status = ski->status;
  const int nb = std::min(4 * num_sms(), ceil_div(m_pad, 256));
  int total = 0;
  for (int cycle = 0; total < max_iter; ++cycle) {
    LOVE_COUNT_LAUNCH(); k_state_init<<<1, 1, 0, s>>>(st, GM_R, 1e-14);
    LOVE_COUNT_LAUNCH(); k_gm_start<<<mblocks, 256, 0, s>>>(m, m_pad, r, V, pp, st, gm, ski->status);
    LOVE_LAUNCH_CHECK();
    const int steps = std::min(GM_R, max_iter - total);
    for (int j = 0; j < steps; ++j) {
      double* vj = V + (int64_t)j * m_pad;
      LOVE_COUNT_LAUNCH(); k_normalize_col<double><<<nb, 256, 0, s>>>(vj, m_pad, st->scal + j, st);
      LOVE_TRY(pmul(vj, pv));
      LOVE_TRY(kmul(pv, kv));
      LOVE_COUNT_LAUNCH(); k_gm_band<<<mblocks, 256, 0, s>>>(m, m_pad, Gb.as<double>(), kv, pv, gh.noise, yv, st);
      LOVE_LAUNCH_CHECK();
      ta.j = j;
      LOVE_TRY(tile_run<double, MODE_DOT>(ta, s));
      LOVE_TRY(tile_run<double, MODE_UPDATE_DOT>(ta, s));
      LOVE_TRY(tile_run<double, MODE_UPDATE_NORM>(ta, s));
      LOVE_COUNT_LAUNCH(); k_gm_givens<<<1, 1, 0, s>>>(st, gm, j, ski->status);
      LOVE_LAUNCH_CHECK();
      if (j % 6 == 5) {   // stop launching once the cycle has converged
        int done = 0;
        LOVE_CUDA(cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        LOVE_CUDA(cudaStreamSynchronize(s));
        if (done) break;
      }
    }
    // z += P V y; a = K z
    LOVE_COUNT_LAUNCH(); k_gm_solve<<<1, 1, 0, s>>>(gm);
    LOVE_COUNT_LAUNCH(); k_gm_combine<<<mblocks, 256, 0, s>>>(m, V, m_pad, gm, u);
    LOVE_TRY(pmul(u, pv));
    LOVE_COUNT_LAUNCH(); k_gm_add<<<mblocks, 256, 0, s>>>(m, z, pv);
    LOVE_TRY(kmul(z, a));
    LOVE_LAUNCH_CHECK();
    int hs[2] = {0, 0};   // columns, converged
    LOVE_CUDA(cudaMemcpyAsync(&hs[0], &gm->ncols, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaMemcpyAsync(&hs[1], &gm->converged, sizeof(int), cudaMemcpyDeviceToHost, s));
    LOVE_CUDA(cudaStreamSynchronize(s));
    total += hs[0];
    if (hs[1]) *converged = true;
    if (hs[1] || hs[0] == 0) break;   // converged, or no progress possible
    // restart from the recomputed residual r = b - A z
    LOVE_COUNT_LAUNCH(); k_gm_resid<<<mblocks, 256, 0, s>>>(m, Gb.as<double>(), a, z, b, gh.noise, r);
    LOVE_LAUNCH_CHECK();
  }
  if (iters) *iters = total;
  return LOVE_OK;
}

template love_status mean_grid_gmres<float>(love_ski*, double, int, double*, int*, bool*, cudaStream_t);
template love_status mean_grid_gmres<double>(love_ski*, double, int, double*, int*, bool*, cudaStream_t);

}  // namespace love
