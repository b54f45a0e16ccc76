// umma.cuh -- helpers for the 5th-generation tensor cores (tcgen05) shared by
// the tensor-core products: split TF32 operands, shared-memory matrix and
// instruction descriptors for kind::tf32 with 128 x 128 tiles, the MMA, its
// commit to an mbarrier, tensor-memory loads and the canonical operand layout.
#pragma once
#include "love_internal.cuh"

namespace love {

// Split TF32: each FP32 operand is split into two TF32 parts, x = hi + lo (hi = x rounded to
// TF32, lo = the rounded remainder), and each product is accumulated as
// hi*hi + hi*lo + lo*hi in FP32 (the lo*lo term, ~2^-22 relative, is dropped):
// close to FP32 accuracy on the TF32 tensor path.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

constexpr int UM = 128, UN = 128, UKC = 24;   // tile and K chunk (3 K steps of 8)
constexpr uint32_t U_TILE_BYTES = UM * UKC * 4;   // one operand part per chunk (12 KB)
constexpr uint32_t U_SLICE_BYTES = UM * 16;       // one 16-byte K slice of 128 rows (2 KB)
constexpr size_t U_SMEM = 2 * 4 * (size_t)U_TILE_BYTES + 64;   // two buffers of 4 parts + barriers

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr) {
  // start address >> 4 | leading (K) byte offset >> 4 | stride (M/N) byte offset >> 4 |
  // descriptor version 1 (bit 46); no swizzle, base offset 0
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(U_SLICE_BYTES >> 4) << 16) |
         ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
}
// instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t U_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(UN >> 3) << 17) |
                             ((uint32_t)(UM >> 4) << 24);

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(U_IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// byte offset of element (row r, column k) of a chunk tile in the canonical layout
__device__ __forceinline__ uint32_t umma_off(int r, int k) {
  return (uint32_t)(k >> 2) * U_SLICE_BYTES + (uint32_t)(r >> 3) * 128u + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

// tensor-memory allocation of ncols columns by one whole warp (the address is
// written to *slot in shared memory), and its release
__device__ __forceinline__ void tmem_alloc_warp(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_warp(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// a row-major FP32 operand tile (128 rows of ld floats, 16-byte aligned rows)
// held in registers for one K chunk: thread -> row tid / 2, 4-column groups
// (tid & 1) * 4 + 8 q (q < UKC / 8); zero past `rows` and past `kmax`
struct RowTileRegs {
  float4 v[UKC / 8];
  __device__ __forceinline__ void load(const float* base, int64_t ld, int64_t row0, int64_t rows, int c0, int kmax,
                                       int tid) {
    const int64_t r = row0 + (tid >> 1);
    const int k0 = (tid & 1) * 4;
    const float* p = base + r * ld + c0;
#pragma unroll
    for (int q = 0; q < UKC / 8; ++q) {
      const int k = k0 + 8 * q;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows && c0 + k < kmax) {
        if (c0 + k + 3 < kmax) {
          x = *reinterpret_cast<const float4*>(p + k);
        } else {
          x.x = p[k];
          if (c0 + k + 1 < kmax) x.y = p[k + 1];
          if (c0 + k + 2 < kmax) x.z = p[k + 2];
        }
      }
      v[q] = x;
    }
  }
  // split into TF32 hi / lo parts, one 16-byte core-matrix row per store
  __device__ __forceinline__ void store(unsigned char* hi, unsigned char* lo, int kc, int tid) const {
    const int r = tid >> 1, k0 = (tid & 1) * 4;
#pragma unroll
    for (int q = 0; q < UKC / 8; ++q) {
      if (k0 + 8 * q < kc) {
        uint4 h, l;
        split_tf32(v[q].x, h.x, l.x);
        split_tf32(v[q].y, h.y, l.y);
        split_tf32(v[q].z, h.z, l.z);
        split_tf32(v[q].w, h.w, l.w);
        const uint32_t o = umma_off(r, k0 + 8 * q);
        *reinterpret_cast<uint4*>(hi + o) = h;
        *reinterpret_cast<uint4*>(lo + o) = l;
      }
    }
  }
};

// the three split-TF32 MMAs of each K step of a chunk (one thread)
__device__ __forceinline__ void umma_chunk(uint32_t tmem, const unsigned char* Ahi, const unsigned char* Alo,
                                           const unsigned char* Bhi, const unsigned char* Blo, int kc,
                                           bool first) {
  const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
  for (int q = 0; q < kc / 8; ++q) {
    const uint32_t off = (uint32_t)q * 2u * U_SLICE_BYTES;
    umma_tf32(tmem, umma_smem_desc(ahi + off), umma_smem_desc(bhi + off), (first && q == 0) ? 0u : 1u);
    umma_tf32(tmem, umma_smem_desc(ahi + off), umma_smem_desc(blo + off), 1u);
    umma_tf32(tmem, umma_smem_desc(alo + off), umma_smem_desc(bhi + off), 1u);
  }
}

}  // namespace love
