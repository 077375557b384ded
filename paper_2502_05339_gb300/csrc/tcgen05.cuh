// tcgen05 / UMMA helpers shared by the tensor-core kernels (sm_103a): tensor
// memory allocation, fences, MMA issue (A in shared or tensor memory),
// tensor-memory loads and stores, shared-memory matrix descriptors of the
// K-major no-swizzle layout, and the bf16 hi / lo splits of FP32 operands.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "ptx.cuh"

namespace dmd {

namespace {

// ------------------------------------------------------------ PTX helpers
// (mbarrier, TMA and bulk-copy helpers are in ptx.cuh)

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, FP32 accumulation.
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]^T (A: 128 lanes = rows, 8 columns per 16-wide K-slice)
__device__ __forceinline__ void umma_bf16_ta(uint32_t d, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// ---- CTA-pair forms (a 2-CTA cluster; a kernel uses one form only).  The
// allocation is issued by one warp of each CTA of the pair; the products are
// issued by the even CTA and span both: A (M = 256) is the lanes of both
// CTAs' tensor memory or shared memory at the same address, B's N columns
// are split, the first half from the even CTA's shared memory, the second
// from its peer's at the same address; D is split by rows like A.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_pair_ta(uint32_t d, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                             uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive on the mbarrier at the same shared-memory offset in both CTAs of the
// pair once the issuing thread's earlier products have finished.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          su32(bar)),
      "h"((uint16_t)3)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// As tmem_ld16 without the wait: several loads can be in flight before one
// tmem_ld_wait().
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle.  lbo: byte distance
// between K-adjacent core matrices, sbo: between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of tcgen05
  return d;                 // base offset 0, absolute LBO mode, layout type 0 = no swizzle
}
constexpr uint32_t kLBO = 128, kSBO = 256;

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of the 16-byte chunk (row, half) of a rows x 16 K-slice.
__device__ __forceinline__ uint32_t kslice_off(int row, int half) {
  return (uint32_t)((row >> 3) * 256 + half * 128 + (row & 7) * 16);
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Split 16 consecutive-K FP32 values into hi/lo and store them as one K-slice
// row (two 16-byte chunks each) at `hi` and `lo` (slice bases).
__device__ __forceinline__ void split_store_row(const float* x, uint8_t* hi, uint8_t* lo, int row) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(x[2 * i + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
    h[i] = pack2(h0, h1);
    l[i] = pack2(l0, l1);
  }
  *reinterpret_cast<uint4*>(hi + kslice_off(row, 0)) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(hi + kslice_off(row, 1)) = make_uint4(h[4], h[5], h[6], h[7]);
  *reinterpret_cast<uint4*>(lo + kslice_off(row, 0)) = make_uint4(l[0], l[1], l[2], l[3]);
  *reinterpret_cast<uint4*>(lo + kslice_off(row, 1)) = make_uint4(l[4], l[5], l[6], l[7]);
}

// 3-way split x = hi + mid + lo (bf16 each; exact for FP32 x up to the last
// bit of lo) stored as three K-slice planes spaced `plane` bytes apart.
__device__ __forceinline__ void split3_store_row(const float* x, uint8_t* base, uint32_t plane, int row) {
  uint32_t h[8], m[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    __nv_bfloat16 hv[2], mv[2], lv[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float v = x[2 * i + t];
      hv[t] = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(hv[t]);
      mv[t] = __float2bfloat16_rn(r1);
      lv[t] = __float2bfloat16_rn(r1 - __bfloat162float(mv[t]));
    }
    h[i] = pack2(hv[0], hv[1]);
    m[i] = pack2(mv[0], mv[1]);
    l[i] = pack2(lv[0], lv[1]);
  }
  uint8_t* p0 = base;
  uint8_t* p1 = base + plane;
  uint8_t* p2 = base + 2 * plane;
  *reinterpret_cast<uint4*>(p0 + kslice_off(row, 0)) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(p0 + kslice_off(row, 1)) = make_uint4(h[4], h[5], h[6], h[7]);
  *reinterpret_cast<uint4*>(p1 + kslice_off(row, 0)) = make_uint4(m[0], m[1], m[2], m[3]);
  *reinterpret_cast<uint4*>(p1 + kslice_off(row, 1)) = make_uint4(m[4], m[5], m[6], m[7]);
  *reinterpret_cast<uint4*>(p2 + kslice_off(row, 0)) = make_uint4(l[0], l[1], l[2], l[3]);
  *reinterpret_cast<uint4*>(p2 + kslice_off(row, 1)) = make_uint4(l[4], l[5], l[6], l[7]);
}

// Round a dynamic shared-memory pointer up to 1024 bytes by pointer
// arithmetic (an integer round trip would lose the shared address space and
// turn every later access into a generic one).
__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return p + ((1024u - (su32(p) & 1023u)) & 1023u);
}

}  // namespace

}  // namespace dmd
