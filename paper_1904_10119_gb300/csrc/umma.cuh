// umma.cuh -- inline-PTX wrappers for the Blackwell fifth-generation tensor
// cores (tcgen05): tensor-memory allocation, loads and stores between
// registers and tensor memory, BF16 MMAs with the A operand in tensor memory
// and the B operand in shared memory, and their completion through an
// mbarrier.
//
// Conventions (PTX ISA, tcgen05):
//   - a tensor-memory address is (lane << 16) | column; a warp reaches only
//     the 32 lanes 32*(warp % 4) .. +31;
//   - A (M x K, BF16) in tensor memory: row m in lane m, two K-consecutive
//     BF16 values per 32-bit column, the smaller K index in the low half;
//   - B (N x K, BF16) in shared memory, K-major with the 128-byte swizzle:
//     row n of 64 K values (128 bytes) at (n / 8) * 1024 + (n % 8) * 128 in a
//     1024-byte aligned block, its 16-byte chunk c stored at chunk c ^ (n % 8);
//     a K step of 16 values advances the descriptor's start address by 32 bytes;
//   - D (M x N, FP32) in tensor memory: row m in lane m, column n in column n.
#pragma once

#include <stdint.h>

#include "tma.cuh"

namespace fft3 {

// ------------------------------------------------------- allocation ------ //
// Whole-warp operations.  ncols: a power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ----------------------------------------------------------- fences ------ //
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ------------------------------------------- registers <-> tensor memory - //
// 32x32b shape: thread i of the warp moves lane (taddr lane + i), columns
// [col, col + 16).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
                 "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// --------------------------------------------------------------- MMA ----- //
// Instruction descriptor of kind::f16 with BF16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4)                     // D format: F32
           | (1u << 7) | (1u << 10)      // A, B format: BF16
           | ((uint32_t)(N >> 3) << 17)  // N / 8
           | ((uint32_t)(M >> 4) << 24); // M / 16
}

// Shared-memory descriptor of a K-major operand with the 128-byte swizzle
// whose 8-row atoms are 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// D (+)= A * B^T: A in tensor memory, B through its descriptor.
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            bool accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
                 : "memory");
}

// The mbarrier receives one arrival once every MMA this thread issued before
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// --------------------------------------------------- split BF16 ---------- //
// (re, im) -> hi = (bf16(re), bf16(im)) and lo = (bf16(re - hi.re),
// bf16(im - hi.im)), packed with re in the low half (round to nearest even).
__device__ __forceinline__ void split_c(float re, float im, uint32_t &hi, uint32_t &lo)
{
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(im), "f"(re));
    const float hr = __uint_as_float(hi << 16), hm = __uint_as_float(hi & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(im - hm), "f"(re - hr));
}

} // namespace fft3
