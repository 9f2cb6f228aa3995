// Fifth-generation tensor-core helpers (tcgen05, sm_103a): shared-memory matrix
// descriptors for the no-swizzle K-major layout, instruction descriptors of
// kind::f16, the MMA, its commit to an mbarrier, tensor-memory allocation and the
// fences around thread synchronisation.  Inline PTX only.
#pragma once
#include <cstdint>

#include "async_copy.cuh"

namespace asicp {

// Byte offset of element (row, k) of a 16-bit matrix in the no-swizzle K-major
// layout: 8-row x 16-byte core matrices, K-adjacent core matrices lbo bytes
// apart, 8-row groups sbo bytes apart.
__host__ __device__ constexpr unsigned kmajor_offset(int row, int k, unsigned lbo, unsigned sbo)
{
    return (unsigned)(row / 8) * sbo + (unsigned)(k / 8) * lbo + (unsigned)(row % 8) * 16u + (unsigned)(k % 8) * 2u;
}

// Shared-memory matrix descriptor (no swizzle) of the matrix starting at shared
// address addr.
__device__ __forceinline__ uint64_t tc_smem_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16 with a float32 accumulator, both operands
// K-major: bf16 = true for bfloat16 operands (both), false for f16; N columns, M rows.
__host__ __device__ constexpr uint32_t tc_idesc_f16(bool bf16, int n, int m)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

// D (tensor memory) = A B (accumulate = 0) or D + A B (accumulate != 0), issued by one thread.
__device__ __forceinline__ void tc_mma_f16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier at bar completes one arrival when every earlier tcgen05 operation of
// this thread is done.
__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Allocate ncols tensor-memory columns (a power of two >= 32) for the CTA; the
// whole warp calls it; the base address lands in *slot.
__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t base, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// 32 consecutive accumulator columns of this thread's lane (32x32b shape, x32),
// loaded and waited for in one statement.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace asicp
