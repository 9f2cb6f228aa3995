// Shared-memory staging helpers: 1D bulk copies (TMA, cp.async.bulk) completing on
// mbarriers, and bounded mbarrier waits that give up instead of hanging.
#pragma once

namespace asicp {

constexpr long long kWaitCycles = 1LL << 32;   // bounded mbarrier wait (~2 s)
constexpr long long kTestWaitCycles = 1000;    // the wait made to expire when testing the timeout path

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive on the mbarrier at shared-memory address addr.
__device__ __forceinline__ void mbar_arrive_at(unsigned addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) { mbar_arrive_at(smem_u32(bar)); }

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bytes (a multiple of 16) from global src to shared dst (both 16-byte aligned)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_at(unsigned addr, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    return mbar_try_wait_at(smem_u32(bar), parity);
}

// Bounded wait on an mbarrier phase: false when the budget (SM clock cycles) ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit = kWaitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// The same for a whole warp (barrier at shared-memory address addr): every lane
// polls, so the warp waits converged (a single polling lane with the others parked
// at a shuffle measured slower: the tensor-core screening 0.80 -> 0.69 ms per
// paper-scale launch when its reduction warps switched to this form).  Returns
// the same verdict on every lane.  Call with all 32 lanes.
__device__ __forceinline__ bool mbar_wait_warp_at(unsigned addr, unsigned parity)
{
    bool ok = true;
    if (!mbar_try_wait_at(addr, parity)) {
        const long long t0 = clock64();
        while (!mbar_try_wait_at(addr, parity)) {
            if (clock64() - t0 > kWaitCycles) { ok = false; break; }
        }
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ bool mbar_wait_warp(unsigned long long *bar, unsigned parity)
{
    return mbar_wait_warp_at(smem_u32(bar), parity);
}

}  // namespace asicp
