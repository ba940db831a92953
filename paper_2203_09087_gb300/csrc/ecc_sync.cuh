// ecc_sync.cuh -- bounded device-side waits (device only).
//
// Every wait in the library's kernels ends: it polls against %globaltimer
// and gives up after a limit, after which the caller records DEV_TIMEOUT in
// the device status word (read by the host through ecc_status_get) and
// leaves without hanging the GPU.  The scan's look-back spins on a flag, the
// TMA ring waits on mbarrier phases; ecc_selftest_wait_timeout makes both
// kinds run out on purpose.
#pragma once

#include <stdint.h>

#include "ecc_internal.h"

namespace ecc {
namespace sync {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the mbarrier phase `parity` to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kSpinLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

// Wait until *flag != 0; returns the flag, or 0 after limit_ns.
__device__ __forceinline__ int flag_wait(volatile int *flag, unsigned long long limit_ns = kSpinLimitNs)
{
    int v = *flag;
    if (v) return v;
    const unsigned long long t0 = globaltimer();
    while ((v = *flag) == 0)
        if (globaltimer() - t0 > limit_ns) return 0;
    return v;
}

}  // namespace sync
}  // namespace ecc
