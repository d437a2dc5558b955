// Tensor-memory-accelerator (TMA) copies into shared memory, completed on an
// mbarrier: the building blocks the binned push uses to stage a bin's field
// tile with one bulk tensor copy.  Inline PTX for sm_103a; no library.
//
// Waits are bounded: a copy that has not completed within the limit makes the
// waiting CTA report ST_TIMEOUT instead of spinning for ever.
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (the 128-byte tensor-map descriptor)
#include <cuda_runtime.h>

namespace rsol {

// Longest wait for a bulk copy, in SM clocks (about 0.2 s at 2 GHz).
constexpr long long kTmaWaitCycles = 400000000ll;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One-phase barrier with `count` arrivals; visible to the async proxy (the
// TMA unit) once the caller has synchronised the CTA after this call.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Retire a barrier before its shared memory is used again.
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Arrive once and announce `bytes` of asynchronous transfer on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// True once the barrier's phase `parity` has completed (the hardware may
// suspend the thread for a while inside one call).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` for at most `max_cycles` SM clocks; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long max_cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > max_cycles)
            return false;
    return true;
}

// 4D tiled bulk copy global -> shared of the box at coordinates (c0..c3)
// (innermost first) of the tensor described by `map`, completing `bar`'s
// transaction count.  dst must be 128-byte aligned; c0 * element size must be
// a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

} // namespace rsol
