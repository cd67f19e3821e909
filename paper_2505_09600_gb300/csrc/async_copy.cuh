// Bulk asynchronous copies global -> shared memory (the 1-D form of the
// tensor memory accelerator: cp.async.bulk) completed through an mbarrier,
// with bounded waits.
//
// Rules the callers follow:
//  - source and destination start on 16-byte boundaries and the size is a
//    multiple of 16 bytes (checked by the caller before issuing);
//  - one elected thread arms the barrier with the byte count and issues the
//    copies; every consumer waits on the barrier's phase parity;
//  - a wait gives up after kAsyncSpinLimit polls (with a short sleep between
//    polls, about a second in all): it then sets bit 0 of the device status
//    word (whose address the launch arguments carry; lisa_device_status reads
//    it) and the block leaves its work after waiting (again bounded) for its
//    own copies to land.
#pragma once

#include <stdint.h>

namespace lisa {

// Device address of the status word on the current device (host side).
unsigned int* device_status_ptr();

constexpr unsigned kAsyncSpinLimit = 1u << 23;   // x 100 ns ~ 0.8 s

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Invalidate a barrier (no operation pending on it) before its memory is
// reused for other data.
__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Non-blocking test of the phase with the given parity (test_wait never
// suspends the thread, so the poll count bounds the wait).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity: false after kAsyncSpinLimit polls
// 100 ns apart (about a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    for (unsigned it = 0; it < kAsyncSpinLimit; ++it) {
        if (mbar_test_wait(bar, parity)) return true;
        __nanosleep(100);
    }
    return false;
}

__device__ __forceinline__ void flag_timeout(unsigned int* status)
{
    if (status) atomicOr(status, 1u);
}

}  // namespace lisa
