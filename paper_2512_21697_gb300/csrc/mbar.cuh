// mbar.cuh -- shared-memory mbarriers and the bulk-copy engine (cp.async.bulk), with bounded waits
// (the ring buffers of the owner/gather passes), and the asynchronous copies with which the
// factorised apply stages its tables.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace dg {
namespace {

constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz: bulk-copy wait limit

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// try_wait with a suspend-time hint: a waiting warp sleeps until the phase completes (or the hint
// runs out) instead of spinning, so warps that wait leave the issue slots to those that compute
constexpr uint32_t SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(SUSPEND_NS)
        : "memory");
    return ok != 0;
}

// wait for a ring stage; false after the time limit (the caller records the failure)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = WAIT_CYCLES)
{
    long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// the same wait without the suspend-time hint: for rings whose consumers have nothing else to do and
// whose stages complete within a few microseconds, polling keeps the wake-up latency at one poll
__device__ __forceinline__ bool mbar_test_poll(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_poll(uint64_t* bar, uint32_t parity, long long limit = WAIT_CYCLES)
{
    long long t0 = clock64();
    while (!mbar_test_poll(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// asynchronous global -> shared copy (cp.async) of 16 bytes, zero fill when src_bytes is 0;
// completion by cp_async_wait_all
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace
}  // namespace dg
