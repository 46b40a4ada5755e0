// Bulk asynchronous copies (the copy engine of sm_90+ / sm_103a) and mbarrier
// completion, as inline PTX (internal header).
//
// Rules the callers keep:
//   - every global and shared address of a bulk copy is 16-byte aligned and every
//     size a multiple of 16 bytes;
//   - the bytes announced with mbar_arrive_expect_tx equal the bytes of the copies
//     that complete on that barrier in the same phase;
//   - a thread that wrote shared memory which a bulk store will read executes
//     fence_proxy_async_shared() before the barrier that precedes the store;
//   - every wait is bounded (mbar_wait_bounded): a kernel never spins forever.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {
namespace bulk {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the copy engine before any copy names it.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One bounded probe of the barrier's phase; suspends at most about `hint_ns`.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; gives up after about a
// second (2^20 probes of at most ~1 us each) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (int it = 0; it < (1 << 20); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// global -> shared bulk copy completing on `bar` (complete_tx of `bytes`).
__device__ __forceinline__ void g2s(void *dst_smem, const void *src_gmem, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared -> global bulk copy, tracked by the issuing thread's bulk async-group.
__device__ __forceinline__ void s2g(void *dst_gmem, const void *src_smem, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst_gmem),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// Wait until the issuing thread's committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// Order this thread's generic-proxy writes to shared memory before later async-proxy reads.
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Hint: pull `bytes` (multiple of 16, 16-byte aligned) of global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void *src_gmem, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src_gmem), "r"(bytes) : "memory");
}

}  // namespace bulk
}  // namespace fps
