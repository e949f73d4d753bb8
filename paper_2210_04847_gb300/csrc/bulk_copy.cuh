// bulk_copy.cuh -- bulk copies from global into shared memory whose completion
// is counted on an mbarrier, and the bounded waits on them (the render kernels
// that stage their chunks in shared memory).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nacc {

// ---------------------------------------------------------------------------
// bulk copies global -> shared memory, completion counted on an mbarrier
// ---------------------------------------------------------------------------
//
// cp.async.bulk moves a contiguous run of bytes (16-byte aligned at both ends,
// a multiple of 16 bytes long) into shared memory without holding registers;
// the transfer's bytes are counted down on an mbarrier whose phase completes
// once its one expected arrival (arrive.expect_tx by the issuing lane) and all
// announced bytes have landed. Waits poll try_wait a bounded number of times.

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the asynchronous proxy (the copies).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One poll: the thread is suspended until the phase completes or about
// kWaitHintNs nanoseconds have passed (no spinning while the copies are in flight).
constexpr unsigned kWaitHintNs = 1000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return done != 0;
}

// Waits (at most `limit` polls, each at most about kWaitHintNs) for the phase of
// the given parity to complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// As bulk_copy_g2s, with the destination and barrier as shared-memory addresses.
__device__ __forceinline__ void bulk_copy_g2s_addr(uint32_t dst, const void* src, unsigned bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Orders this thread's earlier shared-memory accesses before later bulk copies
// into the same memory (reuse of a stage that was read with ordinary loads).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace nacc
