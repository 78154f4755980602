// Bulk asynchronous copies global -> shared (the TMA engine's untiled form,
// cp.async.bulk) completed through a shared-memory mbarrier, with bounded
// waits.  Source and destination 16-byte aligned, size a multiple of 16.
#pragma once

#include <stdint.h>

namespace gfbp {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// An mbarrier expecting one arrival per phase.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Make the initialisations visible to the copy engine (before any use).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's generic-proxy accesses before later bulk copies (and
// the copies' writes before its later generic accesses).
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

// The calling thread's arrival on the barrier's current phase, announcing
// `bytes` of copies that complete on it (at most 2^20 - 1).
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// A copy of `bytes` (> 0) from global src to shared dst, completing on bar.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// The calling thread's arrival announcing `bytes` of copies on this phase,
// then the copy of `bytes` from global src to shared dst (bytes may be 0:
// the phase then completes on the arrival alone).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    mbar_arrive_expect(bar, bytes);
    if (bytes) bulk_copy(dst, src, bytes, bar);
}

// A wait gives up after about a second (the global nanosecond timer; a poll
// may suspend the thread for microseconds), or after kBulkWaitLimit polls.
constexpr unsigned long long kBulkWaitNs = 1000000000ull;
constexpr int kBulkWaitLimit = 1 << 24;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of the phase with the given parity; false when the
// bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (int n = 0; n < kBulkWaitLimit; n++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((n & 63) == 63 && global_ns() - t0 > kBulkWaitNs) return false;
    }
    return false;
}

}  // namespace
}  // namespace gfbp
