// Shared-memory addresses, L2 cache policies, 1-D bulk copies (TMA) and bounded mbarrier
// waits, shared by the product kernels (spmv.cu, stage.cu).
#pragma once
#include <stdint.h>

namespace spmv {

// Polls of an mbarrier before a wait gives up (the kernel then reports ST_TIMEOUT).
constexpr long long MW_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// L2 eviction policies: the streamed matrix arrays are read once (evict first), the gathered
// x is reused across the whole product (evict last), so the stream does not push x out of L2.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 1-D bulk copy global -> shared (TMA), completion counted on an mbarrier.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol) : "memory");
}

// Bounded wait for phase `parity` of a slot barrier (all lanes); false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = MW_SPIN_LIMIT) {
    uint32_t done = 0;
    for (long long it = 0; it < limit && !done; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return __all_sync(0xffffffffu, done);
}

}  // namespace spmv
