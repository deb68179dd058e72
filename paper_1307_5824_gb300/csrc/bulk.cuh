// bulk.cuh -- one-dimensional bulk copies global -> shared memory through the tensor
// memory accelerator (cp.async.bulk, completion counted on an mbarrier), with a bounded
// wait.  Shared by the kernels that stage a contiguous block (an image) in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace firm {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One arrival expected (the issuing thread's arrive.expect_tx); call from one thread,
// then __syncthreads before any thread waits on it.
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issuing thread: the barrier's phase completes when `bytes` have landed in dst.
// dst, src 16-byte aligned, bytes a multiple of 16.  The caller orders earlier generic
// accesses of dst before the copy (fence.proxy.async after a barrier).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Waits for phase `parity` of the barrier, at most `max_tries` polls (each a try_wait
// that may suspend the thread for a short, hardware-chosen time).  Returns false if it
// gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, uint32_t max_tries = 1u << 22) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < max_tries; ++i) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace firm
