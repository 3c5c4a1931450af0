// common.cuh -- device helpers shared by the sm_103a kernels of the search
// library: shared-memory address conversion, mbarrier + bulk-copy (TMA)
// wrappers, the bounded-wait clock and the plan's device status latch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hp_internal.h"

namespace hp {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Latch the first device-side failure of a launch sequence (HP_ERR_*).
__device__ __forceinline__ void latch_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_parity(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// As mbar_wait_bounded, but also gives up as soon as *abort becomes non-zero
// (another thread of the block already timed out).
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                   uint64_t limit_ns, volatile int* abort) {
    if (mbar_try_wait_parity(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        if (mbar_try_wait_parity(bar, parity)) return true;
        if (*abort) return false;
        if (global_timer_ns() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// Wait until the barrier's phase with the given parity has completed, giving
// up after `limit_ns` of global time.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait_parity(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        if (mbar_try_wait_parity(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy global -> shared completing on an mbarrier.  Both addresses
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst_smem, const void* src_gmem,
                                              uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Median of five values (the third smallest), by a fixed network of nine
// compare-exchanges.
__device__ __forceinline__ int32_t median5(int32_t a, int32_t b, int32_t c, int32_t d, int32_t e) {
#define HP_CX(x, y) { const int32_t lo_ = min(x, y); y = max(x, y); x = lo_; }
    HP_CX(a, b); HP_CX(d, e); HP_CX(c, e); HP_CX(c, d); HP_CX(a, d); HP_CX(a, c); HP_CX(b, e);
    HP_CX(b, d); HP_CX(b, c);
#undef HP_CX
    return c;
}

// Named barrier `id` (1-15; 0 is __syncthreads) over `nthreads` threads (a
// multiple of 32): wait for all, or arrive without waiting.
__device__ __forceinline__ void named_barrier_sync(int id, int nthreads) {
    asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void named_barrier_arrive(int id, int nthreads) {
    asm volatile("barrier.cta.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Floor division for a positive divisor.
__device__ __forceinline__ long long floor_div_pos(long long a, long long b) {
    long long q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

}  // namespace hp
