// peaks.cu -- microbenchmarks of the issue rates that bound dedispersion:
// 32-bit integer adds, byte permutes (PRMT) and conflict-free 32-bit shared
// memory loads.  Each kernel runs independent dependency chains on every SM;
// rates are the best of three event-timed launches after a warm-up.
#include "../../include/hp_bench.h"
#include "common.cuh"
#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kIters = 2048;
constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

__global__ void __launch_bounds__(kThreads) int_add_bench(uint32_t* out, uint32_t seed) {
    uint32_t a[kChains], b[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        a[i] = seed + threadIdx.x + i;
        b[i] = seed * 3u + (uint32_t)i;
    }
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b[i]));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(b[i]) : "r"(a[i]));
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= a[i] ^ b[i];
    if (s == 0x9e3779b9u) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) prmt_bench(uint32_t* out, uint32_t seed) {
    uint32_t a[kChains], b[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        a[i] = seed ^ (threadIdx.x * 2654435761u) ^ (uint32_t)i;
        b[i] = seed + 77u * (uint32_t)i;
    }
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            asm volatile("prmt.b32 %0, %0, %1, 0x4240;" : "+r"(a[i]) : "r"(b[i]));
            asm volatile("prmt.b32 %0, %0, %1, 0x3715;" : "+r"(b[i]) : "r"(a[i]));
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= a[i] ^ b[i];
    if (s == 0x9e3779b9u) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) lds_bench(uint32_t* out, uint32_t seed) {
    __shared__ uint32_t buf[4096];
    for (int i = threadIdx.x; i < 4096; i += kThreads) buf[i] = seed + (uint32_t)i;
    __syncthreads();
    uint32_t acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = 0;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            const uint32_t idx = ((uint32_t)(it * kChains + i) * 32u + warp * 512u + lane) & 4095u;
            uint32_t v;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(&buf[idx])));
            acc[i] ^= v;
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= acc[i];
    if (s == 0x9e3779b9u) out[0] = s;
}

template <typename K>
double best_ms(K kernel, int blocks, uint32_t* out) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kernel<<<blocks, kThreads>>>(out, 1u);
    double best = 1e30;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        kernel<<<blocks, kThreads>>>(out, 2u + (uint32_t)r);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// The bounded waits of the staged kernels, exercised on barriers whose state
// is known: A never completes (one expected arrival, none made), B completes
// (its one arrival is made before anyone waits).  flags: status, warp 0 ran
// out on A, warp 1 gave up on A, B's wait succeeded.
__global__ void bounded_wait_kernel(uint64_t limit_ns, int* flags) {
    __shared__ uint64_t bars[2];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0) mbar_arrive(&bars[1]);
    __syncthreads();
    volatile int* abort = &abort_flag;
    const bool b_done = mbar_wait_bounded(&bars[1], 0, limit_ns);
    const bool a_done = mbar_wait_or_abort(&bars[0], 0, limit_ns, abort);
    if (!a_done) latch_status(flags, HP_ERR_TIMEOUT);
    if (lane == 0) {
        if (warp == 0 && !a_done) atomicExch(&flags[1], 1);
        if (warp == 1 && !a_done) atomicExch(&flags[2], 1);
    }
    if (tid == 0 && b_done) atomicExch(&flags[3], 1);
}

}  // namespace
}  // namespace hp

extern "C" int hp_selftest_bounded_wait(int64_t limit_ns, int32_t out[4]) {
    if (!out || limit_ns <= 0 || limit_ns > 10000000000LL) return HP_ERR_INVALID_ARG;
    int* d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(int)) != cudaSuccess) return HP_ERR_CUDA;
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        hp::bounded_wait_kernel<<<1, 64>>>((uint64_t)limit_ns, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return HP_ERR_CUDA;
    for (int i = 0; i < 4; ++i) out[i] = h[i];
    return HP_OK;
}

extern "C" int hp_dedisp_config(int config, int32_t out[8]) {
    if (!out || config < 0 || config >= hp::kNumDedispConfigs) return HP_ERR_INVALID_ARG;
    const hp::DedispConfig& c = hp::kDedispConfigs[config];
    const int32_t v[8] = {c.RD, c.NW, c.WD, c.WT, c.stage_bytes, c.stages, c.unroll, c.threads()};
    for (int i = 0; i < 8; ++i) out[i] = v[i];
    return HP_OK;
}

extern "C" int hp_measure_peaks(hp_peaks* out) {
    using namespace hp;
    if (!out) return HP_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HP_ERR_CUDA;
    uint32_t* scratch = nullptr;
    if (cudaMalloc(&scratch, 256) != cudaSuccess) return HP_ERR_CUDA;
    const int blocks = sms * kBlocksPerSM;
    const double lanes = (double)blocks * kThreads * kIters * kChains;
    const double t_add = best_ms(int_add_bench, blocks, scratch);
    const double t_prmt = best_ms(prmt_bench, blocks, scratch);
    const double t_lds = best_ms(lds_bench, blocks, scratch);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFree(scratch);
    if (e != cudaSuccess) return HP_ERR_CUDA;
    out->int_add_ops_per_s = 2.0 * lanes / (t_add * 1e-3);
    out->prmt_ops_per_s = 2.0 * lanes / (t_prmt * 1e-3);
    out->lds32_bytes_per_s = 4.0 * lanes / (t_lds * 1e-3);
    out->sm_count = sms;
    out->reserved = 0;
    return HP_OK;
}
