// subband.cu -- stage 2 of the sub-band (two-stage) dedispersion variant.
//
// Stage 1 (the segmented byte-row kernel in dedisp.cu) leaves, per chunk of
// groups, the partial sums B[s][g][u] of every sub-band s at the nominal trial
// of every group g.  Stage 2 forms each trial's series as the sum over
// sub-bands of B[s][g(d)] shifted by the delay of the sub-band's first
// channel at the trial's own DM:
//     D~[d][t] = sum_s B[s][g(d)][t + top[d][s]].
// A block takes up to kSubbandTrials trials of one group (one consumer warp
// each) and kSubbandTile output samples.  For every sub-band a producer warp
// copies the window of B's row that the block's trials read -- the tile plus
// the spread of the trials' shifts -- into a ring of shared-memory slots with
// one bulk copy (cp.async.bulk, completion on an mbarrier); the consumer warps
// add their shifted slices from shared memory (consecutive lanes, consecutive
// words: no bank conflicts) into registers.  Each window is read from L2/HBM
// once per block, and the tile is wide enough that the windows overlap by a
// small fraction of it.  Every wait is bounded.
#include <algorithm>

#include "common.cuh"
#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kSumK = kSubbandTile / 32;   // samples per lane: lane + 32 k
constexpr int kSumSlots = 4;               // shared-memory ring of windows

__device__ __forceinline__ int32_t lds_s32(uint32_t addr) {
    int32_t v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__global__ void __launch_bounds__(32 * (kSubbandTrials + 1))
subband_sum_kernel(const __grid_constant__ SubbandArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int bpg = (a.G + kSubbandTrials - 1) / kSubbandTrials;   // blocks per group
    const int g = a.g_begin + (int)blockIdx.y / bpg;
    const int d_first = g * a.G + ((int)blockIdx.y % bpg) * kSubbandTrials;
    const int nd = min(kSubbandTrials, min((g + 1) * a.G, a.ndm) - d_first);
    if (g >= a.g_end || nd <= 0) return;                           // the whole block
    const int64_t t0 = (int64_t)blockIdx.x * kSubbandTile;
    const int64_t nvalid = a.nout - t0;                            // > 0
    const uint32_t slot_bytes = 4u * (uint32_t)a.win_cap;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kSumSlots * slot_bytes);
    uint64_t* empty = full + kSumSlots;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int b = 0; b < kSumSlots; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kSubbandTrials);
        }
        mbar_fence_init();
        abort_flag = 0;
    }
    __syncthreads();
    volatile int* abort = &abort_flag;
    const int64_t row0 = (int64_t)(g / a.gchunk - a.c0) * a.nsub * a.gchunk + g % a.gchunk;
    const int32_t* top_first = a.top + (int64_t)d_first * a.nsub;
    const int32_t* top_last = a.top + (int64_t)(d_first + nd - 1) * a.nsub;

    if (warp == kSubbandTrials) {
        // ------------------------------------------------------- producer
        if (lane != 0) return;
        int issued = 0;
        for (int s = 0; s < a.nsub; ++s) {
            const int b = s % kSumSlots;
            if (s >= kSumSlots &&
                !mbar_wait_or_abort(&empty[b], (uint32_t)(s / kSumSlots - 1) & 1u, a.timeout_ns,
                                    abort))
                break;
            // window [a0, a0 + n): 16-byte aligned start, whole 16-byte units,
            // never past the row's end
            const int64_t a0 = (t0 + top_first[s]) & ~(int64_t)3;
            int64_t n = (t0 + top_last[s] + kSubbandTile - a0 + 3) & ~(int64_t)3;
            n = min(n, a.bpitch - a0);
            mbar_arrive_expect_tx(&full[b], (uint32_t)(4 * n));
            bulk_copy_g2s(smem + b * slot_bytes, a.B + (row0 + (int64_t)s * a.gchunk) * a.bpitch + a0,
                          (uint32_t)(4 * n), &full[b]);
            issued = s + 1;
        }
        if (*abort) {
            latch_status(a.status, HP_ERR_TIMEOUT);
            for (int x = issued - kSumSlots > 0 ? issued - kSumSlots : 0; x < issued; ++x)
                mbar_wait_bounded(&full[x % kSumSlots], (uint32_t)(x / kSumSlots) & 1u, a.timeout_ns);
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    const bool active = warp < nd;
    const int32_t* top_d = a.top + (int64_t)(d_first + (active ? warp : 0)) * a.nsub;
    const uint32_t sbase = smem_u32(smem) + 4u * (uint32_t)lane;
    int32_t acc[kSumK];
#pragma unroll
    for (int k = 0; k < kSumK; ++k) acc[k] = 0;
    const bool whole = nvalid >= kSubbandTile;
    for (int s = 0; s < a.nsub; ++s) {
        const int b = s % kSumSlots;
        if (!__all_sync(0xffffffffu, mbar_wait_or_abort(&full[b], (uint32_t)(s / kSumSlots) & 1u,
                                                        a.timeout_ns, abort)))
            return;
        if (active) {
            const int64_t a0 = (t0 + top_first[s]) & ~(int64_t)3;
            const uint32_t w = sbase + b * slot_bytes + 4u * (uint32_t)(t0 + top_d[s] - a0);
            if (whole) {
#pragma unroll
                for (int k = 0; k < kSumK; ++k) acc[k] += lds_s32(w + 128u * k);
            } else {
#pragma unroll
                for (int k = 0; k < kSumK; ++k)
                    if (lane + 32 * k < nvalid) acc[k] += lds_s32(w + 128u * k);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
    if (!active) return;
    int32_t* o = a.out + (int64_t)(d_first + warp) * a.out_pitch + t0;
#pragma unroll
    for (int k = 0; k < kSumK; ++k)
        if (lane + 32 * k < nvalid) o[lane + 32 * k] = acc[k];
}

}  // namespace

cudaError_t launch_subband_sum(const SubbandArgs& a, cudaStream_t s) {
    if (a.nout <= 0 || a.g_end <= a.g_begin) return cudaSuccess;
    if (a.win_cap < kSubbandTile + 8 || a.win_cap % 4 != 0 || a.bpitch % 4 != 0)
        return cudaErrorInvalidValue;
    const int64_t nx = (a.nout + kSubbandTile - 1) / kSubbandTile;
    const int64_t bpg = (a.G + kSubbandTrials - 1) / kSubbandTrials;
    const size_t smem = (size_t)kSumSlots * 4 * a.win_cap + 2 * kSumSlots * 8;
    if (nx > 0x7fffffff || smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(subband_sum_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // at most 65535 blocks along y per launch
    const int gpl = (int)std::max<int64_t>(1, 65535 / bpg);
    for (int g0 = a.g_begin; g0 < a.g_end; g0 += gpl) {
        SubbandArgs part = a;
        part.g_begin = g0;
        part.g_end = std::min(g0 + gpl, a.g_end);
        const unsigned ny = (unsigned)((part.g_end - part.g_begin) * bpg);
        subband_sum_kernel<<<dim3((unsigned)nx, ny), 32 * (kSubbandTrials + 1), smem, s>>>(part);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hp
