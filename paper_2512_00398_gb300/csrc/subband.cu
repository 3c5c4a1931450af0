// subband.cu -- stage 2 of the sub-band (two-stage) dedispersion variant.
//
// Stage 1 (the segmented byte-row kernel in dedisp.cu) leaves, per chunk of
// groups, the partial sums B[s][g][u] of every sub-band s at the nominal trial
// of every group g.  Stage 2 forms each trial's series as the sum over
// sub-bands of B[s][g(d)] shifted by the delay of the sub-band's first
// channel at the trial's own DM:
//     D~[d][t] = sum_s B[s][g(d)][t + top[d][s]].
// The values are int32 partial sums; the work is one add per sub-band and
// sample, the reads one int32 each (the rows of a warp's trial are read at a
// warp-uniform offset, 32 consecutive samples per load instruction), so the
// kernel is bound by the L1/L2 bandwidth of those reads.  The warps of a
// block are consecutive trials, mostly of one group: they read the same rows
// at nearby offsets, which L1 serves.
#include <algorithm>

#include "common.cuh"
#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kSumWarps = 8;      // trials per block
constexpr int kSumK = 16;         // samples per lane: lane + 32 k

__global__ void __launch_bounds__(32 * kSumWarps)
subband_sum_kernel(const __grid_constant__ SubbandArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = a.d_begin + (int)blockIdx.y * kSumWarps + warp;
    if (d >= a.d_end) return;
    const int64_t t0 = (int64_t)blockIdx.x * (32 * kSumK);
    const int64_t nvalid = a.nout - t0;          // > 0 for every block of the grid
    const int g = d / a.G;
    const int64_t row0 = (int64_t)(g / a.gchunk - a.c0) * a.nsub * a.gchunk + g % a.gchunk;
    const int32_t* top = a.top + (int64_t)d * a.nsub;
    int32_t acc[kSumK];
#pragma unroll
    for (int k = 0; k < kSumK; ++k) acc[k] = 0;
    if (nvalid >= 32 * kSumK) {
        for (int s = 0; s < a.nsub; ++s) {
            const int32_t* row = a.B + (row0 + (int64_t)s * a.gchunk) * a.bpitch + t0 + __ldg(top + s);
#pragma unroll
            for (int k = 0; k < kSumK; ++k) acc[k] += __ldg(row + lane + 32 * k);
        }
    } else {
        for (int s = 0; s < a.nsub; ++s) {
            const int32_t* row = a.B + (row0 + (int64_t)s * a.gchunk) * a.bpitch + t0 + __ldg(top + s);
#pragma unroll
            for (int k = 0; k < kSumK; ++k)
                if (lane + 32 * k < nvalid) acc[k] += __ldg(row + lane + 32 * k);
        }
    }
    int32_t* o = a.out + (int64_t)d * a.out_pitch + t0;
#pragma unroll
    for (int k = 0; k < kSumK; ++k)
        if (lane + 32 * k < nvalid) o[lane + 32 * k] = acc[k];
}

}  // namespace

cudaError_t launch_subband_sum(const SubbandArgs& a, cudaStream_t s) {
    if (a.nout <= 0 || a.d_end <= a.d_begin) return cudaSuccess;
    const int64_t nx = (a.nout + 32 * kSumK - 1) / (32 * kSumK);
    if (nx > 0x7fffffff) return cudaErrorInvalidValue;
    // at most 65535 blocks along y per launch
    constexpr int kTrialsPerLaunch = 65535 * kSumWarps;
    for (int d0 = a.d_begin; d0 < a.d_end; d0 += kTrialsPerLaunch) {
        SubbandArgs part = a;
        part.d_begin = d0;
        part.d_end = (int)std::min<int64_t>((int64_t)d0 + kTrialsPerLaunch, a.d_end);
        const unsigned ny = (unsigned)((part.d_end - part.d_begin + kSumWarps - 1) / kSumWarps);
        subband_sum_kernel<<<dim3((unsigned)nx, ny), 32 * kSumWarps, 0, s>>>(part);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hp
