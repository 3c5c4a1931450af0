// rfi.cu -- RFI mitigation before dedispersion (Section II-B "RFI
// Mitigation", Section III-C: broadband interference is found on the DM = 0
// series, narrowband interference is confined to a few channels).  Reading:
//   m_c = lower median of channel c, s_c = lower median of |x - m_c| (exact,
//   from 256-bin counts); channel c is narrowband RFI iff |m_c - M_m| >
//   nb_k max(D_m, 1) or |s_c - M_s| > nb_k max(D_s, 1), with M, D the lower
//   median and median absolute deviation of m_c (s_c) across channels;
//   z[t] = sum_c x[t][c] with flagged channels at m_c; with the search's
//   baseline and robust sigma of z, sample t is broadband RFI iff
//   |z - b|[t] >= bb_k sigma_z; flagged channels and samples take m_c.
// All integer except sigma_z and its threshold, which are computed exactly as
// the per-trial thresholds of the search (FP64, correctly rounded, ceil).
#include "common.cuh"

namespace hp {
namespace {

constexpr int kRfiChunk = 16384;   // samples of one channel per histogram block

// 256-bin histogram of channel rows of xt (samples t < nsamps only); one
// sub-histogram per warp against shared-memory atomic contention.
__global__ void __launch_bounds__(256) chan_hist_kernel(const uint8_t* __restrict__ xt,
                                                        int64_t pitch, int64_t nsamps,
                                                        uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[8][256];
    const int c = blockIdx.y, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint8_t* row = xt + (int64_t)c * pitch;
    const int64_t t0 = (int64_t)blockIdx.x * kRfiChunk;
    const int64_t t1 = min(nsamps, t0 + kRfiChunk);
    for (int64_t t = t0 + 16 * threadIdx.x; t < t1; t += 16 * blockDim.x) {
        const uint4 q = *reinterpret_cast<const uint4*>(row + t);   // rows are 16-byte aligned
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
        const int nb = (int)min((int64_t)16, t1 - t);
#pragma unroll
        for (int b = 0; b < 16; ++b)
            if (b < nb) atomicAdd(&h[warp][(w[b >> 2] >> (8 * (b & 3))) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 256; v += blockDim.x) {
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += h[k][v];
        if (sum) atomicAdd(&hist[(int64_t)c * 256 + v], sum);
    }
}

// lower median (element (n-1)/2 of the sorted values) from 256 counts
__device__ int median256(const uint32_t* h, int64_t n) {
    const int64_t k = (n - 1) / 2;
    int64_t c = 0;
    for (int v = 0; v < 256; ++v) {
        c += h[v];
        if (c > k) return v;
    }
    return 255;
}

// per channel: m_c and s_c (the latter from the same counts: |v - m| = d
// collects the bins m - d and m + d)
__global__ void chan_median_kernel(const uint32_t* __restrict__ hist, int64_t nsamps, int nch,
                                   int32_t* __restrict__ med, int32_t* __restrict__ spread) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    const uint32_t* h = hist + (int64_t)c * 256;
    const int m = median256(h, nsamps);
    const int64_t k = (nsamps - 1) / 2;
    int64_t cum = 0;
    int s = 255;
    for (int d = 0; d < 256; ++d) {
        cum += (m - d >= 0 ? h[m - d] : 0) + (d > 0 && m + d < 256 ? h[m + d] : 0);
        if (cum > k) { s = d; break; }
    }
    med[c] = m;
    spread[c] = s;
}

// one block: the cross-channel statistics and the channel flags (also sets the
// width list {1} of the zero-DM statistics)
__global__ void __launch_bounds__(1024) nb_flag_kernel(const int32_t* __restrict__ med,
                                                       const int32_t* __restrict__ spread, int nch,
                                                       int nb_k, uint8_t* __restrict__ flag,
                                                       int32_t* __restrict__ one) {
    __shared__ uint32_t hm[256], hs[256];
    __shared__ int s_M[2], s_D[2];
    for (int v = threadIdx.x; v < 256; v += blockDim.x) { hm[v] = 0; hs[v] = 0; }
    if (threadIdx.x == 0) *one = 1;
    __syncthreads();
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        atomicAdd(&hm[med[c]], 1u);
        atomicAdd(&hs[spread[c]], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_M[0] = median256(hm, nch); s_M[1] = median256(hs, nch); }
    __syncthreads();
    const int Mm = s_M[0], Ms = s_M[1];
    for (int v = threadIdx.x; v < 256; v += blockDim.x) { hm[v] = 0; hs[v] = 0; }
    __syncthreads();
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        atomicAdd(&hm[abs(med[c] - Mm)], 1u);
        atomicAdd(&hs[abs(spread[c] - Ms)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_D[0] = median256(hm, nch); s_D[1] = median256(hs, nch); }
    __syncthreads();
    const int64_t lim_m = (int64_t)nb_k * max(s_D[0], 1), lim_s = (int64_t)nb_k * max(s_D[1], 1);
    for (int c = threadIdx.x; c < nch; c += blockDim.x)
        flag[c] = (abs(med[c] - Mm) > lim_m || abs(spread[c] - Ms) > lim_s) ? 1 : 0;
}

// z[t] = sum over channels of xt[c][t] (flagged channels already hold m_c):
// each thread owns 16 consecutive samples, walks the channels with 16-byte
// loads (coalesced along time), sums the bytes in 16-bit lanes and flushes
// them into int32 before 257 channels
__global__ void __launch_bounds__(256) zero_dm_kernel(const uint8_t* __restrict__ xt,
                                                      int64_t pitch, int64_t nsamps, int nch,
                                                      int32_t* __restrict__ z) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t t = g << 4;
    if (t >= nsamps) return;
    uint32_t tot[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) tot[k] = 0;
    for (int c0 = 0; c0 < nch; c0 += 256) {
        uint32_t lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};   // bytes (0, 2) and (1, 3)
        const int c1 = min(nch, c0 + 256);
        for (int c = c0; c < c1; ++c) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(xt + (int64_t)c * pitch + t));
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                lo[k] += __byte_perm(w[k], 0, 0x4240);
                hi[k] += __byte_perm(w[k], 0, 0x4341);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            tot[4 * k + 0] += lo[k] & 0xFFFFu;
            tot[4 * k + 2] += lo[k] >> 16;
            tot[4 * k + 1] += hi[k] & 0xFFFFu;
            tot[4 * k + 3] += hi[k] >> 16;
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (t + k < nsamps) z[t + k] = (int32_t)tot[k];
}

// broadband flags from y_z = z - b and the integer threshold ceil(bb_k sigma_z)
__global__ void samp_flag_kernel(const int32_t* __restrict__ y, int64_t nsamps,
                                 const int64_t* __restrict__ tint, uint8_t* __restrict__ sflag,
                                 int64_t nflag) {
    const int64_t thr = tint[0];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nflag;
         t += (int64_t)gridDim.x * blockDim.x) {
        bool f = false;
        if (t < nsamps) {
            const int64_t v = y[t];
            f = (v < 0 ? -v : v) >= thr;     // thr is LLONG_MAX when sigma_z = 0
        }
        sflag[t] = f ? 1 : 0;
    }
}

__device__ __forceinline__ uint32_t replace_bytes(uint32_t v, uint32_t f, uint32_t m4) {
    const uint32_t mask = f * 255u;          // bytes 0 / 1 -> 0x00 / 0xFF
    return (v & ~mask) | (m4 & mask);
}

// xt rows in place: a flagged channel takes m_c for every t < nsamps; other
// channels take m_c at flagged samples (only 16-byte groups with a flag are
// read and written)
__global__ void __launch_bounds__(256) apply_xt_kernel(uint8_t* __restrict__ xt, int64_t pitch,
                                                       int64_t nsamps,
                                                       const uint8_t* __restrict__ cflag,
                                                       const uint8_t* __restrict__ sflag,
                                                       const int32_t* __restrict__ med,
                                                       int samples) {
    // samples == 0: flagged channels (whole rows); 1: flagged samples of the others
    const int c = blockIdx.y;
    if ((cflag[c] != 0) == (samples != 0)) return;
    const uint32_t m4 = 0x01010101u * (uint32_t)med[c];
    const bool whole = samples == 0;
    uint8_t* row = xt + (int64_t)c * pitch;
    const int64_t ngroups = (nsamps + 15) >> 4;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = g << 4;
        uint4 f = *reinterpret_cast<const uint4*>(sflag + t);   // zero beyond nsamps
        if (whole) {
            // all 16 samples, but never past nsamps (the zero tail stays zero)
            const int nb = (int)min((int64_t)16, nsamps - t);
            const uint32_t lim[4] = {nb > 0 ? 0x01010101u >> (8 * max(0, 4 - nb)) : 0u,
                                     nb > 4 ? 0x01010101u >> (8 * max(0, 8 - nb)) : 0u,
                                     nb > 8 ? 0x01010101u >> (8 * max(0, 12 - nb)) : 0u,
                                     nb > 12 ? 0x01010101u >> (8 * max(0, 16 - nb)) : 0u};
            f = make_uint4(lim[0], lim[1], lim[2], lim[3]);
        }
        if (!(f.x | f.y | f.z | f.w)) continue;
        uint4* p = reinterpret_cast<uint4*>(row + t);
        uint4 v = *p;
        v.x = replace_bytes(v.x, f.x, m4);
        v.y = replace_bytes(v.y, f.y, m4);
        v.z = replace_bytes(v.z, f.z, m4);
        v.w = replace_bytes(v.w, f.w, m4);
        *p = v;
    }
}

// the cleaned filterbank in its own layout [nsamps][nch] (out = x elsewhere)
__global__ void __launch_bounds__(256) apply_x_kernel(const uint8_t* __restrict__ x,
                                                      uint8_t* __restrict__ out, int64_t nsamps,
                                                      int nch, const uint8_t* __restrict__ cflag,
                                                      const uint8_t* __restrict__ sflag,
                                                      const int32_t* __restrict__ med) {
    const int64_t total = nsamps * nch;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / nch;
        const int c = (int)(i - t * nch);
        out[i] = (cflag[c] || sflag[t]) ? (uint8_t)med[c] : x[i];
    }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t launch_rfi(const RfiArgs& r, cudaStream_t s, int64_t* nlaunch) {
    cudaError_t e;
    const int nch = r.nch;
    const int64_t n = r.nsamps;
    if (n <= 0 || nch <= 0) return cudaSuccess;
    if (!r.xt) return cudaErrorInvalidValue;   // the statistics come from the transposed copy
    if (nch > 65535) return cudaErrorInvalidValue;   // one grid row per channel
    if ((e = cudaMemsetAsync(r.hist, 0, (size_t)nch * 256 * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(r.samp_flag, 0, (size_t)((n + 15) / 16 * 16 + 16), s)) != cudaSuccess)
        return e;
    ++*nlaunch;
    chan_hist_kernel<<<dim3((unsigned)cdiv(n, kRfiChunk), nch), 256, 0, s>>>(r.xt, r.xt_pitch, n,
                                                                           r.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    chan_median_kernel<<<(unsigned)cdiv(nch, 128), 128, 0, s>>>(r.hist, n, nch, r.med, r.spread);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    nb_flag_kernel<<<1, 1024, 0, s>>>(r.med, r.spread, nch, r.nb_k, r.chan_flag, r.one);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ngroups = (n + 15) / 16;
    const dim3 agrid((unsigned)min(cdiv(ngroups, 256), (int64_t)64), nch);
    ++*nlaunch;
    apply_xt_kernel<<<agrid, 256, 0, s>>>(r.xt, r.xt_pitch, n, r.chan_flag, r.samp_flag, r.med, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    zero_dm_kernel<<<(unsigned)cdiv(ngroups, 256), 256, 0, s>>>(r.xt, r.xt_pitch, n, nch,
                                                               const_cast<int32_t*>(r.z.D));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_search(r.z, s, nlaunch)) != cudaSuccess) return e;
    const int64_t nflag = ngroups * 16 + 16;
    ++*nlaunch;
    samp_flag_kernel<<<(unsigned)min(cdiv(nflag, 256), (int64_t)152 * 16), 256, 0, s>>>(
        r.z.Y, n, r.z.tint, r.samp_flag, nflag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    apply_xt_kernel<<<agrid, 256, 0, s>>>(r.xt, r.xt_pitch, n, r.chan_flag, r.samp_flag, r.med, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (r.out) {
        ++*nlaunch;
        apply_x_kernel<<<(unsigned)min(cdiv(n * nch, 256), (int64_t)152 * 32), 256, 0, s>>>(
            r.x, r.out, n, nch, r.chan_flag, r.samp_flag, r.med);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hp
