// dedisp.cu -- incoherent dedispersion on sm_103a (Section II-B, "Incoherent
// Dedispersion"): D[d][t] = sum_c x[t + delay(c,d)][c], exact integers.
//
// Two kernels:
//  * transpose_kernel: time-major uint8 [nsamps][nchans] -> channel-major
//    [nchans][xt_pitch], zero padded, so that every channel row is a
//    contiguous byte stream a bulk copy can stage.
//  * dedisp_kernel: one block per (DM tile, time tile).  Channel rows are
//    staged into shared memory with cp.async.bulk (TMA, completion on an
//    mbarrier, two stages in flight).  Three byte-shifted copies of each row
//    are built so that every (trial, channel) read is an aligned 32-bit word
//    holding four consecutive samples.  Bytes are split into two 16-bit lanes
//    (PRMT) and summed SIMD-within-a-register; at most 256 channels are
//    summed per stage, so a lane never exceeds 256 * 255 < 2^16, and the
//    lanes are flushed into int32 sums after every stage.  No tensor cores:
//    the sum is not a dense contraction.
#include <cstring>

#include "common.cuh"

namespace hp {

const DedispConfig kDedispConfigs[kNumDedispConfigs] = {
    {2, 4, 8, 1, 48 * 1024},   // BD 16, BT 512
    {4, 2, 8, 1, 48 * 1024},   // BD 32, BT 256
    {2, 4, 4, 2, 48 * 1024},   // BD 8,  BT 1024
    {4, 4, 8, 1, 52 * 1024},   // BD 32, BT 512
};

namespace {

constexpr int kTT = 64;

__global__ void __launch_bounds__(256) transpose_kernel(const uint8_t* __restrict__ x,
                                                        int64_t nsamps, int nch, int vec,
                                                        uint8_t* __restrict__ xt, int64_t pitch) {
    __shared__ __align__(16) uint8_t tile[kTT][kTT + 16];
    const int64_t t0 = (int64_t)blockIdx.x * kTT;
    const int c0 = blockIdx.y * kTT;
    const int tid = threadIdx.x;
    {
        const int row = tid >> 2, seg = tid & 3;
        const int64_t t = t0 + row;
        const int c = c0 + seg * 16;
        uint4 q = make_uint4(0, 0, 0, 0);
        if (t < nsamps) {
            if (vec && c + 16 <= nch) {
                q = __ldg(reinterpret_cast<const uint4*>(x + t * nch + c));
            } else {
                uint8_t v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = (c + i < nch) ? x[t * nch + c + i] : 0;
                memcpy(&q, v, 16);
            }
        }
        *reinterpret_cast<uint4*>(&tile[row][seg * 16]) = q;
    }
    __syncthreads();
    {
        const int cr = tid >> 2, seg = tid & 3;
        const int c = c0 + cr;
        const int64_t t = t0 + seg * 16;
        if (c < nch && t < pitch) {
            uint8_t v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = tile[seg * 16 + i][cr];
            uint4 q;
            memcpy(&q, v, 16);
            *reinterpret_cast<uint4*>(xt + (int64_t)c * pitch + t) = q;
        }
    }
}

__host__ __device__ constexpr uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

template <int RD, int NW, int WD, int WT>
__global__ void __launch_bounds__(256, 2)
dedisp_kernel(const __grid_constant__ DedispBatch batch, int stage_bytes, int* status,
              uint64_t timeout_ns) {
    constexpr int BD = WD * RD;
    constexpr int NT = 256;
    constexpr int BT = WT * NW * 128;
    static_assert(WD * WT * 32 == NT, "block is 8 warps");
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes);

    const int64_t blk = blockIdx.x;
    int jb = 0;
    while (jb + 1 < batch.njobs && batch.prefix[jb + 1] <= blk) ++jb;
    const DedispJob& J = batch.jobs[jb];
    const int64_t item = blk - batch.prefix[jb];
    const int tt = (int)(item % J.ntt);
    const int dt = (int)(item / J.ntt);
    const TileDesc T = J.tiles[dt];
    const int64_t t0 = (int64_t)tt * BT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wd = warp % WD, wt = warp / WD;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    uint32_t acc_lo[RD][NW], acc_hi[RD][NW];
    uint32_t sum[RD][NW][4];
#pragma unroll
    for (int r = 0; r < RD; ++r)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            acc_lo[r][k] = 0;
            acc_hi[r][k] = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) sum[r][k][e] = 0;
        }

    // warp 0 stages channel descriptors, the word-address table and the rows
    auto issue = [&](int s, int buf) {
        const StageDesc S = J.stages[T.stage_begin + s];
        uint8_t* B = smem + buf * stage_bytes;
        if (lane == 0) {
            mbar_arrive_expect_tx(&bars[buf], S.tx_bytes);
            bulk_copy_g2s(B, J.chans + S.chan_begin, S.nchan * (uint32_t)sizeof(ChanDesc),
                          &bars[buf]);
            bulk_copy_g2s(B + S.addr_off, J.addr + (size_t)S.chan_begin * BD,
                          S.nchan * BD * (uint32_t)sizeof(uint16_t), &bars[buf]);
        }
        __syncwarp();
        for (uint32_t i = lane; i < S.nchan; i += 32) {
            const ChanDesc cd = J.chans[S.chan_begin + i];
            const uint8_t* src = J.xt + (int64_t)cd.c * J.xt_pitch + t0 + cd.goff;
            bulk_copy_g2s(B + cd.offB, src, align16(4 * cd.nwords + 4), &bars[buf]);
        }
    };

    const int nst = T.nstages;
    if (warp == 0) issue(0, 0);
    // stage s waits on barrier s & 1 for its (s >> 1)-th phase
    for (int s = 0; s < nst; ++s) {
        const int buf = s & 1;
        const uint32_t par = (uint32_t)(s >> 1) & 1u;
        const bool ok = mbar_wait_bounded(&bars[buf], par, timeout_ns);
        if (__syncthreads_or(!ok)) {
            // a staging copy never completed: record it, give the copy one more
            // bounded wait so no write lands after the block is gone, and leave
            if (tid == 0) {
                latch_status(status, HP_ERR_TIMEOUT);
                mbar_wait_bounded(&bars[buf], par, timeout_ns);
            }
            __syncthreads();
            return;
        }
        uint8_t* B = smem + buf * stage_bytes;
        const StageDesc S = J.stages[T.stage_begin + s];
        const ChanDesc* cds = reinterpret_cast<const ChanDesc*>(B);

        // byte-shifted copies 1..3 of every staged row
        for (uint32_t i = 0; i < S.nchan; ++i) {
            const ChanDesc cd = cds[i];
            const uint32_t* Bw = reinterpret_cast<const uint32_t*>(B + cd.offB);
            uint32_t* V = reinterpret_cast<uint32_t*>(B + cd.offB + align16(4 * cd.nwords + 4));
            const uint32_t nw = cd.nwords;
            for (uint32_t q = tid; q < nw; q += NT) {
                const uint32_t a = Bw[q], b = Bw[q + 1];
                V[q] = __byte_perm(a, b, 0x4321);
                V[q + nw] = __byte_perm(a, b, 0x5432);
                V[q + 2 * nw] = __byte_perm(a, b, 0x6543);
            }
        }
        __syncthreads();
        if (warp == 0 && s + 1 < nst) issue(s + 1, buf ^ 1);

        const uint16_t* addr = reinterpret_cast<const uint16_t*>(B + S.addr_off) + wd * RD;
        const uint32_t* W = reinterpret_cast<const uint32_t*>(B) + lane + wt * 32 * NW;
        uint32_t i = 0;
        for (; i + 1 < S.nchan; i += 2) {
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint32_t a0 = addr[i * BD + r];
                const uint32_t a1 = addr[(i + 1) * BD + r];
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const uint32_t w0 = W[a0 + 32 * k];
                    const uint32_t w1 = W[a1 + 32 * k];
                    acc_lo[r][k] += __byte_perm(w0, 0, 0x4240) + __byte_perm(w1, 0, 0x4240);
                    acc_hi[r][k] += __byte_perm(w0, 0, 0x4341) + __byte_perm(w1, 0, 0x4341);
                }
            }
        }
        if (i < S.nchan) {
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint32_t a0 = addr[i * BD + r];
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const uint32_t w0 = W[a0 + 32 * k];
                    acc_lo[r][k] += __byte_perm(w0, 0, 0x4240);
                    acc_hi[r][k] += __byte_perm(w0, 0, 0x4341);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RD; ++r)
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                sum[r][k][0] += acc_lo[r][k] & 0xFFFFu;
                sum[r][k][2] += acc_lo[r][k] >> 16;
                sum[r][k][1] += acc_hi[r][k] & 0xFFFFu;
                sum[r][k][3] += acc_hi[r][k] >> 16;
                acc_lo[r][k] = 0;
                acc_hi[r][k] = 0;
            }
        fence_proxy_async_smem();
        __syncthreads();
    }

#pragma unroll
    for (int r = 0; r < RD; ++r) {
        const int dl = wd * RD + r;
        if (dl >= T.nd) continue;
        int32_t* row = J.out + (int64_t)(T.d0 + dl) * J.out_pitch;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int64_t t = t0 + 4 * (lane + 32 * k) + wt * 128 * NW;
            if (t + 3 < J.nout) {
                *reinterpret_cast<int4*>(row + t) =
                    make_int4((int)sum[r][k][0], (int)sum[r][k][1], (int)sum[r][k][2],
                              (int)sum[r][k][3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (t + e < J.nout) row[t + e] = (int)sum[r][k][e];
            }
        }
    }
}

template <int RD, int NW, int WD, int WT>
cudaError_t run_dedisp(const DedispBatch& b, int stage_bytes, int* status, uint64_t timeout_ns,
                       cudaStream_t s) {
    const int64_t total = b.prefix[b.njobs];
    if (total <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)stage_bytes + 16;
    auto k = dedisp_kernel<RD, NW, WD, WT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)total, 256, smem, s>>>(b, stage_bytes, status, timeout_ns);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transpose(const uint8_t* x, int64_t nsamps, int nchans, uint8_t* xt,
                             int64_t xt_pitch, cudaStream_t s) {
    const int vec = ((nchans & 15) == 0) && (((uintptr_t)x & 15u) == 0);
    dim3 grid((unsigned)((xt_pitch + kTT - 1) / kTT), (unsigned)((nchans + kTT - 1) / kTT));
    transpose_kernel<<<grid, 256, 0, s>>>(x, nsamps, nchans, vec, xt, xt_pitch);
    return cudaGetLastError();
}

cudaError_t launch_dedisp(int cfg, const DedispBatch& b, int* status, uint64_t timeout_ns,
                          cudaStream_t s) {
    const int sb = kDedispConfigs[cfg].stage_bytes;
    switch (cfg) {
        case 0: return run_dedisp<2, 4, 8, 1>(b, sb, status, timeout_ns, s);
        case 1: return run_dedisp<4, 2, 8, 1>(b, sb, status, timeout_ns, s);
        case 2: return run_dedisp<2, 4, 4, 2>(b, sb, status, timeout_ns, s);
        case 3: return run_dedisp<4, 4, 8, 1>(b, sb, status, timeout_ns, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hp
