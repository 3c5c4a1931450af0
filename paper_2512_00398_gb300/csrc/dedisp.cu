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
    {2, 4, 8, 1, 36 * 1024},    // 256 threads, BD 16, BT 512, 2 blocks per SM
    {2, 4, 16, 1, 72 * 1024},   // 512 threads, BD 32, BT 512, 1 block per SM
    {4, 2, 8, 1, 36 * 1024},    // 256 threads, BD 32, BT 256, 2 blocks per SM
    {2, 4, 8, 2, 72 * 1024},    // 512 threads, BD 16, BT 1024, 1 block per SM
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


// 32-bit shared-memory accesses on shared-window addresses.
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z),
                 "r"(w)
                 : "memory");
}

template <int RD, int NW, int WD, int WT>
__global__ void __launch_bounds__(32 * WD * WT, (WD * WT <= 8) ? 2 : 1)
dedisp_kernel(const __grid_constant__ DedispBatch batch, int stage_bytes, int* status,
              uint64_t timeout_ns) {
    constexpr int BD = WD * RD;
    constexpr int NT = 32 * WD * WT;
    constexpr int BT = WT * NW * 128;
    constexpr int NB = kDedispStages;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NB * stage_bytes);
    const uint32_t sbase = smem_u32(smem);

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
#pragma unroll
        for (int b = 0; b < NB; ++b) mbar_init(&bars[b], 1);
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

    // warp 0: stage s's channel descriptors, address table and rows -> buffer s % NB
    auto issue = [&](int s) {
        const int buf = s % NB;
        const StageDesc S = J.stages[T.stage_begin + s];
        uint8_t* B = smem + buf * stage_bytes;
        if (lane == 0) {
            mbar_arrive_expect_tx(&bars[buf], S.tx_bytes);
            bulk_copy_g2s(B, J.chans + S.chan_begin, S.nchan * (uint32_t)sizeof(ChanDesc),
                          &bars[buf]);
            bulk_copy_g2s(B + S.addr_off, J.addr + S.addr_begin, S.addr_bytes, &bars[buf]);
        }
        __syncwarp();
        for (uint32_t i = lane; i < S.nchan; i += 32) {
            const ChanDesc cd = J.chans[S.chan_begin + i];
            const uint8_t* src = J.xt + (int64_t)cd.c * J.xt_pitch + t0 + cd.goff;
            bulk_copy_g2s(B + cd.offB, src, 4 * cd.nwords + 16, &bars[buf]);
        }
    };
    auto wait = [&](int s) {
        return mbar_wait_bounded(&bars[s % NB], (uint32_t)(s / NB) & 1u, timeout_ns);
    };
    // all threads: byte-shifted copies 1..3 of every row of stage s.  Row
    // copies and word counts are multiples of 16 bytes / 4 words, so each lane
    // turns 4 words (plus its neighbour's first word) into 4 words of each copy
    // with 16-byte loads and stores.
    auto build = [&](int s) {
        constexpr uint32_t NWARP = NT / 32;
        const uint32_t B = sbase + (uint32_t)((s % NB) * stage_bytes);
        const uint32_t nchan = J.stages[T.stage_begin + s].nchan;
        // 128-word segments of all rows, dealt round-robin to the warps
        uint32_t seg0 = 0;
        for (uint32_t i = 0; i < nchan; ++i) {
            const uint4 cd = lds128(B + 16 * i);          // {c, goff, offB, nwords}
            const uint32_t row = B + cd.z, nw = cd.w;
            const uint32_t nseg = (nw + 127) / 128;
            const uint32_t v1 = row + 4 * nw + 16;        // = row + align16(4 nw + 4)
            uint32_t sg = ((uint32_t)warp + NWARP - seg0 % NWARP) % NWARP;
            for (; sg < nseg; sg += NWARP) {
                const uint32_t q = 128u * sg + 4u * (uint32_t)lane;
                // words q..q+3; q <= nw stays inside the row copy (4 nw + 16 bytes)
                const uint4 w = q <= nw ? lds128(row + 4 * q) : make_uint4(0, 0, 0, 0);
                uint32_t w4 = __shfl_down_sync(0xffffffffu, w.x, 1);
                if (lane == 31 && q < nw) w4 = lds32(row + 4 * q + 16);
                if (q < nw) {
                    sts128(v1 + 4 * q, __byte_perm(w.x, w.y, 0x4321), __byte_perm(w.y, w.z, 0x4321),
                           __byte_perm(w.z, w.w, 0x4321), __byte_perm(w.w, w4, 0x4321));
                    sts128(v1 + 4 * (q + nw), __byte_perm(w.x, w.y, 0x5432),
                           __byte_perm(w.y, w.z, 0x5432), __byte_perm(w.z, w.w, 0x5432),
                           __byte_perm(w.w, w4, 0x5432));
                    sts128(v1 + 4 * (q + 2 * nw), __byte_perm(w.x, w.y, 0x6543),
                           __byte_perm(w.y, w.z, 0x6543), __byte_perm(w.z, w.w, 0x6543),
                           __byte_perm(w.w, w4, 0x6543));
                }
            }
            seg0 += nseg;
        }
    };
    // a staging copy never completed: record it, give every stage still in
    // flight (first .. last) one more bounded wait so no copy lands after the
    // block has left, then leave
    auto abort_stages = [&](int first, int last) {
        if (tid == 0) {
            latch_status(status, HP_ERR_TIMEOUT);
            for (int x = first; x <= last; ++x) wait(x);
        }
        __syncthreads();
    };

    const int nst = T.nstages;
    if (warp == 0) {
        issue(0);
        if (nst > 1) issue(1);
    }
    bool ok = wait(0);
    if (ok) build(0);
    if (__syncthreads_or(!ok)) { abort_stages(0, nst > 1 ? 1 : 0); return; }

    for (int s = 0; s < nst; ++s) {
        const uint32_t B = sbase + (uint32_t)((s % NB) * stage_bytes);
        const StageDesc S = J.stages[T.stage_begin + s];
        const uint32_t tbase = B + 4u * (uint32_t)(lane + wt * 32 * NW);
        const uint32_t tab = B + S.addr_off + (uint32_t)(wd * RD * 8);
        const uint32_t npair = S.nchan >> 1;
        for (uint32_t pr = 0; pr < npair; ++pr) {
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint2 ad = lds64(tab + pr * (BD * 8) + r * 8);
                const uint32_t a0 = tbase + ad.x, a1 = tbase + ad.y;
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const uint32_t w0 = lds32(a0 + 128 * k);
                    const uint32_t w1 = lds32(a1 + 128 * k);
                    acc_lo[r][k] += __byte_perm(w0, 0, 0x4240) + __byte_perm(w1, 0, 0x4240);
                    acc_hi[r][k] += __byte_perm(w0, 0, 0x4341) + __byte_perm(w1, 0, 0x4341);
                }
            }
        }
        if (S.nchan & 1u) {
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint32_t a0 = tbase + lds32(tab + npair * (BD * 8) + r * 8);
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const uint32_t w0 = lds32(a0 + 128 * k);
                    acc_lo[r][k] += __byte_perm(w0, 0, 0x4240);
                    acc_hi[r][k] += __byte_perm(w0, 0, 0x4341);
                }
            }
        }
        // the next stage's copies were issued two stages ago: wait and build them
        // while the 16-bit lanes are flushed
        ok = true;
        if (s + 1 < nst) {
            ok = wait(s + 1);
            if (ok) build(s + 1);
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
        if (__syncthreads_or(!ok)) { abort_stages(s + 1, s + 1); return; }
        // buffer (s + 2) % NB last held stage s - 1, which every thread has finished
        if (warp == 0 && s + 2 < nst) issue(s + 2);
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
    const size_t smem = (size_t)kDedispStages * stage_bytes + 64;
    auto k = dedisp_kernel<RD, NW, WD, WT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)total, 32 * WD * WT, smem, s>>>(b, stage_bytes, status, timeout_ns);
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
        case 1: return run_dedisp<2, 4, 16, 1>(b, sb, status, timeout_ns, s);
        case 2: return run_dedisp<4, 2, 8, 1>(b, sb, status, timeout_ns, s);
        case 3: return run_dedisp<2, 4, 8, 2>(b, sb, status, timeout_ns, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hp
