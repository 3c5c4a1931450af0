// dedisp.cu -- incoherent dedispersion on sm_103a (Section II-B, "Incoherent
// Dedispersion"): D[d][t] = sum_c x[t + delay(c,d)][c], exact integers.
//
//  * transpose_kernel: time-major uint8 [nsamps][nchans] -> channel-major
//    [nchans][xt_pitch], zero padded, so that every channel row is a
//    contiguous byte stream a bulk copy can stage.
//  * dedisp_rows_kernel: one block per (DM tile, time tile).  One producer
//    warp stages byte-row windows of the tile's channels into a ring of
//    shared-memory buffers with cp.async.bulk (TMA, completion on an
//    mbarrier); consumer warps align each row to a trial's byte offset in
//    registers (one PRMT per 4-sample word) and sum the bytes exactly in
//    16-bit lanes (SIMD within a register), flushed into int32 sums before a
//    lane could exceed 16 bits.  Its SEG instance writes per-segment partial
//    sums for the sub-band variant's first stage.
//    No tensor cores: the sum is not a dense contraction.
#include <cstring>

#include "common.cuh"

namespace hp {

// {RD, NW, WD, WT, stage bytes, stage buffers, unroll}: RD trials x NW words
// (4 samples each) per lane, WD x WT consumer warps + 1 producer warp, BD = WD RD
// trials and BT = WT NW 128 samples per block.
const DedispConfig kDedispConfigs[kNumDedispConfigs] = {
    {2, 5, 8, 2, 36 * 1024, 6, 1},   //  0: 16+1 warps, BD 16, BT 1280
    {2, 5, 16, 1, 36 * 1024, 6, 1},  //  1: 16+1 warps, BD 32, BT 640
    {2, 3, 8, 2, 36 * 1024, 6, 1},   //  2: 16+1 warps, BD 16, BT 768
    {4, 3, 8, 2, 36 * 1024, 6, 1},   //  3: 16+1 warps, BD 32, BT 768
    {2, 7, 12, 1, 36 * 1024, 6, 1},  //  4: 12+1 warps, BD 24, BT 896
    {2, 7, 6, 2, 36 * 1024, 6, 1},   //  5: 12+1 warps, BD 12, BT 1792
    {2, 5, 12, 1, 36 * 1024, 6, 1},  //  6: 12+1 warps, BD 24, BT 640
    {2, 5, 8, 2, 54 * 1024, 4, 1},   //  7: 16+1 warps, BD 16, BT 1280, 4 x 54 KB
    {2, 5, 8, 2, 27 * 1024, 8, 1},   //  8: 16+1 warps, BD 16, BT 1280, 8 x 27 KB
    {2, 5, 8, 2, 72 * 1024, 3, 1},   //  9: 16+1 warps, BD 16, BT 1280, 3 x 72 KB
    {2, 7, 12, 1, 54 * 1024, 4, 1},  // 10: 12+1 warps, BD 24, BT 896, 4 x 54 KB
    {2, 5, 12, 1, 54 * 1024, 4, 1},  // 11: 12+1 warps, BD 24, BT 640, 4 x 54 KB
    {2, 7, 12, 1, 54 * 1024, 4, 2},  // 12: as 10, channel-pair loop unrolled twice
    {2, 5, 8, 2, 72 * 1024, 3, 2},   // 13: as 9, channel-pair loop unrolled twice
    {1, 7, 24, 1, 54 * 1024, 4, 2},  // 14: 24+1 warps, 1 trial per warp, BD 24, BT 896
    {1, 5, 30, 1, 54 * 1024, 4, 2},  // 15: 30+1 warps, 1 trial per warp, BD 30, BT 640
    {1, 7, 16, 1, 54 * 1024, 4, 2},  // 16: 16+1 warps, 1 trial per warp, BD 16, BT 896
    // one trial per warp over 17 words (68 samples) per lane: 18 loads per 17
    // words and the table entry and loop overhead spread over twice the words
    {1, 17, 15, 1, 72 * 1024, 3, 1},   // 17: 15+1 warps, BD 15, BT 2176, 3 x 72 KB (default)
    {1, 17, 15, 1, 108 * 1024, 2, 1},  // 18: as 17, 2 x 108 KB
    {1, 19, 11, 1, 72 * 1024, 3, 1},   // 19: 11+1 warps, BD 11, BT 2432
};

namespace {

constexpr int kTC = 128;   // channels per transpose tile (whole 128-byte lines of a row)
constexpr int kTS = 256;   // samples per transpose tile

// One 256 x 128 byte tile of the transpose: rows t0.., channels c0.. of x
// [nsamps][nch] -> xt [nch][pitch] (zero beyond nsamps).  With ring_len > 0
// row t is absolute sample a0 + t of a ring of ring_slots slots of ring_len
// rows (a streamed beam's recent gulps).  Reading, eight lanes take one row's
// 128 bytes (each thread has eight 16-byte loads in flight); writing, the lanes
// of a warp take 32 consecutive channels and write 16 samples of each per
// step, half of the warps the even and half the odd 16-sample pieces.
__device__ __forceinline__ void transpose_tile(const uint8_t* __restrict__ x, int64_t nsamps,
                                               int nch, int vec, uint8_t* __restrict__ xt,
                                               int64_t pitch, int64_t t0, int c0,
                                               int64_t ring_len = 0, int64_t a0 = 0,
                                               int ring_slots = 1) {
    __shared__ __align__(16) uint8_t tile[kTS][kTC + 16];
    const int tid = threadIdx.x;
    {
        constexpr int kSegs = kTC / 16, kRowsPer = 256 / kSegs;
        const int seg = tid % kSegs;
        uint4 q[kTS / kRowsPer];
#pragma unroll
        for (int r = 0; r < kTS / kRowsPer; ++r) {
            const int row = tid / kSegs + kRowsPer * r;
            const int64_t t = t0 + row;
            const int c = c0 + seg * 16;
            q[r] = make_uint4(0, 0, 0, 0);
            if (t < nsamps) {
                int64_t rr = t;
                if (ring_len > 0) {
                    const int64_t a = a0 + t;
                    rr = (a / ring_len) % ring_slots * ring_len + a % ring_len;
                }
                const uint8_t* xr = x + rr * nch;
                if (vec && c + 16 <= nch) {
                    q[r] = __ldg(reinterpret_cast<const uint4*>(xr + c));
                } else {
                    uint8_t v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = (c + i < nch) ? xr[c + i] : 0;
                    memcpy(&q[r], v, 16);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kTS / kRowsPer; ++r)
            *reinterpret_cast<uint4*>(&tile[tid / kSegs + kRowsPer * r][seg * 16]) = q[r];
    }
    __syncthreads();
    {
        const int warp = tid >> 5;
        const int cr = (warp % (kTC / 32)) * 32 + (tid & 31);
        const int half = warp / (kTC / 32);               // even or odd pieces
        const int c = c0 + cr;
#pragma unroll
        for (int k = 0; k < kTS / 32; ++k) {
            const int row0 = (2 * k + half) * 16;
            const int64_t t = t0 + row0;
            if (c < nch && t < pitch) {
                uint8_t v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = tile[row0 + i][cr];
                uint4 q;
                memcpy(&q, v, 16);
                *reinterpret_cast<uint4*>(xt + (int64_t)c * pitch + t) = q;
            }
        }
    }
}

__global__ void __launch_bounds__(256) transpose_kernel(const uint8_t* __restrict__ x,
                                                        int64_t nsamps, int nch, int vec,
                                                        uint8_t* __restrict__ xt, int64_t pitch) {
    transpose_tile(x, nsamps, nch, vec, xt, pitch, (int64_t)blockIdx.x * kTS, blockIdx.y * kTC);
}

// Every file of a batch in one launch: block b handles tile b - prefix[j] of file j.
__global__ void __launch_bounds__(256) transpose_batch_kernel(const __grid_constant__ TransposeBatch tb) {
    const int64_t blk = blockIdx.x;
    int j = 0;
    while (j + 1 < tb.njobs && tb.prefix[j + 1] <= blk) ++j;
    const TransposeJob& J = tb.jobs[j];
    const int64_t item = blk - tb.prefix[j];
    const int64_t tt = item % J.ttiles;
    const int ct = (int)(item / J.ttiles);
    transpose_tile(J.x, J.nsamps, J.nch, J.vec, J.xt, J.pitch, tt * kTS, ct * kTC, J.ring_len,
                   J.a0, J.ring_slots);
}

// 32-bit shared-memory accesses on shared-window addresses.
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
// dedisp_rows_kernel: byte rows only in shared memory, aligned in registers.
// One producer warp only issues bulk copies into a ring of NB stage buffers
// (barriers full[b] / empty[b]); 32*WD*WT consumer warps each own RD trials and
// NW consecutive words (4 samples each) per lane.  A lane loads its NW + 1
// words of a channel row (NW odd, so the lanes of a warp hit 32 distinct
// banks) and aligns them to the trial's byte offset with one PRMT, giving the
// word v = b0 + 2^8 b1 + 2^16 b2 + 2^24 b3 of its four samples.  Over at most
// 256 channels the lane keeps two sums per word:
//   A = sum v (mod 2^32)   and   H = sum (b1 + 2^16 b3)   (PRMT with zeros);
// H is exact (each 16-bit field <= 256 * 255 < 2^16), and so is
//   A - 2^8 H = sum b0 + 2^16 sum b2   (mod 2^32, both fields < 2^16),
// so the four per-sample sums come back at the flush: two PRMTs per word
// (align, odd bytes) instead of three (align, then both 16-bit lanes).  The
// adds are IMADs by a runtime 1, which keeps them on the FMA pipe while the
// PRMTs use the ALU pipe.  No block-wide barrier after set-up; every wait is
// bounded.
constexpr int kTimeGroup = 16;   // time tiles per block group (byte-row kernel)

__device__ __forceinline__ uint32_t imad_add(uint32_t acc, uint32_t x, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(one), "r"(acc));
    return r;
}

// SEG: the tile's stages form segments (sub-band stage 1); the sums are
// written to rows seg_row + trial after the last stage of each segment.
template <int RD, int NW, int WD, int WT, int NB, int UNR = 1, bool SEG = false, bool LV = false>
__global__ void __launch_bounds__(32 * (WD * WT + 1), 1)
dedisp_rows_kernel(const __grid_constant__ DedispBatch batch, int stage_bytes, int* status,
                   uint64_t timeout_ns, uint32_t one) {
    constexpr int BD = WD * RD;
    constexpr int NCW = WD * WT;                 // consumer warps
    constexpr int BT = WT * NW * 128;
    static_assert(NW % 2 == 1, "an odd word count per lane keeps row loads conflict-free");
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NB * stage_bytes);
    uint64_t* empty = full + NB;
    __shared__ int abort_flag;
    __shared__ int done_warps;   // LV: consumer warps that consumed every stage
    const uint32_t sbase = smem_u32(smem);

    const int64_t blk = blockIdx.x;
    int jb = 0;
    while (jb + 1 < batch.njobs && batch.prefix[jb + 1] <= blk) ++jb;
    const DedispJob& J = batch.jobs[jb];
    const int64_t item = blk - batch.prefix[jb];
    // Blocks in groups of kTimeGroup time tiles, every DM tile of a group before
    // the next group: the blocks resident together read neighbouring windows of
    // the same channel rows, which L2 then serves (DM-tile-major order re-reads
    // the whole input from DRAM once per DM tile).
    // (half as many of the long tiles of 2048 samples and more, so that a group's
    // row windows still fit in L2)
    constexpr int TG = BT >= 2048 ? kTimeGroup / 2 : kTimeGroup;
    const int64_t per = (int64_t)TG * J.ndt;
    const int64_t grp = item / per;
    const int64_t rem = item - grp * per;
    const int64_t gsz = min((int64_t)TG, (int64_t)J.ntt - grp * TG);
    const int dt = (int)(rem / gsz);
    const int tt = (int)(grp * TG + rem % gsz);
    const TileDesc T = J.tiles[dt];
    const int64_t t0 = (int64_t)tt * BT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nst = T.nstages;

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], NCW);
        }
        mbar_fence_init();
        abort_flag = 0;
        done_warps = 0;
    }
    __syncthreads();
    volatile int* abort = &abort_flag;

    if (warp == NCW) {
        // ------------------------------------------------------- producer
        int issued = 0, used = 0;
        for (int s = 0; s < nst; ++s) {
            // q: the ring position (SEG: stages of segments this time tile does not
            // need are skipped by the producer and the consumers alike)
            int q = s;
            if constexpr (SEG) {
                if (t0 >= J.nout - (int64_t)(J.stages[T.stage_begin + s].seg_info >> 1)) continue;
                q = used++;
            }
            const int b = q % NB;
            if (q >= NB &&
                !__all_sync(0xffffffffu, mbar_wait_or_abort(&empty[b], (uint32_t)(q / NB - 1) & 1u,
                                                            timeout_ns, abort)))
                break;
            const StageDesc S = J.stages[T.stage_begin + s];
            uint8_t* B = smem + b * stage_bytes;
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[b], S.tx_bytes);
                bulk_copy_g2s(B, J.chans + S.chan_begin, S.nchan * (uint32_t)sizeof(ChanDesc),
                              &full[b]);
                bulk_copy_g2s(B + S.addr_off, J.addr + S.addr_begin, S.addr_bytes, &full[b]);
            }
            __syncwarp();
            for (uint32_t i = lane; i < S.nchan; i += 32) {
                const ChanDesc cd = J.chans[S.chan_begin + i];
                const uint8_t* src = J.xt + (int64_t)cd.c * J.xt_pitch + t0 + cd.goff;
                bulk_copy_g2s(B + cd.offB, src, 4 * cd.nwords, &full[b]);
            }
            issued = q + 1;
        }
        if (lane == 0 && *abort) {
            latch_status(status, HP_ERR_TIMEOUT);
            // only the last NB issued stages can still be in flight
            for (int x = issued - NB > 0 ? issued - NB : 0; x < issued; ++x)
                mbar_wait_bounded(&full[x % NB], (uint32_t)(x / NB) & 1u, timeout_ns);
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    const int wd = warp % WD, wt = warp / WD;
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
    // byte offset of this lane's first word inside a staged row
    const uint32_t lane_off = 4u * (uint32_t)(wt * 32 * NW + NW * lane);
    // the sums of trial dl go to row row0 + dl (samples t < nout)
    auto write_rows = [&](int64_t row0) {
#pragma unroll
        for (int r = 0; r < RD; ++r) {
            const int dl = wd * RD + r;
            if (dl >= T.nd) continue;
            int32_t* row = J.out + (row0 + dl) * J.out_pitch;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const int64_t t = t0 + wt * 128 * NW + 4 * (NW * lane + k);
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
    };
    uint32_t held = 0;
    int used = 0;
    for (int s = 0; s < nst; ++s) {
        int q = s;
        if constexpr (SEG) {
            if (t0 >= J.nout - (int64_t)(J.stages[T.stage_begin + s].seg_info >> 1)) continue;
            q = used++;
        }
        const int b = q % NB;
        if (!__all_sync(0xffffffffu,
                        mbar_wait_or_abort(&full[b], (uint32_t)(q / NB) & 1u, timeout_ns, abort))) {
            // LV: the epilogue's barrier counts this warp too
            if constexpr (LV) named_barrier_arrive(1, 32 * NCW);
            return;
        }
        const uint32_t B = sbase + (uint32_t)(b * stage_bytes);
        const StageDesc S = J.stages[T.stage_begin + s];
        uint32_t tab = B + S.addr_off + (uint32_t)(wd * RD * 16);
        const uint32_t tb = B + lane_off;
        const uint32_t nchan = S.nchan;
        // one channel of trial r: NW + 1 row words at byte address a, aligned by
        // selector sel; A += v, H += (b1, 0, b3, 0) of v
        auto add_row = [&](int r, uint32_t a, uint32_t sel) {
            uint32_t w[NW + 1];
#pragma unroll
            for (int i = 0; i <= NW; ++i) w[i] = lds32(a + 4 * i);
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const uint32_t v = __byte_perm(w[i], w[i + 1], sel);
                acc_lo[r][i] = imad_add(acc_lo[r][i], v, one);
                acc_hi[r][i] = imad_add(acc_hi[r][i], __byte_perm(v, 0, 0x4341), one);
            }
        };
        // channel pairs: table entry {offset ch0, offset ch1, selector ch0, selector ch1}
#pragma unroll UNR
        for (uint32_t pr = nchan >> 1; pr > 0; --pr, tab += BD * 16) {
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint4 e = lds128(tab + r * 16);
                add_row(r, tb + e.x, e.z);
                add_row(r, tb + e.y, e.w);
            }
        }
        if (nchan & 1) {   // the odd last channel (its pair entry repeats it as ch1)
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint4 e = lds128(tab + r * 16);
                add_row(r, tb + e.x, e.z);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
        held += nchan;
        const bool seg_end = SEG && (S.seg_info & 1u) != 0u;
        const uint32_t next_n = s + 1 < nst ? J.stages[T.stage_begin + s + 1].nchan : 256u;
        if (seg_end || held + next_n > 256u) {
            held = 0;
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    // acc_lo = A, acc_hi = H = (S1, S3); A - 2^8 H = (S0, S2)
                    const uint32_t lo = acc_lo[r][k] - (acc_hi[r][k] << 8);
                    sum[r][k][0] += lo & 0xFFFFu;
                    sum[r][k][2] += lo >> 16;
                    sum[r][k][1] += acc_hi[r][k] & 0xFFFFu;
                    sum[r][k][3] += acc_hi[r][k] >> 16;
                    acc_lo[r][k] = 0;
                    acc_hi[r][k] = 0;
                }
        }
        if (seg_end) {
            write_rows(S.seg_row);
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) sum[r][k][e] = 0;
        }
    }
    if constexpr (!SEG) write_rows(T.d0);
    if constexpr (LV) {
        // Second remedian level of the block's sums.  Every consumer warp comes
        // to this barrier, a warp whose wait gave up by arriving from the stage
        // loop (each wait is bounded); the finished warps then all read the same
        // count and go on only if no warp gave up.
        if (lane == 0) atomicAdd(&done_warps, 1);
        named_barrier_sync(1, 32 * NCW);
        if (*reinterpret_cast<volatile int*>(&done_warps) != NCW) return;
        // The ring is free (every stage consumed, no copy in flight): the sums of
        // trial dl go to row dl of BT samples.  A lane's NW 16-byte pieces lie
        // 16 NW bytes apart from the next lane's (NW odd: no bank conflict).
        int32_t* tile = reinterpret_cast<int32_t*>(smem);
#pragma unroll
        for (int r = 0; r < RD; ++r) {
            int32_t* trow = tile + (wd * RD + r) * BT + wt * 128 * NW;
#pragma unroll
            for (int k = 0; k < NW; ++k)
                *reinterpret_cast<int4*>(trow + 4 * (NW * lane + k)) =
                    make_int4((int)sum[r][k][0], (int)sum[r][k][1], (int)sum[r][k][2],
                              (int)sum[r][k][3]);
        }
        named_barrier_sync(1, 32 * NCW);
        // the 25-sample groups [25 g, 25 g + 25) inside [t0, min(t0 + BT, nout)):
        // median of the five medians of five (threads a group apart read 25 words
        // apart: no bank conflict)
        const int64_t te = min(t0 + (int64_t)BT, J.nout);
        const int64_t g_lo = (t0 + 24) / 25;
        const int ng = (int)max(te / 25 - g_lo, (int64_t)0);
        const int items = T.nd * ng;
        for (int i = tid; i < items; i += 32 * NCW) {
            const int dl = i / ng, g = i - dl * ng;
            const int32_t* v = tile + dl * BT + (int)(25 * (g_lo + g) - t0);
            int32_t m[5];
#pragma unroll
            for (int j = 0; j < 5; ++j)
                m[j] = median5(v[5 * j], v[5 * j + 1], v[5 * j + 2], v[5 * j + 3], v[5 * j + 4]);
            J.lv[(int64_t)(T.d0 + dl) * J.lv_pitch + g_lo + g] = median5(m[0], m[1], m[2], m[3], m[4]);
        }
    }
}

template <int RD, int NW, int WD, int WT, int NB, int UNR = 1, bool SEG = false>
cudaError_t run_dedisp_rows(const DedispBatch& b, int stage_bytes, int* status,
                            uint64_t timeout_ns, cudaStream_t s) {
    const int64_t total = b.prefix[b.njobs];
    if (total <= 0) return cudaSuccess;
    const size_t smem = (size_t)NB * stage_bytes + 2 * NB * 8;
    // the jobs write the second remedian level (all or none; not the segmented
    // stage); its epilogue lays the block's sums over the ring
    const bool lv = b.jobs[0].lv != nullptr;
    for (int j = 0; j < b.njobs; ++j)
        if ((b.jobs[j].lv != nullptr) != lv) return cudaErrorInvalidValue;
    if (lv && (SEG || (size_t)WD * RD * WT * NW * 128 * 4 > (size_t)NB * stage_bytes))
        return cudaErrorInvalidValue;
    auto k = dedisp_rows_kernel<RD, NW, WD, WT, NB, UNR, SEG, false>;
    if constexpr (!SEG)
        if (lv) k = dedisp_rows_kernel<RD, NW, WD, WT, NB, UNR, false, true>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)total, 32 * (WD * WT + 1), smem, s>>>(b, stage_bytes, status, timeout_ns, 1u);
    return cudaGetLastError();
}


}  // namespace

cudaError_t launch_transpose(const uint8_t* x, int64_t nsamps, int nchans, uint8_t* xt,
                             int64_t xt_pitch, cudaStream_t s) {
    const int vec = ((nchans & 15) == 0) && (((uintptr_t)x & 15u) == 0);
    dim3 grid((unsigned)((xt_pitch + kTS - 1) / kTS), (unsigned)((nchans + kTC - 1) / kTC));
    transpose_kernel<<<grid, 256, 0, s>>>(x, nsamps, nchans, vec, xt, xt_pitch);
    return cudaGetLastError();
}

TransposeJob make_transpose_job(const uint8_t* x, int64_t nsamps, int nchans, uint8_t* xt,
                                int64_t xt_pitch) {
    TransposeJob J;
    J.ring_len = 0;
    J.a0 = 0;
    J.ring_slots = 1;
    J.pad2_ = 0;
    J.x = x;
    J.nsamps = nsamps;
    J.nch = nchans;
    J.vec = ((nchans & 15) == 0) && (((uintptr_t)x & 15u) == 0);
    J.xt = xt;
    J.pitch = xt_pitch;
    J.ttiles = (xt_pitch + kTS - 1) / kTS;
    J.ctiles = (nchans + kTC - 1) / kTC;
    return J;
}

cudaError_t launch_transpose_batch(const TransposeBatch& tb, cudaStream_t s) {
    const int64_t total = tb.prefix[tb.njobs];
    if (total <= 0) return cudaSuccess;
    transpose_batch_kernel<<<(unsigned)total, 256, 0, s>>>(tb);
    return cudaGetLastError();
}

cudaError_t launch_dedisp(int cfg, const DedispBatch& b, int* status, uint64_t timeout_ns,
                          cudaStream_t s) {
    if (cfg < 0 || cfg >= kNumDedispConfigs) return cudaErrorInvalidValue;
    const int sb = kDedispConfigs[cfg].stage_bytes;
    switch (cfg) {
        case 0: return run_dedisp_rows<2, 5, 8, 2, 6>(b, sb, status, timeout_ns, s);
        case 1: return run_dedisp_rows<2, 5, 16, 1, 6>(b, sb, status, timeout_ns, s);
        case 2: return run_dedisp_rows<2, 3, 8, 2, 6>(b, sb, status, timeout_ns, s);
        case 3: return run_dedisp_rows<4, 3, 8, 2, 6>(b, sb, status, timeout_ns, s);
        case 4: return run_dedisp_rows<2, 7, 12, 1, 6>(b, sb, status, timeout_ns, s);
        case 5: return run_dedisp_rows<2, 7, 6, 2, 6>(b, sb, status, timeout_ns, s);
        case 6: return run_dedisp_rows<2, 5, 12, 1, 6>(b, sb, status, timeout_ns, s);
        case 7: return run_dedisp_rows<2, 5, 8, 2, 4>(b, sb, status, timeout_ns, s);
        case 8: return run_dedisp_rows<2, 5, 8, 2, 8>(b, sb, status, timeout_ns, s);
        case 9: return run_dedisp_rows<2, 5, 8, 2, 3>(b, sb, status, timeout_ns, s);
        case 10: return run_dedisp_rows<2, 7, 12, 1, 4>(b, sb, status, timeout_ns, s);
        case 11: return run_dedisp_rows<2, 5, 12, 1, 4>(b, sb, status, timeout_ns, s);
        case 12: return run_dedisp_rows<2, 7, 12, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 13: return run_dedisp_rows<2, 5, 8, 2, 3, 2>(b, sb, status, timeout_ns, s);
        case 14: return run_dedisp_rows<1, 7, 24, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 15: return run_dedisp_rows<1, 5, 30, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 16: return run_dedisp_rows<1, 7, 16, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 17: return run_dedisp_rows<1, 17, 15, 1, 3, 1>(b, sb, status, timeout_ns, s);
        case 18: return run_dedisp_rows<1, 17, 15, 1, 2, 1>(b, sb, status, timeout_ns, s);
        case 19: return run_dedisp_rows<1, 19, 11, 1, 3, 1>(b, sb, status, timeout_ns, s);
        default: return cudaErrorInvalidValue;
    }
}

bool segmented_config(int cfg) {
    return cfg == 7 || cfg == 11 || cfg == 12 || cfg == 14;
}

cudaError_t launch_dedisp_segmented(int cfg, const DedispBatch& b, int* status,
                                    uint64_t timeout_ns, cudaStream_t s) {
    if (cfg < 0 || cfg >= kNumDedispConfigs) return cudaErrorInvalidValue;
    const int sb = kDedispConfigs[cfg].stage_bytes;
    switch (cfg) {
        case 7: return run_dedisp_rows<2, 5, 8, 2, 4, 1, true>(b, sb, status, timeout_ns, s);
        case 11: return run_dedisp_rows<2, 5, 12, 1, 4, 1, true>(b, sb, status, timeout_ns, s);
        case 12: return run_dedisp_rows<2, 7, 12, 1, 4, 2, true>(b, sb, status, timeout_ns, s);
        case 14: return run_dedisp_rows<1, 7, 24, 1, 4, 2, true>(b, sb, status, timeout_ns, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hp
