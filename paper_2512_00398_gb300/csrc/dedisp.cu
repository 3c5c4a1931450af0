// dedisp.cu -- incoherent dedispersion on sm_103a (Section II-B, "Incoherent
// Dedispersion"): D[d][t] = sum_c x[t + delay(c,d)][c], exact integers.
//
//  * transpose_kernel: time-major uint8 [nsamps][nchans] -> channel-major
//    [nchans][xt_pitch], zero padded, so that every channel row is a
//    contiguous byte stream a bulk copy can stage.
//  * The sums: one block per (DM tile, time tile); channel rows are staged in
//    shared memory with cp.async.bulk (TMA, completion on an mbarrier); bytes
//    are summed in two 16-bit lanes per 32-bit word (SIMD within a register);
//    at most 256 channels go into a lane before it is flushed into the int32
//    sums, so a lane never exceeds 256 * 255 < 2^16.  Three shared-memory
//    layouts, selected by the tile shape (kDedispConfigs):
//      layout 0 -- three byte-shifted copies of each row, so every read is an
//        aligned word (dedisp_kernel; dedisp_ws_kernel with producer warps);
//      layout 1 -- rows widened to 16-bit samples (dedisp16_kernel);
//      layout 2 -- byte rows only, aligned in registers by PRMT, a ring of
//        stage buffers fed by one producer warp (dedisp_rows_kernel, the
//        default shapes; its SEG instance writes per-segment partial sums for
//        the sub-band variant's first stage).
//    No tensor cores: the sum is not a dense contraction.
#include <cstring>

#include "common.cuh"

namespace hp {

const DedispConfig kDedispConfigs[kNumDedispConfigs] = {
    {2, 4, 8, 1, 36 * 1024, 0, 0}, // 256 threads, BD 16, BT 512, 2 blocks per SM
    {2, 4, 16, 1, 72 * 1024, 0},   // 512 threads, BD 32, BT 512, 1 block per SM
    {4, 2, 8, 1, 36 * 1024, 0},    // 256 threads, BD 32, BT 256, 2 blocks per SM
    {2, 4, 8, 2, 72 * 1024, 0},    // 512 threads, BD 16, BT 1024, 1 block per SM
    {2, 4, 8, 2, 72 * 1024, 2},    // as 3, plus 2 producer warps (warp-specialised)
    {2, 4, 16, 1, 72 * 1024, 2},   // as 1, plus 2 producer warps (warp-specialised)
    {2, 8, 8, 2, 72 * 1024, 0, 1}, // 16-bit layout: 512 threads, BD 16, BT 1024
    {2, 8, 8, 1, 36 * 1024, 0, 1}, // 16-bit layout: 256 threads, BD 16, BT 512, 2 blocks/SM
    {4, 4, 8, 2, 72 * 1024, 0, 1}, // 16-bit layout: 512 threads, BD 32, BT 512
    {2, 8, 16, 1, 72 * 1024, 0, 1},// 16-bit layout: 512 threads, BD 32, BT 512
    {2, 5, 8, 2, 36 * 1024, 1, 2, 6},  // byte rows: 16+1 warps, BD 16, BT 1280, 6 buffers
    {2, 5, 16, 1, 36 * 1024, 1, 2, 6}, // byte rows: 16+1 warps, BD 32, BT 640, 6 buffers
    {2, 3, 8, 2, 36 * 1024, 1, 2, 6},  // byte rows: 16+1 warps, BD 16, BT 768, 6 buffers
    {4, 3, 8, 2, 36 * 1024, 1, 2, 6},  // byte rows: 16+1 warps, BD 32, BT 768, 6 buffers
    {2, 7, 12, 1, 36 * 1024, 1, 2, 6}, // byte rows: 12+1 warps, BD 24, BT 896, 6 buffers
    {2, 7, 6, 2, 36 * 1024, 1, 2, 6},  // byte rows: 12+1 warps, BD 12, BT 1792, 6 buffers
    {2, 5, 12, 1, 36 * 1024, 1, 2, 6}, // byte rows: 12+1 warps, BD 24, BT 640, 6 buffers
    {2, 5, 8, 2, 54 * 1024, 1, 2, 4},  // byte rows: 16+1 warps, BD 16, BT 1280, 4 x 54 KB
    {2, 5, 8, 2, 27 * 1024, 1, 2, 8},  // byte rows: 16+1 warps, BD 16, BT 1280, 8 x 27 KB
    {2, 5, 8, 2, 72 * 1024, 1, 2, 3},  // byte rows: 16+1 warps, BD 16, BT 1280, 3 x 72 KB
    {2, 7, 12, 1, 54 * 1024, 1, 2, 4}, // byte rows: 12+1 warps, BD 24, BT 896, 4 x 54 KB
    {2, 5, 12, 1, 54 * 1024, 1, 2, 4}, // byte rows: 12+1 warps, BD 24, BT 640, 4 x 54 KB
    {2, 7, 12, 1, 54 * 1024, 1, 2, 4}, // as 20, channel-pair loop unrolled twice
    {2, 5, 8, 2, 72 * 1024, 1, 2, 3},  // as 19, channel-pair loop unrolled twice
    {1, 7, 24, 1, 54 * 1024, 1, 2, 4}, // 24+1 warps, 1 trial per warp, BD 24, BT 896
    {1, 5, 30, 1, 54 * 1024, 1, 2, 4}, // 30+1 warps, 1 trial per warp, BD 30, BT 640
    {1, 7, 16, 1, 54 * 1024, 1, 2, 4}, // 16+1 warps, 1 trial per warp, BD 16, BT 896
};

namespace {

constexpr int kTC = 64;    // channels per transpose tile
constexpr int kTS = 256;   // samples per transpose tile (4 rows of 64 per thread)

// One 256 x 64 byte tile of the transpose: rows t0.., channels c0.. of x
// [nsamps][nch] -> xt [nch][pitch] (zero beyond nsamps).  With ring_len > 0
// row t is absolute sample a0 + t of a ring of ring_slots slots of ring_len
// rows (a streamed beam's recent gulps).  Each thread has four 16-byte loads
// in flight and writes four 16-byte pieces of one channel row.
__device__ __forceinline__ void transpose_tile(const uint8_t* __restrict__ x, int64_t nsamps,
                                               int nch, int vec, uint8_t* __restrict__ xt,
                                               int64_t pitch, int64_t t0, int c0,
                                               int64_t ring_len = 0, int64_t a0 = 0,
                                               int ring_slots = 1) {
    __shared__ __align__(16) uint8_t tile[kTS][kTC + 16];
    const int tid = threadIdx.x;
    const int seg = tid & 3;
    {
        uint4 q[kTS / 64];
#pragma unroll
        for (int r = 0; r < kTS / 64; ++r) {
            const int row = (tid >> 2) + 64 * r;
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
        for (int r = 0; r < kTS / 64; ++r)
            *reinterpret_cast<uint4*>(&tile[(tid >> 2) + 64 * r][seg * 16]) = q[r];
    }
    __syncthreads();
    {
        const int cr = tid >> 2;
        const int c = c0 + cr;
#pragma unroll
        for (int r = 0; r < kTS / 64; ++r) {
            const int row0 = (4 * r + seg) * 16;
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

    uint32_t held = 0;   // channels summed into the 16-bit lanes since the last flush
    for (int s = 0; s < nst; ++s) {
        const uint32_t B = sbase + (uint32_t)((s % NB) * stage_bytes);
        const StageDesc S = J.stages[T.stage_begin + s];
        const uint32_t tbase = B + 4u * (uint32_t)(lane + wt * 32 * NW);
        const uint32_t tab = B + S.addr_off + (uint32_t)(wd * RD * 8);
        const uint32_t npair = S.nchan >> 1;
        // loads are issued in program order (volatile asm), so each pair's words
        // are all requested before any of them is used, and the next pair's
        // address entries are fetched while this pair is summed
        uint2 ad[RD];
#pragma unroll
        for (int r = 0; r < RD; ++r) ad[r] = npair ? lds64(tab + r * 8) : make_uint2(0, 0);
        for (uint32_t pr = 0; pr < npair; ++pr) {
            uint32_t w0[RD][NW], w1[RD][NW];
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    w0[r][k] = lds32(tbase + ad[r].x + 128 * k);
                    w1[r][k] = lds32(tbase + ad[r].y + 128 * k);
                }
            if (pr + 1 < npair) {
#pragma unroll
                for (int r = 0; r < RD; ++r) ad[r] = lds64(tab + (pr + 1) * (BD * 8) + r * 8);
            }
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    acc_lo[r][k] += __byte_perm(w0[r][k], 0, 0x4240) + __byte_perm(w1[r][k], 0, 0x4240);
                    acc_hi[r][k] += __byte_perm(w0[r][k], 0, 0x4341) + __byte_perm(w1[r][k], 0, 0x4341);
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
        // a 16-bit lane holds at most 256 byte sums: flush into the int32 sums
        // only before the next stage could take it past that
        held += S.nchan;
        const uint32_t next_n = s + 1 < nst ? J.stages[T.stage_begin + s + 1].nchan : 256u;
        if (held + next_n > 256u) {
            held = 0;
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

// Warp-specialised variant.  NPW producer warps issue the bulk copies of each
// stage, wait for them (barrier full[b]) and build the shifted row copies, then
// signal ready[b]; 32*WD*WT consumer warps wait for ready[b], accumulate, and
// release the buffer on empty[b].  No block-wide barrier in the main loop.  Every
// wait is bounded; a timeout raises a block-wide abort flag, producers then give
// each issued stage one more bounded wait before leaving.
template <int RD, int NW, int WD, int WT, int NPW>
__global__ void __launch_bounds__(32 * WD * WT + 32 * NPW, 1)
dedisp_ws_kernel(const __grid_constant__ DedispBatch batch, int stage_bytes, int* status,
                 uint64_t timeout_ns) {
    constexpr int BD = WD * RD;
    constexpr int NCW = WD * WT;                 // consumer warps
    constexpr int BT = WT * NW * 128;
    constexpr int NB = kDedispStages;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NB * stage_bytes);
    uint64_t* ready = full + NB;
    uint64_t* empty = ready + NB;
    __shared__ int abort_flag;
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
    const int nst = T.nstages;

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&ready[b], NPW);
            mbar_init(&empty[b], NCW);
        }
        mbar_fence_init();
        abort_flag = 0;
    }
    __syncthreads();
    volatile int* abort = &abort_flag;

    if (warp >= NCW) {
        // ------------------------------------------------------- producers
        const int pw = warp - NCW;
        auto issue = [&](int s) {              // producer warp 0, all lanes
            const int buf = s % NB;
            const StageDesc S = J.stages[T.stage_begin + s];
            uint8_t* B = smem + buf * stage_bytes;
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[buf], S.tx_bytes);
                bulk_copy_g2s(B, J.chans + S.chan_begin, S.nchan * (uint32_t)sizeof(ChanDesc),
                              &full[buf]);
                bulk_copy_g2s(B + S.addr_off, J.addr + S.addr_begin, S.addr_bytes, &full[buf]);
            }
            __syncwarp();
            for (uint32_t i = lane; i < S.nchan; i += 32) {
                const ChanDesc cd = J.chans[S.chan_begin + i];
                const uint8_t* src = J.xt + (int64_t)cd.c * J.xt_pitch + t0 + cd.goff;
                bulk_copy_g2s(B + cd.offB, src, 4 * cd.nwords + 16, &full[buf]);
            }
        };
        int issued = 0, landed = 0;            // stages issued / known complete
        if (pw == 0) {
            for (; issued < NB && issued < nst; ++issued) issue(issued);
        }
        for (int s = 0; s < nst; ++s) {
            const int b = s % NB;
            // every wait decision is made warp-uniform before any warp-collective step
            if (!__all_sync(0xffffffffu,
                            mbar_wait_or_abort(&full[b], (uint32_t)(s / NB) & 1u, timeout_ns, abort)))
                break;
            if (pw == 0) landed = s + 1;
            // shifted copies 1..3 of every row: 128-word segments dealt to producer warps
            const uint32_t B = sbase + (uint32_t)(b * stage_bytes);
            const uint32_t nchan = J.stages[T.stage_begin + s].nchan;
            uint32_t seg0 = 0;
            for (uint32_t i = 0; i < nchan; ++i) {
                const uint4 cd = lds128(B + 16 * i);       // {c, goff, offB, nwords}
                const uint32_t row = B + cd.z, nw = cd.w;
                const uint32_t nseg = (nw + 127) / 128;
                const uint32_t v1 = row + 4 * nw + 16;
                uint32_t sg = ((uint32_t)pw + NPW - seg0 % NPW) % NPW;
                for (; sg < nseg; sg += NPW) {
                    const uint32_t q = 128u * sg + 4u * (uint32_t)lane;
                    const uint4 w = q <= nw ? lds128(row + 4 * q) : make_uint4(0, 0, 0, 0);
                    uint32_t w4 = __shfl_down_sync(0xffffffffu, w.x, 1);
                    if (lane == 31 && q < nw) w4 = lds32(row + 4 * q + 16);
                    if (q < nw) {
                        sts128(v1 + 4 * q, __byte_perm(w.x, w.y, 0x4321),
                               __byte_perm(w.y, w.z, 0x4321), __byte_perm(w.z, w.w, 0x4321),
                               __byte_perm(w.w, w4, 0x4321));
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
            // these generic writes precede later bulk copies into the same buffer
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[b]);
            // refill the buffer of stage s - 1 once the consumers released it
            if (pw == 0 && s >= 1 && issued < nst) {
                const int r = s - 1;
                if (!__all_sync(0xffffffffu, mbar_wait_or_abort(&empty[r % NB], (uint32_t)(r / NB) & 1u,
                                                                 timeout_ns, abort)))
                    break;
                issue(issued);
                ++issued;
            }
        }
        if (pw == 0 && lane == 0 && *abort) {
            latch_status(status, HP_ERR_TIMEOUT);
            // give every issued stage one more bounded wait before leaving
            for (int x = landed; x < issued; ++x)
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
    uint32_t held = 0;
    for (int s = 0; s < nst; ++s) {
        const int b = s % NB;
        if (!__all_sync(0xffffffffu,
                        mbar_wait_or_abort(&ready[b], (uint32_t)(s / NB) & 1u, timeout_ns, abort)))
            return;
        const uint32_t B = sbase + (uint32_t)(b * stage_bytes);
        const StageDesc S = J.stages[T.stage_begin + s];
        const uint32_t tbase = B + 4u * (uint32_t)(lane + wt * 32 * NW);
        const uint32_t tab = B + S.addr_off + (uint32_t)(wd * RD * 8);
        const uint32_t npair = S.nchan >> 1;
        // loads are issued in program order (volatile asm), so each pair's words
        // are all requested before any of them is used, and the next pair's
        // address entries are fetched while this pair is summed
        uint2 ad[RD];
#pragma unroll
        for (int r = 0; r < RD; ++r) ad[r] = npair ? lds64(tab + r * 8) : make_uint2(0, 0);
        for (uint32_t pr = 0; pr < npair; ++pr) {
            uint32_t w0[RD][NW], w1[RD][NW];
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    w0[r][k] = lds32(tbase + ad[r].x + 128 * k);
                    w1[r][k] = lds32(tbase + ad[r].y + 128 * k);
                }
            if (pr + 1 < npair) {
#pragma unroll
                for (int r = 0; r < RD; ++r) ad[r] = lds64(tab + (pr + 1) * (BD * 8) + r * 8);
            }
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    acc_lo[r][k] += __byte_perm(w0[r][k], 0, 0x4240) + __byte_perm(w1[r][k], 0, 0x4240);
                    acc_hi[r][k] += __byte_perm(w0[r][k], 0, 0x4341) + __byte_perm(w1[r][k], 0, 0x4341);
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
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
        held += S.nchan;
        const uint32_t next_n = s + 1 < nst ? J.stages[T.stage_begin + s + 1].nchan : 256u;
        if (held + next_n > 256u) {
            held = 0;
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
        }
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

template <int RD, int NW, int WD, int WT, int NPW>
cudaError_t run_dedisp_ws(const DedispBatch& b, int stage_bytes, int* status,
                          uint64_t timeout_ns, cudaStream_t s) {
    const int64_t total = b.prefix[b.njobs];
    if (total <= 0) return cudaSuccess;
    const size_t smem = (size_t)kDedispStages * stage_bytes + 3 * kDedispStages * 8;
    auto k = dedisp_ws_kernel<RD, NW, WD, WT, NPW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)total, 32 * (WD * WT + NPW), smem, s>>>(b, stage_bytes, status, timeout_ns);
    return cudaGetLastError();
}


// Layout-1 variant: every staged byte row is widened in shared memory into two
// copies of 16-bit samples, one word = samples (2m, 2m+1) ("even") and one word
// = samples (2m+1, 2m+2) ("odd"), so a trial whose offset is rel reads aligned
// words of copy rel & 1.  A word already holds two 16-bit lanes, so summing two
// channels is one three-input add per 4 byte-adds, with no byte splitting; the
// price is 2 shared-memory bytes per add instead of 1.
template <int RD, int NW, int WD, int WT>
__global__ void __launch_bounds__(32 * WD * WT, (WD * WT <= 8) ? 2 : 1)
dedisp16_kernel(const __grid_constant__ DedispBatch batch, int stage_bytes, int* status,
                uint64_t timeout_ns) {
    constexpr int BD = WD * RD;
    constexpr int NT = 32 * WD * WT;
    constexpr int BT = WT * NW * 64;
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

    uint32_t acc[RD][NW];        // two 16-bit lanes: samples 2m, 2m+1
    uint32_t sum[RD][NW][2];
#pragma unroll
    for (int r = 0; r < RD; ++r)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            acc[r][k] = 0;
            sum[r][k][0] = 0;
            sum[r][k][1] = 0;
        }

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
            bulk_copy_g2s(B + cd.offB, src, 2 * cd.nwords + 16, &bars[buf]);
        }
    };
    auto wait = [&](int s) {
        return mbar_wait_bounded(&bars[s % NB], (uint32_t)(s / NB) & 1u, timeout_ns);
    };
    // all threads: widen every byte row into its even and odd 16-bit copies.
    // A lane takes 16 bytes (16 samples) -> 8 even words + 8 odd words; the
    // odd copy's last word needs the next lane's first byte.
    auto build = [&](int s) {
        constexpr uint32_t NWARP = NT / 32;
        const uint32_t B = sbase + (uint32_t)((s % NB) * stage_bytes);
        const uint32_t nchan = J.stages[T.stage_begin + s].nchan;
        uint32_t seg0 = 0;
        for (uint32_t i = 0; i < nchan; ++i) {
            const uint4 cd = lds128(B + 16 * i);          // {c, goff, offB, nwords}
            const uint32_t row = B + cd.z, nw = cd.w;     // nw: words per 16-bit copy
            const uint32_t ev = row + 2 * nw + 16;        // even copy, odd copy follows
            const uint32_t od = ev + 4 * nw;
            const uint32_t nseg = (nw + 255) / 256;       // 256 words of each copy per warp step
            uint32_t sg = ((uint32_t)warp + NWARP - seg0 % NWARP) % NWARP;
            for (; sg < nseg; sg += NWARP) {
                const uint32_t m = 256u * sg + 8u * (uint32_t)lane;   // first word of the lane
                // bytes 2m .. 2m+15; 2m <= nw keeps them inside the row (2 nw + 16 bytes)
                const uint4 w = m <= nw ? lds128(row + 2 * m) : make_uint4(0, 0, 0, 0);
                uint32_t w4 = __shfl_down_sync(0xffffffffu, w.x, 1);
                if (lane == 31 && m < nw) w4 = lds32(row + 2 * m + 16);
                if (m < nw) {
                    const uint32_t e0 = __byte_perm(w.x, 0, 0x4140), e1 = __byte_perm(w.x, 0, 0x4342);
                    const uint32_t e2 = __byte_perm(w.y, 0, 0x4140), e3 = __byte_perm(w.y, 0, 0x4342);
                    const uint32_t e4 = __byte_perm(w.z, 0, 0x4140), e5 = __byte_perm(w.z, 0, 0x4342);
                    const uint32_t e6 = __byte_perm(w.w, 0, 0x4140), e7 = __byte_perm(w.w, 0, 0x4342);
                    const uint32_t e8 = __byte_perm(w4, 0, 0x4140);
                    sts128(ev + 4 * m, e0, e1, e2, e3);
                    sts128(ev + 4 * m + 16, e4, e5, e6, e7);
                    sts128(od + 4 * m, __byte_perm(e0, e1, 0x5432), __byte_perm(e1, e2, 0x5432),
                           __byte_perm(e2, e3, 0x5432), __byte_perm(e3, e4, 0x5432));
                    sts128(od + 4 * m + 16, __byte_perm(e4, e5, 0x5432), __byte_perm(e5, e6, 0x5432),
                           __byte_perm(e6, e7, 0x5432), __byte_perm(e7, e8, 0x5432));
                }
            }
            seg0 += nseg;
        }
    };
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

    uint32_t held = 0;
    for (int s = 0; s < nst; ++s) {
        const uint32_t B = sbase + (uint32_t)((s % NB) * stage_bytes);
        const StageDesc S = J.stages[T.stage_begin + s];
        const uint32_t tbase = B + 4u * (uint32_t)(lane + wt * 32 * NW);
        const uint32_t tab = B + S.addr_off + (uint32_t)(wd * RD * 8);
        const uint32_t npair = S.nchan >> 1;
        // all words of a pair are requested before any is summed (volatile asm
        // keeps program order); the next pair's entries load meanwhile
        uint2 ad[RD];
#pragma unroll
        for (int r = 0; r < RD; ++r) ad[r] = npair ? lds64(tab + r * 8) : make_uint2(0, 0);
        for (uint32_t pr = 0; pr < npair; ++pr) {
            uint32_t w0[RD][NW], w1[RD][NW];
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    w0[r][k] = lds32(tbase + ad[r].x + 128 * k);
                    w1[r][k] = lds32(tbase + ad[r].y + 128 * k);
                }
            if (pr + 1 < npair) {
#pragma unroll
                for (int r = 0; r < RD; ++r) ad[r] = lds64(tab + (pr + 1) * (BD * 8) + r * 8);
            }
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) acc[r][k] += w0[r][k] + w1[r][k];
        }
        if (S.nchan & 1u) {
#pragma unroll
            for (int r = 0; r < RD; ++r) {
                const uint32_t a0 = tbase + lds32(tab + npair * (BD * 8) + r * 8);
#pragma unroll
                for (int k = 0; k < NW; ++k) acc[r][k] += lds32(a0 + 128 * k);
            }
        }
        ok = true;
        if (s + 1 < nst) {
            ok = wait(s + 1);
            if (ok) build(s + 1);
        }
        held += S.nchan;
        const uint32_t next_n = s + 1 < nst ? J.stages[T.stage_begin + s + 1].nchan : 256u;
        if (held + next_n > 256u) {
            held = 0;
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    sum[r][k][0] += acc[r][k] & 0xFFFFu;
                    sum[r][k][1] += acc[r][k] >> 16;
                    acc[r][k] = 0;
                }
        }
        fence_proxy_async_smem();
        if (__syncthreads_or(!ok)) { abort_stages(s + 1, s + 1); return; }
        if (warp == 0 && s + 2 < nst) issue(s + 2);
    }

#pragma unroll
    for (int r = 0; r < RD; ++r) {
        const int dl = wd * RD + r;
        if (dl >= T.nd) continue;
        int32_t* row = J.out + (int64_t)(T.d0 + dl) * J.out_pitch;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int64_t t = t0 + 2 * (lane + 32 * k) + wt * 64 * NW;
            if (t + 1 < J.nout) {
                *reinterpret_cast<int2*>(row + t) = make_int2((int)sum[r][k][0], (int)sum[r][k][1]);
            } else if (t < J.nout) {
                row[t] = (int)sum[r][k][0];
            }
        }
    }
}

template <int RD, int NW, int WD, int WT>
cudaError_t run_dedisp16(const DedispBatch& b, int stage_bytes, int* status, uint64_t timeout_ns,
                         cudaStream_t s) {
    const int64_t total = b.prefix[b.njobs];
    if (total <= 0) return cudaSuccess;
    const size_t smem = (size_t)kDedispStages * stage_bytes + 64;
    auto k = dedisp16_kernel<RD, NW, WD, WT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)total, 32 * WD * WT, smem, s>>>(b, stage_bytes, status, timeout_ns);
    return cudaGetLastError();
}


// Layout-2 kernel: byte rows only in shared memory, aligned in registers.
// One producer warp only issues bulk copies into a ring of NB stage buffers
// (barriers full[b] / empty[b]); 32*WD*WT consumer warps each own RD trials and
// NW consecutive words (4 samples each) per lane.  A lane loads its NW + 1
// words of a channel row (NW odd, so the lanes of a warp hit 32 distinct
// banks), aligns them to the trial's byte offset with one PRMT and splits each
// into two 16-bit lanes with two more; the lanes are summed with IMADs by a
// runtime 1, which keeps the adds on the FMA pipe while the PRMTs use the ALU
// pipe.  No block-wide barrier after set-up; every wait is bounded.
constexpr int kTimeGroup = 16;   // time tiles per block group (byte-row kernel)

__device__ __forceinline__ uint32_t imad_add(uint32_t acc, uint32_t x, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(one), "r"(acc));
    return r;
}

// SEG: the tile's stages form segments (sub-band stage 1); the sums are
// written to rows seg_row + trial after the last stage of each segment.
template <int RD, int NW, int WD, int WT, int NB, int UNR = 1, bool SEG = false>
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
    const int64_t per = (int64_t)kTimeGroup * J.ndt;
    const int64_t grp = item / per;
    const int64_t rem = item - grp * per;
    const int64_t gsz = min((int64_t)kTimeGroup, (int64_t)J.ntt - grp * kTimeGroup);
    const int dt = (int)(rem / gsz);
    const int tt = (int)(grp * kTimeGroup + rem % gsz);
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
                        mbar_wait_or_abort(&full[b], (uint32_t)(q / NB) & 1u, timeout_ns, abort)))
            return;
        const uint32_t B = sbase + (uint32_t)(b * stage_bytes);
        const StageDesc S = J.stages[T.stage_begin + s];
        uint32_t tab = B + S.addr_off + (uint32_t)(wd * RD * 16);
        const uint32_t tb = B + lane_off;
        const uint32_t nchan = S.nchan;
        // one channel of trial r: NW + 1 row words at byte address a, aligned by
        // selector sel and added into the trial's 16-bit lanes
        auto add_row = [&](int r, uint32_t a, uint32_t sel) {
            uint32_t w[NW + 1];
#pragma unroll
            for (int i = 0; i <= NW; ++i) w[i] = lds32(a + 4 * i);
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const uint32_t v = __byte_perm(w[i], w[i + 1], sel);
                acc_lo[r][i] = imad_add(acc_lo[r][i], __byte_perm(v, 0, 0x4240), one);
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
                    sum[r][k][0] += acc_lo[r][k] & 0xFFFFu;
                    sum[r][k][2] += acc_lo[r][k] >> 16;
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
    if (!SEG) write_rows(T.d0);
}

template <int RD, int NW, int WD, int WT, int NB, int UNR = 1, bool SEG = false>
cudaError_t run_dedisp_rows(const DedispBatch& b, int stage_bytes, int* status,
                            uint64_t timeout_ns, cudaStream_t s) {
    const int64_t total = b.prefix[b.njobs];
    if (total <= 0) return cudaSuccess;
    const size_t smem = (size_t)NB * stage_bytes + 2 * NB * 8;
    auto k = dedisp_rows_kernel<RD, NW, WD, WT, NB, UNR, SEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)total, 32 * (WD * WT + 1), smem, s>>>(b, stage_bytes, status, timeout_ns, 1u);
    return cudaGetLastError();
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
    const int sb = kDedispConfigs[cfg].stage_bytes;
    switch (cfg) {
        case 0: return run_dedisp<2, 4, 8, 1>(b, sb, status, timeout_ns, s);
        case 1: return run_dedisp<2, 4, 16, 1>(b, sb, status, timeout_ns, s);
        case 2: return run_dedisp<4, 2, 8, 1>(b, sb, status, timeout_ns, s);
        case 3: return run_dedisp<2, 4, 8, 2>(b, sb, status, timeout_ns, s);
        case 4: return run_dedisp_ws<2, 4, 8, 2, 2>(b, sb, status, timeout_ns, s);
        case 5: return run_dedisp_ws<2, 4, 16, 1, 2>(b, sb, status, timeout_ns, s);
        case 6: return run_dedisp16<2, 8, 8, 2>(b, sb, status, timeout_ns, s);
        case 7: return run_dedisp16<2, 8, 8, 1>(b, sb, status, timeout_ns, s);
        case 8: return run_dedisp16<4, 4, 8, 2>(b, sb, status, timeout_ns, s);
        case 9: return run_dedisp16<2, 8, 16, 1>(b, sb, status, timeout_ns, s);
        case 10: return run_dedisp_rows<2, 5, 8, 2, 6>(b, sb, status, timeout_ns, s);
        case 11: return run_dedisp_rows<2, 5, 16, 1, 6>(b, sb, status, timeout_ns, s);
        case 12: return run_dedisp_rows<2, 3, 8, 2, 6>(b, sb, status, timeout_ns, s);
        case 13: return run_dedisp_rows<4, 3, 8, 2, 6>(b, sb, status, timeout_ns, s);
        case 14: return run_dedisp_rows<2, 7, 12, 1, 6>(b, sb, status, timeout_ns, s);
        case 15: return run_dedisp_rows<2, 7, 6, 2, 6>(b, sb, status, timeout_ns, s);
        case 16: return run_dedisp_rows<2, 5, 12, 1, 6>(b, sb, status, timeout_ns, s);
        case 17: return run_dedisp_rows<2, 5, 8, 2, 4>(b, sb, status, timeout_ns, s);
        case 18: return run_dedisp_rows<2, 5, 8, 2, 8>(b, sb, status, timeout_ns, s);
        case 19: return run_dedisp_rows<2, 5, 8, 2, 3>(b, sb, status, timeout_ns, s);
        case 20: return run_dedisp_rows<2, 7, 12, 1, 4>(b, sb, status, timeout_ns, s);
        case 21: return run_dedisp_rows<2, 5, 12, 1, 4>(b, sb, status, timeout_ns, s);
        case 22: return run_dedisp_rows<2, 7, 12, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 23: return run_dedisp_rows<2, 5, 8, 2, 3, 2>(b, sb, status, timeout_ns, s);
        case 24: return run_dedisp_rows<1, 7, 24, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 25: return run_dedisp_rows<1, 5, 30, 1, 4, 2>(b, sb, status, timeout_ns, s);
        case 26: return run_dedisp_rows<1, 7, 16, 1, 4, 2>(b, sb, status, timeout_ns, s);
        default: return cudaErrorInvalidValue;
    }
}

bool segmented_config(int cfg) { return cfg == 17 || cfg == 21 || cfg == 22 || cfg == 24; }

cudaError_t launch_dedisp_segmented(int cfg, const DedispBatch& b, int* status,
                                    uint64_t timeout_ns, cudaStream_t s) {
    if (cfg < 0 || cfg >= kNumDedispConfigs) return cudaErrorInvalidValue;
    const int sb = kDedispConfigs[cfg].stage_bytes;
    switch (cfg) {
        case 17: return run_dedisp_rows<2, 5, 8, 2, 4, 1, true>(b, sb, status, timeout_ns, s);
        case 21: return run_dedisp_rows<2, 5, 12, 1, 4, 1, true>(b, sb, status, timeout_ns, s);
        case 22: return run_dedisp_rows<2, 7, 12, 1, 4, 2, true>(b, sb, status, timeout_ns, s);
        case 24: return run_dedisp_rows<1, 7, 24, 1, 4, 2, true>(b, sb, status, timeout_ns, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hp
