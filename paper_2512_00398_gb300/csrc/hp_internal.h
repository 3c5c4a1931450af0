// hp_internal.h -- plan object, device table layouts and kernel launchers of
// the search library.  Host code (plan.cpp) and the .cu files share this
// header; nothing here is part of the public C ABI (include/hp.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hp.h"

namespace hp {

// ------------------------------------------------------------------ limits
constexpr int kMaxChans = 65536;
constexpr int kMaxWidths = 32;
constexpr int kMaxWidth = 16384;         // widest boxcar (detect tile halo in shared memory)
constexpr int kMaxDMs = 1 << 20;
constexpr int kStageMaxChans = 256;      // 16-bit lanes hold <= 257 sums of bytes
constexpr int kHistFine = 4096;          // |y| < 4096 binned exactly
constexpr int kHistBins = 8192;          // + 4096 coarse bins of |y| >> 12
constexpr int kDetectTile = 4096;        // boxcar starts per detect block
constexpr int kSortChunk = 2048;         // keys sorted per block before merging
constexpr int kKeyDmShift = 43;          // sort key: dm << 43 | sample << 5 | width
constexpr int kKeySampleShift = 5;
constexpr int64_t kMaxSamples = (int64_t)1 << 38;
constexpr int64_t kMaxMergeGap = 1000000000000000LL;   // |t_gap| bound (1e15 samples)

// ------------------------------------------------------ dedispersion tiles
// Thread tile: RD trials x NW words (4 byte samples each) per lane; WD warps
// along the trial axis, WT along time, plus one producer warp.
struct DedispConfig {
    int RD, NW, WD, WT;
    int stage_bytes;   // shared memory per stage buffer
    int stages;        // stage buffers in the ring
    int unroll;        // channel-pair loop unroll
    int BD() const { return WD * RD; }
    int BT() const { return WT * NW * 128; }
    int threads() const { return 32 * (WD * WT + 1); }
};
constexpr int kNumDedispConfigs = 20;
constexpr int kDefaultDedispConfig = 17;
// stage 1 of the sub-band variant: its tile shape unless one was set
constexpr int kDefaultSubbandConfig = 12;
extern const DedispConfig kDedispConfigs[kNumDedispConfigs];

// One staged channel row of a DM tile (16 bytes, copied into shared memory).
struct ChanDesc {
    uint32_t c;        // channel index
    int32_t goff;      // first input sample of the row relative to the time tile
    uint32_t offB;     // byte offset of the row copy in the stage buffer
    uint32_t nwords;   // 32-bit words per shifted / widened copy
};
static_assert(sizeof(ChanDesc) == 16, "ChanDesc layout");

// One channel stage of a DM tile.  In the stage buffer: nchan channel
// descriptors, then the address table [pair][BD][2] (uint32 byte offsets of
// the first word each trial reads in each channel of a channel pair), then
// the rows with their shifted copies.
struct StageDesc {
    uint32_t chan_begin;  // index into the channel-descriptor array
    uint32_t nchan;
    uint32_t addr_off;    // byte offset of the address table in the buffer
    uint32_t tx_bytes;    // bytes landing in shared memory for this stage
    uint32_t addr_begin;  // index of the stage's table in the address array
    uint32_t addr_bytes;  // table bytes (pairs * BD * 8, layout 2: pairs * BD * 16)
    // Segments (sub-band stage 1, byte-row kernel): the tile's channels are cut
    // into segments that no stage straddles; after the last stage of a segment
    // the block writes its sums to rows seg_row + trial and starts from zero.
    // seg_info: bit 0 = last stage of its segment; bits 1.. = trim: the segment's
    // rows are needed only below nout - trim, so time tiles from there on skip it.
    int32_t seg_row;
    uint32_t seg_info;
};
static_assert(sizeof(StageDesc) == 32, "StageDesc layout");

struct TileDesc {
    int32_t d0, nd;            // first trial, trial count (<= BD)
    int32_t stage_begin, nstages;
};

// Host copy of the tiling of one plan for one config.
struct DedispTiling {
    int cfg = -1;
    int BD = 0, BT = 0;
    std::vector<TileDesc> tiles;
    std::vector<StageDesc> stages;
    std::vector<ChanDesc> chans;
    std::vector<uint32_t> addr;    // per stage [pair][BD][2] byte offsets in the stage buffer
    int64_t max_reach = 0;         // max over rows of goff + row bytes
};

// Device view of one dedispersion job (one filterbank).
struct DedispJob {
    const uint8_t* xt;         // transposed input [nchans][xt_pitch]
    int64_t xt_pitch;
    int32_t* out;              // [ndm][out_pitch]
    int64_t out_pitch;
    int64_t nout;
    int32_t ntt;               // time tiles
    int32_t ndt;               // DM tiles
    const TileDesc* tiles;
    const StageDesc* stages;
    const ChanDesc* chans;
    const uint32_t* addr;
    // Median baseline only: the second remedian level of every trial (the median
    // of the five medians of five consecutive sums of a 25-sample group) for the
    // groups that lie inside one time tile and below nout, formed from the
    // block's sums before it leaves, [ndm][lv_pitch]; null: not written (every
    // job of a launch or none).  The groups that straddle a tile edge or nout are
    // left to the search.
    int32_t* lv;
    int64_t lv_pitch;
};

// Jobs of one dedispersion launch, passed by value as the kernel parameter.
// Block b works on item b - prefix[j] of the job j with prefix[j] <= b < prefix[j+1];
// item i of a job is (DM tile i / ntt, time tile i % ntt).
constexpr int kMaxJobs = 32;
struct DedispBatch {
    int32_t njobs;
    int32_t pad_;
    int64_t prefix[kMaxJobs + 1];
    DedispJob jobs[kMaxJobs];
};

// One file of a batched transpose.
struct TransposeJob {
    // row t of the input is x + t * nch, or with ring_len > 0 the row of
    // absolute sample a = a0 + t in a ring of ring_slots slots of ring_len rows:
    // x + ((a / ring_len) % ring_slots * ring_len + a % ring_len) * nch
    int64_t ring_len, a0;
    int32_t ring_slots, pad2_;
    const uint8_t* x;
    int64_t nsamps;
    int32_t nch, vec;
    uint8_t* xt;
    int64_t pitch;
    int64_t ttiles;            // 256-sample tiles along time (of the padded pitch)
    int32_t ctiles, pad_;      // 64-channel tiles
};
struct TransposeBatch {
    int32_t njobs, pad_;
    int64_t prefix[kMaxJobs + 1];   // tiles of files before j (tiles = ttiles * ctiles)
    TransposeJob jobs[kMaxJobs];
};

// ------------------------------------------------------------- launchers
// All return cudaSuccess or the launch error.
cudaError_t launch_transpose(const uint8_t* x, int64_t nsamps, int nchans, uint8_t* xt,
                             int64_t xt_pitch, cudaStream_t s);
cudaError_t launch_dedisp(int cfg, const DedispBatch& batch, int* status, uint64_t timeout_ns,
                          cudaStream_t s);
// The same tilings run segment by segment (stage 1 of the sub-band variant):
// rows are written at the end of every segment (StageDesc::seg_row / seg_info)
// and time tiles past a segment's needed length skip its stages.
// Byte-row configs for which segmented_config() holds only.
bool segmented_config(int cfg);
cudaError_t launch_dedisp_segmented(int cfg, const DedispBatch& batch, int* status,
                                    uint64_t timeout_ns, cudaStream_t s);

// Stage 2 of the sub-band variant: for the trials d of groups [g_begin, g_end),
// out[d][t] = sum over sub-bands s of B[row(g, s)][t + top[d][s]], t < nout,
// with row(g, s) = ((g / gchunk - c0) * nsub + s) * gchunk + g % gchunk, g = d / G.
// A block takes up to kSubbandTrials trials of one group and one time tile;
// win_cap (int32 per staged window, a multiple of 4) must hold the tile plus
// the largest spread top[d_last][s] - top[d_first][s] of a block, plus 8.
constexpr int kSubbandTrials = 8;
constexpr int kSubbandTile = 2048;       // output samples per block
struct SubbandArgs {
    const int32_t* B;
    int64_t bpitch;            // int32 per row, a multiple of 4
    const int32_t* top;        // [ndm][nsub] delay of each sub-band's first channel
    int32_t nsub, G, gchunk, c0;
    int32_t g_begin, g_end, ndm, win_cap;
    int32_t* out;
    int64_t out_pitch;
    int64_t nout;
    int* status;
    uint64_t timeout_ns;
};
cudaError_t launch_subband_sum(const SubbandArgs& a, cudaStream_t s);
TransposeJob make_transpose_job(const uint8_t* x, int64_t nsamps, int nchans, uint8_t* xt,
                                int64_t xt_pitch);
cudaError_t launch_transpose_batch(const TransposeBatch& tb, cudaStream_t s);

// A run that left the detect tile's halo, to be finished by tail_kernel.
struct TailRec {
    int32_t trial, k;
    int64_t u;        // first boxcar start not yet examined
    int64_t S_prev;   // S at u - 1 (above threshold)
    int64_t best_S, best_t;
};
constexpr int64_t kTailCap = 1 << 20;

// Radix selection of the lower median of |S_k| for one (trial, width): pass
// `level` (0 = done) counts, among the values with v >> shift == prefix, the
// next digit (the first pass: v >> shift, plus an overflow range).
struct WsigState {
    int32_t level, shift;
    int64_t prefix;
    int64_t rank;              // rank of the median among the values still counted
};

struct SearchArgs {
    const int32_t* D;          // [ndm][pitch]
    int64_t pitch, nout;
    int ndm;
    int nw;
    const int32_t* widths;     // device [nw]
    int32_t wmax;
    float thr;
    int baseline_mode;         // 0 median, 1 mean
    int levels;                // remedian levels (median mode)
    int64_t win;               // window in samples (mean mode half width = win/2)
    // second remedian level of D from the dedispersion (levels >= 2), [ndm][lv2_pitch],
    // every group of 25 samples inside one of its lv2_bt-sample time tiles; the
    // groups straddling a tile edge or nout are formed from D here.  Null: the
    // remedian starts from D.
    int32_t* lv2;
    int64_t lv2_pitch, lv2_bt;
    // scratch (device)
    int32_t* lvl_a;            // remedian pass buffers [ndm][lvl_pitch]
    int32_t* lvl_b;
    int64_t lvl_pitch_a, lvl_pitch_b;
    int64_t* mean_pre;         // mean mode block prefix [ndm][mean_pitch]
    int64_t mean_pitch;
    uint32_t* hist;            // [ndm][kHistBins]
    int32_t* refine_bucket;    // [ndm]
    int64_t* refine_rank;      // [ndm]
    int64_t* mad;              // [ndm]
    // [ndm] upper bound of max |y| per trial from its |y| histogram (-1: none
    // known), or null; a trial with ybound * ybound_w < 2^31 - 1 has every
    // boxcar sum in int32 (ybound_w = the widest boxcar of the series y)
    int64_t* ybound;
    int64_t ybound_w;
    double* sigma;             // [ndm]
    int64_t* tint;             // [ndm][nw] integer thresholds
    int32_t* Y;                // [ndm][ypitch] baseline-subtracted series y = D - b, written
    int64_t ypitch;            // by the histogram pass (may alias D in median mode)
    hp_raw_cand* raw;          // output
    int64_t raw_cap;
    int64_t* raw_count;
    TailRec* tails;            // scratch [tail_cap]
    int64_t tail_cap;
    int64_t* tail_count;
    int* status;
    // streamed search (one gulp's buffer): runs are reported only when their
    // first start t < nwin, and not when t == 0 while carry_in[trial][k] is
    // set; carry_out[trial][k] = start nwin - 1 above threshold (carry_in and
    // carry_out are distinct [ndm][nw] arrays, or null).  Reported samples are
    // t + t_offset.  A plain search has nwin = nout, no carries, offset 0.
    int64_t nwin;
    const uint8_t* carry_in;
    uint8_t* carry_out;
    int64_t t_offset;
    // 1: stop after sigma and the integer thresholds (no detection); used for the
    // zero-DM series of the RFI stage
    int stats_only;
    // 1: per-width sigmas (sigma_k = 1.482602218505602 * lower median of |S_k|
    // over every start) replace sigma * sqrt(W) in the thresholds and the S/N
    int width_sigma;
    uint32_t* whist;           // [ndm][nw][2 * 4096] radix-selection counts
    WsigState* wstate;         // [ndm][nw]
    int64_t* wmad;             // [ndm][nw] lower median of |S_k|
    double* sigw;              // [ndm][nw] sigma_k
    // reported samples are t * sample_mul + t_offset (1 but on a scrunched series)
    int64_t sample_mul;
    // decimated boxcars: widths W > decimate that are multiples of it run on the
    // series summed in blocks of q = W / decimate; ndec distinct q (ascending),
    // level l's series at ydec + dec_off[l] with pitch dec_pitch[l], thresholds
    // tint_lv [ndec][ndm][nw], widths widths_lv [ndec][nw] (W / q, or 1)
    int decimate, ndec;
    int32_t dec_q[kMaxWidths];
    int64_t dec_off[kMaxWidths], dec_pitch[kMaxWidths];
    int32_t* ydec;
    int64_t* tint_lv;
    int32_t* widths_lv;
};
cudaError_t launch_search(const SearchArgs& a, cudaStream_t s, int64_t* nlaunch);

// RFI mitigation of one filterbank before dedispersion (rfi.cu).  Works on the
// transposed copy xt [nch][xt_pitch] (cleaned in place); the time-major input
// x [nsamps][nch] is read only for the optional cleaned copy `out`.
struct RfiArgs {
    const uint8_t* x;          // [nsamps][nch]
    uint8_t* xt;               // [nch][xt_pitch], NULL: leave it alone
    int64_t xt_pitch;
    int64_t nsamps;
    int nch;
    int nb_k;                  // narrowband threshold (channel-statistics MADs)
    uint32_t* hist;            // scratch [nch][256]
    int32_t* med;              // [nch] channel medians m_c
    int32_t* spread;           // [nch] channel median |x - m_c|
    uint8_t* chan_flag;        // [round16(nch)] 1 = narrowband channel
    uint8_t* samp_flag;        // [round16(nsamps) + 16] 1 = broadband sample
    int32_t* one;              // device int32 holding 1 (the width list of the z search)
    SearchArgs z;              // statistics of the zero-DM series z (stats_only)
    uint8_t* out;              // optional [nsamps][nch] cleaned copy of x
};
cudaError_t launch_rfi(const RfiArgs& r, cudaStream_t s, int64_t* nlaunch);

struct MergeArgs {
    const hp_raw_cand* raw;
    const int64_t* nraw;
    int64_t cap;               // capacity of raw (== of every scratch array below)
    const double* sigma;       // [ndm]
    const double* sigw;        // [ndm][nw] per-width sigmas, or null (sigma * sqrt(W))
    const int32_t* widths;     // device [nw]
    int nw;
    int32_t wmax;
    int dm_tol;
    int64_t t_gap;
    int w_tol;
    // scratch
    uint64_t* keys[2];
    int64_t* vals[2];
    int32_t* parent;
    uint64_t* best_bits;
    int32_t* rep;
    int32_t* members;
    int32_t* dm_lo;
    int32_t* dm_hi;
    unsigned long long* t_lo;
    unsigned long long* t_hi;
    int32_t* scan;             // [cap]
    int32_t* block_sums;       // [cap / 1024 + 1]
    int64_t* n_clamped;        // one int64
    int64_t* trial_start;      // [ndm + 1]: first sorted entry of each trial, or null
    int ndm;                   // trials (rows of trial_start - 1)
    hp_cand* out;
    int64_t out_cap;
    int64_t* out_count;
    int* status;
};
cudaError_t launch_merge(const MergeArgs& a, cudaStream_t s, int64_t* nlaunch);

int merge_sort_passes(int64_t cap);

}  // namespace hp
