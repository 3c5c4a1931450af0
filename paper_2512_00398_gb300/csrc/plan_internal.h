// plan_internal.h -- the plan object and the host helpers that the plan,
// batch and stream runtimes share (plan.cpp, stream.cpp).  Not part of the
// public C ABI (include/hp.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "hp_internal.h"

namespace hp {

// Byte offsets of every array of a search workspace for one input length.
struct Layout {
    int64_t nsamps = 0, nout = 0;
    int64_t xt_pitch = 0, dpitch = 0;
    int64_t lvl_pitch_a = 0, lvl_pitch_b = 0, mean_pitch = 0;
    size_t xt = 0, D = 0, lvl_a = 0, lvl_b = 0, mean = 0, hist = 0, rbucket = 0, rrank = 0,
           mad = 0, ybound = 0, sigma = 0, tint = 0, raw = 0, raw_count = 0, keys0 = 0, keys1 = 0,
           vals0 = 0, vals1 = 0, parent = 0, best = 0, rep = 0, members = 0, dmlo = 0,
           dmhi = 0, tlo = 0, thi = 0, scan = 0, bsums = 0, nclamp = 0, tails = 0, tcount = 0,
           tstart = 0;
    // RFI stage: channel counts, statistics and flags, the zero-DM series and
    // the scratch of its statistics (a one-trial stats-only search)
    size_t r_hist = 0, r_med = 0, r_spread = 0, r_cflag = 0, r_sflag = 0, r_one = 0, r_z = 0,
           r_lvl_a = 0, r_lvl_b = 0, r_mean = 0, r_zhist = 0, r_bucket = 0, r_rank = 0,
           r_mad = 0, r_sigma = 0, r_tint = 0, r_y = 0;
    int64_t r_zpitch = 0, r_lvl_pitch_a = 0, r_lvl_pitch_b = 0, r_mean_pitch = 0;
    size_t whist = 0, wstate = 0, wmad = 0, sigw = 0;   // per-width sigmas (if enabled)
    size_t ydec = 0, tint_lv = 0, widths_lv = 0;         // decimated boxcars (if enabled)
    int ndec = 0;
    int32_t dec_q[kMaxWidths] = {};
    int64_t dec_off[kMaxWidths] = {}, dec_pitch[kMaxWidths] = {};
    size_t sb = 0;             // sub-band partial sums (sub-band variant)
    int64_t sb_pitch = 0, sb_len = 0;
    int sb_chunks = 0;         // DM-tile chunks whose partial sums fit `sb` at once
    // second remedian level of D, written by the dedispersion (median baseline,
    // at least two levels, direct dedispersion): [ndm][lv2_pitch]
    size_t lv2 = 0;
    int64_t lv2_pitch = 0;
    size_t y = 0;              // baseline-subtracted series (unless it overwrites D)
    int64_t ypitch = 0;
    bool y_in_D = false;
    size_t total = 0;
    size_t search_begin = 0;   // everything from here on is search/merge scratch
};

}  // namespace hp

struct hp_plan {
    int nchans = 0;
    double f_top = 0, chan_bw = 0, tsamp = 0;
    std::vector<float> dm_list;
    std::vector<int32_t> widths;
    float thr = 0;
    int baseline_mode = 0;
    double baseline_s = 2.0;
    int dm_tol = 1;
    int64_t t_gap = 0;
    int w_tol = 0;
    int64_t raw_capacity = (int64_t)1 << 22;
    bool fuse_levels = false;          // second remedian level in the dedispersion epilogue
    int dedisp_cfg = hp::kDefaultDedispConfig;
    bool dedisp_cfg_set = false;       // a tile shape was set (or autotuned) by the caller
    uint64_t timeout_ns = 1000000000ull;

    std::vector<int32_t> delays;   // [ndm][nchans]
    int32_t maxd = 0, wmax = 0;    // maxd: of the table the dedispersion realises

    // sub-band variant (sb_chans > 0): sub-bands of sb_chans channels, groups of
    // sb_group trials; sb_eff is the effective table [ndm][nchans]
    int sb_chans = 0, sb_group = 8;
    std::vector<int32_t> sb_eff;
    int32_t sb_nsub = 0, sb_ngrp = 0, sb_gchunk = 0, sb_nchunks = 0;
    int32_t sb_maxrel = 0;         // largest in-sub-band delay at a nominal trial
    int32_t sb_maxtop = 0;         // largest delay of a sub-band's first channel
    int32_t sb_spread = 0;         // largest first-channel delay spread of a stage-2 block
    const int32_t* d_sbtop = nullptr;

    hp::DedispTiling tiling;           // for dedisp_cfg

    // device state
    int device = -1;
    void* tables = nullptr;        // plan-owned constant tables + status word
    size_t tables_bytes = 0;
    int tables_cfg = -1;
    int64_t tables_sb = -1;        // (sb_chans, sb_group) the tables were built for
    int* status = nullptr;
    const hp::TileDesc* d_tiles = nullptr;
    const hp::StageDesc* d_stages = nullptr;
    const hp::ChanDesc* d_chans = nullptr;
    const uint32_t* d_addr = nullptr;
    int32_t* d_widths = nullptr;

    // device allocator for the plan's tables and workspace (default cudaMalloc)
    bool width_sigma = false;      // per-width sigmas instead of sigma * sqrt(W)
    int decimate = 0;              // decimated boxcars: R (0 = every start)
    const double* last_sigw = nullptr;   // where the last search put them ([ndm][nw])
    const int64_t* last_wmad = nullptr;
    bool rfi = false;              // RFI mitigation before dedispersion
    int rfi_nb_k = 5;
    float rfi_bb_k = 5.0f;
    int pending_status = 0;        // latched status kept while the tables are reallocated
    hp_alloc_fn alloc_fn = nullptr;
    hp_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;

    void* ws_user = nullptr;
    size_t ws_user_bytes = 0;
    void* ws_own = nullptr;
    size_t ws_own_bytes = 0;

    // stage timing (events on the launching stream) and launch accounting
    bool timing = false;
    std::vector<cudaEvent_t> ev[HP_NUM_STAGES];   // pairs (begin, end)
    int ev_used[HP_NUM_STAGES] = {};
    int64_t launches = 0;
    int64_t device_allocs = 0;     // successful device allocations since creation

    int ndm() const { return (int)dm_list.size(); }
    int nw() const { return (int)widths.size(); }
};

namespace hp {

int check_cuda(cudaError_t e);
int plan_alloc(hp_plan* p, size_t bytes, void** out);
void plan_free(hp_plan* p, void* ptr, size_t bytes);
int ensure_device_tables(hp_plan* p);
int ensure_workspace(hp_plan* p, size_t need, uint8_t** base);
Layout make_layout(const hp_plan* p, int64_t nsamps, bool with_dedisp);
int64_t xt_pitch_for(int64_t nsamps);
int validate_search_input(const hp_plan* p, const void* ptr, int64_t nsamps);
bool reach_ok(const hp_plan* p, int64_t nout, int64_t xt_pitch);
DedispJob make_job(const hp_plan* p, const uint8_t* xt, int64_t xt_pitch, int32_t* out,
                   int64_t out_pitch, int64_t nout);
// Stages 1 and 2 of the sub-band variant on the transposed input at ws + L.xt.
int run_subband(hp_plan* p, const Layout& L, uint8_t* ws, int32_t* out, int64_t out_pitch,
                cudaStream_t s);
// The dedispersion of the plan's own series also writes the second remedian
// level, and the search of that series (dedispersed with tile shape cfg)
// starts from it; no-ops unless the layout holds the level buffer.
void fuse_levels(DedispJob& J, const Layout& L, uint8_t* ws);
void fuse_levels(SearchArgs& a, const Layout& L, uint8_t* ws, int cfg);
SearchArgs make_search_args(hp_plan* p, const Layout& L, uint8_t* ws, const int32_t* D,
                            int64_t pitch, int64_t nout, hp_raw_cand* raw, int64_t raw_cap,
                            int64_t* raw_count);
RfiArgs make_rfi_args(hp_plan* p, const Layout& L, uint8_t* ws, const uint8_t* x, uint8_t* xt,
                      int64_t xt_pitch, int64_t nsamps, uint8_t* out);
MergeArgs make_merge_args(hp_plan* p, const Layout& L, uint8_t* ws, const hp_raw_cand* raw,
                          const int64_t* nraw, int64_t raw_cap, const double* sigma,
                          hp_cand_buf* out);

}  // namespace hp
