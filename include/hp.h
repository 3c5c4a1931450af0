/*
 * hp.h -- C ABI of the GB300 single-pulse search library (the data-parallel
 * hot path of Heimdall++, arXiv 2512.00398).
 *
 * Pipeline (Section II-B stage list; Algorithm 1):
 *   incoherent dedispersion over every trial DM  ->  per trial: baseline
 *   removal, normalisation, boxcar matched filtering, peak detection  ->
 *   candidate merging / clustering in (DM, time, width).
 * RFI mitigation (first GPU stage of Algorithm 1) is not part of this path.
 *
 * Conventions shared by every call:
 *   - Return value: HP_OK (0) or a negative HP_ERR_* code.  Argument errors are
 *     reported before anything is enqueued.
 *   - Device pointers are CUDA global-memory addresses on the current device;
 *     host pointers are ordinary process memory.  Ownership never transfers:
 *     the caller owns every buffer it passes in, the plan owns its scratch.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously; nothing synchronises the host
 *     unless the call says so.  Device-side results (counts, statuses) are
 *     valid once the stream has completed.
 *   - A plan is not safe for concurrent use from several host threads or on
 *     several streams at once: calls on one plan must be ordered.
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define HP_OK 0
#define HP_ERR_INVALID_ARG (-1)      /* bad argument or plan state */
#define HP_ERR_CUDA (-2)             /* a CUDA runtime call failed */
#define HP_ERR_OOM (-3)              /* device allocation failed / workspace too small */
#define HP_ERR_CAND_OVERFLOW (-4)    /* more raw candidates than the plan's capacity */
#define HP_ERR_TIMEOUT (-5)          /* a bounded device wait gave up */
#define HP_ERR_NSAMPS_TOO_SHORT (-6) /* nsamps <= max delay + widest boxcar */

/* Human-readable name of a status code (static string, never NULL). */
const char* hp_status_str(int status);

/* ------------------------------------------------------------------ types */
typedef struct hp_plan hp_plan;

/* A merged candidate (one cluster of Section II-B "Candidate Merging and
 * Clustering"): the member with the highest S/N stands for the cluster.
 * 48 bytes, natural alignment. */
typedef struct {
    int32_t dm_idx;     /* trial index of the representative */
    int32_t width_idx;  /* boxcar index of the representative */
    int64_t sample;     /* start of the representative's boxcar, in dedispersed
                           samples (arrival time at f_top / tsamp) */
    float snr;          /* representative S/N, S / (sigma * sqrt(W)) */
    int32_t members;    /* raw candidates in the cluster */
    int32_t dm_lo;      /* smallest / largest member trial index */
    int32_t dm_hi;
    int64_t t_lo;       /* smallest member start sample */
    int64_t t_hi;       /* largest member boxcar end (start + W, exclusive) */
} hp_cand;

/* Caller-owned device buffer for merged candidates.  After the stream
 * completes, *count holds the TRUE number of clusters; only the first
 * min(*count, capacity) entries are written.  Clusters are ordered by their
 * smallest member (dm_idx, sample, width_idx). */
typedef struct {
    hp_cand* data;      /* device, capacity entries */
    int64_t capacity;
    int64_t* count;     /* device, one int64 */
} hp_cand_buf;

/* A raw (pre-merge) candidate: one maximal above-threshold run of one
 * (trial, width), placed at the run's largest boxcar sum.  24 bytes. */
typedef struct {
    int32_t dm_idx;
    int32_t width_idx;
    int64_t sample;     /* boxcar start of the peak */
    int64_t S;          /* exact integer boxcar sum at the peak */
} hp_raw_cand;

/* Caller-owned device buffer for raw candidates.  Same count convention as
 * hp_cand_buf; order is unspecified (hp_merge sorts). */
typedef struct {
    hp_raw_cand* data;  /* device, capacity entries */
    int64_t capacity;
    int64_t* count;     /* device, one int64 */
} hp_raw_buf;

/* ------------------------------------------------------------ plan set-up */

/* Create a search plan (host only; no CUDA call is made until the first
 * search).  Computes the delay table of Section II-B (Eq. 1 with the
 * cold-plasma law): for channel c at f_c = f_top + c*chan_bw MHz and trial
 * DM d, delay = rint(4148.808 * DM_d * (f_c^-2 - f_top^-2) / tsamp) samples,
 * evaluated in FP64.
 *   nchans        1..65536 channels, channel 0 at f_top_MHz
 *   chan_bw_MHz   < 0 (frequency falls with channel index); the lowest
 *                 channel frequency must stay > 0
 *   tsamp_s       > 0, sampling time in seconds
 *   dm_list       host, ndm finite values >= 0, non-decreasing (copied)
 *   boxcar_widths host, nw (1..32) strictly increasing widths in 1..16384 (copied)
 *   snr_threshold > 0 (finite)
 * Defaults: running-median baseline over 2.0 s, dm_tol 1, t_gap 0,
 * w_tol = nw (any width), raw-candidate capacity 2^22.
 * On error *out is set to NULL. */
int hp_plan_create(hp_plan** out, int nchans, double f_top_MHz, double chan_bw_MHz,
                   double tsamp_s, const float* dm_list, int ndm, const int* boxcar_widths,
                   int nw, float snr_threshold);

/* Release the plan, its device tables and any scratch it allocated itself.
 * Synchronises the device work it enqueued.  NULL is accepted. */
int hp_plan_destroy(hp_plan* plan);

/* Tunable parameters (hp_plan_set_param / hp_plan_get_param). */
#define HP_PARAM_BASELINE_MODE 0  /* 0 = running median (remedian), 1 = moving mean */
#define HP_PARAM_BASELINE_S 1     /* baseline window in seconds (> 0) */
#define HP_PARAM_DM_TOL 2         /* merge: max |trial index difference| (>= 0) */
#define HP_PARAM_T_GAP 3          /* merge: max gap between boxcar windows, samples */
#define HP_PARAM_W_TOL 4          /* merge: max |width index difference| (>= 0) */
#define HP_PARAM_RAW_CAPACITY 5   /* raw-candidate scratch capacity (>= 1024) */
#define HP_PARAM_DEDISP_CONFIG 6  /* dedispersion tile shape index (0..HP_NUM_DEDISP_CONFIGS-1), default 17;
                                     12 while HP_PARAM_SUBBAND_CHANS > 0 unless a shape was set */
#define HP_PARAM_STAGE_TIMING 7   /* 1 = record CUDA events around every stage launch */
#define HP_PARAM_TIMEOUT_S 8      /* limit of every bounded device wait, seconds (> 0) */
#define HP_PARAM_RFI 9            /* 1 = RFI mitigation before dedispersion (default 0) */
#define HP_PARAM_RFI_NB_K 10      /* narrowband threshold, integer >= 0 (default 5) */
#define HP_PARAM_RFI_BB_K 11      /* broadband threshold in sigma of the zero-DM series (> 0, default 5) */
/* Sub-band (two-stage) dedispersion, a variant the paper does not use: fewer
 * additions per trial for a bounded loss of sensitivity.  With S =
 * HP_PARAM_SUBBAND_CHANS > 0 the channels are cut into sub-bands of S
 * consecutive channels (first channel top(s) = s*S) and the trials into groups
 * of G = HP_PARAM_SUBBAND_GROUP consecutive trials with nominal trial
 * n(g) = g*G + (len(g) - 1) / 2 (len(g) = the group's size).  Stage 1 sums each
 * sub-band at each nominal trial, B[s][g][u] = sum over c in s of
 * x[u + delay(c,n(g)) - delay(top(s),n(g))][c]; stage 2 sums, per trial, the
 * shifted partial sums D~[d][t] = sum over s of B[s][g(d)][t + delay(top(s),d)].
 * This equals direct dedispersion with the effective table
 * e(c,d) = delay(top(s),d) + delay(c,n(g(d))) - delay(top(s),n(g(d))), which
 * hp_plan_delays then returns (hp_plan_max_delay its maximum; nout = nsamps -
 * that maximum).  hp_search, hp_dedisperse, hp_plan_autotune, batches (the
 * variant's files through their own two stages; hp_batch_autotune refuses it)
 * and streams (per searched buffer) follow the variant (tile shapes 7, 11,
 * 12 and 14 only).  |e - delay| <= |a_c - a_top| |DM_n - DM_d| + 2, a_c the
 * delay of channel c per unit DM in samples. */
#define HP_PARAM_SUBBAND_CHANS 12 /* S: channels per sub-band, 0 = direct dedispersion (default) */
#define HP_PARAM_SUBBAND_GROUP 13 /* G: trials per group, 1..ndm (default 8) */
/* Per-width normalisation, a variant the paper does not use (Heimdall normalises
 * every boxcar width on its own): with HP_PARAM_WIDTH_SIGMA = 1 every width W_k
 * gets sigma_k = 1.482602218505602 * MAD_k, MAD_k = the lower median of |S_k(t)|
 * over every start 0 <= t <= nout - W_k (exact), the threshold is
 * S >= thr * sigma_k (FP64), the S/N S / sigma_k, and sigma_k = 0 gives no
 * candidates for that width.  On white noise sigma_k ~ sigma sqrt(W_k); on red
 * noise it grows faster.  hp_search, hp_detect, batches and streams follow it
 * (a stream's sigmas are those of each searched buffer).  |S_k| must stay below 2^36 (series within +-2^21 for W <= 16384),
 * else HP_ERR_INVALID_ARG is latched.  hp_width_sigmas returns the sigmas. */
#define HP_PARAM_WIDTH_SIGMA 14   /* 0 = one sigma per trial scaled by sqrt(W) (default), 1 = per width */
/* Decimated boxcars, a variant the paper does not use (Heimdall scrunches the
 * series for its wide boxcars): with HP_PARAM_DECIMATE = R > 0 a width W > R
 * that is a multiple of R is tested only at the starts t = m q, q = W / R --
 * the boxcar of R samples on the series summed in blocks of q; a run is a
 * maximal set of consecutive grid starts above threshold, its candidate the
 * grid start of largest S (ties: the earliest).  Thresholds and sigmas are
 * unchanged (with HP_PARAM_WIDTH_SIGMA the per-width sigmas still count every
 * start).  q <= 1024 (R >= widest boxcar / 1024); series within +-2^21 (the
 * summed blocks are int32).  hp_search, hp_detect and batches follow it;
 * streams refuse it. */
#define HP_PARAM_DECIMATE 15      /* R: 0 = every start (default) */
/* Baseline removal fused into dedispersion (Section II-B runs baseline removal
 * on the dedispersed series; the result is the same either way): with
 * HP_PARAM_FUSE_LEVELS = 1, the median baseline and at least two remedian
 * levels, the dedispersion kernel of hp_search, batches and streams also forms
 * the second remedian level (the median of the five medians of five
 * consecutive sums) of every 25-sample group inside one of its time tiles from
 * the sums it holds on chip, and the search forms only the groups straddling a
 * tile edge or the end of the series from D, so the remedian no longer reads
 * the whole series.  0 (default): the remedian reads D, as hp_dedisperse and
 * hp_detect always do.  On the 4096-channel, 2^20-sample, 1500-trial file the
 * fused kernel instance runs its summation loop 1.4% slower (3.4 ms) and
 * saves 1.0 ms of search, so the default is off.  The sub-band variant keeps
 * the unfused remedian. */
#define HP_PARAM_FUSE_LEVELS 16   /* 1 = second remedian level in the dedispersion epilogue, 0 = off (default) */

#define HP_NUM_DEDISP_CONFIGS 20

int hp_plan_set_param(hp_plan* plan, int param, double value);
int hp_plan_get_param(const hp_plan* plan, int param, double* value);

/* Copy the delay table, int32 [ndm][nchans] row-major, into host memory (the
 * sub-band variant's effective table when HP_PARAM_SUBBAND_CHANS > 0). */
int hp_plan_delays(const hp_plan* plan, int32_t* out_host);

/* Largest delay of the table (samples) and the dedispersed length
 * nout = nsamps - max_delay for a given input length. */
int hp_plan_max_delay(const hp_plan* plan, int32_t* max_delay);

/* Device scratch needed by hp_search for inputs of nsamps samples. */
int hp_plan_workspace_bytes(const hp_plan* plan, int64_t nsamps, size_t* bytes);

/* Give the plan a caller-owned device workspace (256-byte aligned, at least
 * hp_plan_workspace_bytes).  While bound, the plan allocates no scratch (its
 * constant tables, a few MB, are allocated once by the first search); the
 * caller keeps ownership and must keep it alive until the plan is destroyed
 * or another workspace is bound.  Passing NULL unbinds (the plan then
 * allocates its own scratch with cudaMalloc on demand, grow-only).  The size
 * depends on the raw capacity and baseline mode: query it after setting them. */
int hp_plan_bind_workspace(hp_plan* plan, void* workspace_dev, size_t bytes);

/* ----------------------------------------------------------- the hot path */

/* The whole search (Algorithm 1 without RFI mitigation) on one filterbank.
 *   filterbank_dev  device uint8 [nsamps][nchans], time-major, caller-owned
 *   nsamps          > max_delay + widest boxcar (else HP_ERR_NSAMPS_TOO_SHORT)
 *   cand_out        caller-owned merged-candidate buffer
 * Steps: dedispersion D[d][t] = sum_c x[t + delay(c,d)][c] for
 * t in [0, nout); per trial the baseline b (HP_PARAM_BASELINE_MODE), y = D - b,
 * sigma = 1.482602218505602 * median|y|; boxcars S_W(t) = sum_{i<W} y(t+i);
 * candidates = one per maximal run of S_W(t) >= thr*sigma*sqrt(W) at the run's
 * largest S (ties: smallest t); friends-of-friends merge.  Asynchronous;
 * device-side failures (raw-candidate overflow, timeouts) are latched in the
 * plan and returned by hp_plan_sync_status. */
int hp_search(hp_plan* plan, const uint8_t* filterbank_dev, int64_t nsamps, void* stream,
              hp_cand_buf* cand_out);

/* RFI mitigation alone (Section II-B "RFI Mitigation": broadband interference
 * spans every channel, narrowband interference a few; Section III-C: broadband
 * interference is found on the DM = 0 series).  The paper gives no statistic;
 * reading: m_c = lower median of channel c, s_c = lower median of |x - m_c|;
 * channel c is flagged iff |m_c - M_m| > nb_k max(D_m, 1) or |s_c - M_s| >
 * nb_k max(D_s, 1), with M, D the lower median and the median absolute
 * deviation of m_c (of s_c) across channels; z[t] = sum_c x[t][c] with flagged
 * channels at m_c, y = z - b (the plan's baseline), sigma_z = 1.482602218505602
 * median|y|; sample t is flagged iff |y[t]| >= bb_k sigma_z (never when
 * sigma_z = 0); flagged channels and samples take the value m_c.  With
 * HP_PARAM_RFI = 1, hp_search applies it before dedispersion.
 *   filterbank_dev   device uint8 [nsamps][nchans]
 *   cleaned_dev      optional device uint8 [nsamps][nchans] (may not alias the input)
 *   chan_flag_dev    optional device uint8 [nchans] (1 = flagged)
 *   samp_flag_dev    optional device uint8 [nsamps] (1 = flagged)
 *   chan_median_dev  optional device int32 [nchans] (m_c)
 * Uses the plan's workspace; asynchronous on `stream`. */
int hp_rfi_clean(hp_plan* plan, const uint8_t* filterbank_dev, int64_t nsamps, void* stream,
                 uint8_t* cleaned_dev, uint8_t* chan_flag_dev, uint8_t* samp_flag_dev,
                 int32_t* chan_median_dev);

/* Dedispersion alone (Section II-B, "Incoherent Dedispersion"):
 *   out_dev  device int32 [ndm][out_pitch], out_pitch >= nout, a multiple of 4;
 *            samples t >= nout of each row are left untouched. */
int hp_dedisperse(hp_plan* plan, const uint8_t* filterbank_dev, int64_t nsamps,
                  int32_t* out_dev, int64_t out_pitch, void* stream);

/* The per-trial stages (baseline removal, normalisation, matched filtering,
 * peak detection; Algorithm 1's trial loop) on dedispersed series:
 *   series_dev  device int32 [ndm][pitch], nout valid samples per row, values
 *               within +-2^30 (y = D - b is kept as int32); left unchanged
 *   raw_out     caller-owned raw-candidate buffer (count = true number)
 *   sigma_dev   optional device double [ndm]: per-trial sigma (NULL to skip)
 *   mad_dev     optional device int64 [ndm]: per-trial median |y| (NULL to skip) */
int hp_detect(hp_plan* plan, const int32_t* series_dev, int64_t nout, int64_t pitch,
              void* stream, hp_raw_buf* raw_out, double* sigma_dev, int64_t* mad_dev);

/* The per-width sigmas and MADs of the last hp_search / hp_detect / batch search
 * of this plan with HP_PARAM_WIDTH_SIGMA = 1, copied (asynchronously on `stream`)
 * into caller-owned device arrays double [ndm][nw] / int64 [ndm][nw] (either may
 * be NULL).  HP_ERR_INVALID_ARG when the mode is off or nothing was searched in
 * it since it was set. */
int hp_width_sigmas(hp_plan* plan, double* sigma_w_dev, int64_t* mad_w_dev, void* stream);

/* Candidate merging and clustering (Section II-B; Algorithm 1, last stage):
 *   raw_dev / nraw_dev  device raw candidates and their device count (as
 *                       written by hp_detect: dm_idx < the plan's trial count,
 *                       width_idx < its width count; entries beyond capacity
 *                       ignored)
 *   sigma_dev           device double [ndm], per-trial sigma from hp_detect
 *   cand_out            merged clusters (see hp_cand_buf) */
int hp_merge(hp_plan* plan, const hp_raw_cand* raw_dev, const int64_t* nraw_dev,
             int64_t raw_capacity, const double* sigma_dev, void* stream,
             hp_cand_buf* cand_out);

/* Try every dedispersion tile shape (HP_PARAM_DEDISP_CONFIG values 0 ..
 * HP_NUM_DEDISP_CONFIGS - 1) on this input (transpose + dedispersion, two timed
 * passes each after a warm-up, events on `stream`, synchronising), keep the fastest in the
 * plan (HP_PARAM_DEDISP_CONFIG) and report it.  best_config / best_ms are
 * optional host outputs.  The tile shape is the only thing tuned; results do
 * not depend on it. */
int hp_plan_autotune(hp_plan* plan, const uint8_t* filterbank_dev, int64_t nsamps, void* stream,
                     int* best_config, float* best_ms);

/* ------------------------------------------------------------ batching */
/* Many filterbanks of uneven length, channel count and sampling time searched
 * together -- the multi-file workload that the paper (Section IV-C) serves
 * with a two-stage pipeline of CPU threads and task queues.  Here every file's
 * dedispersion tiles go into ONE kernel launch, the per-file search and merge
 * chains run side by side on internal streams, and the whole sequence is
 * captured once into a CUDA graph and replayed while the inputs, sizes and
 * outputs stay the same.  Results are identical to hp_search per file.
 *   plans  host array of nfiles (1..HP_BATCH_MAX_FILES) caller-owned plans, one
 *          per file; they must outlive the batch, and the batch sets the
 *          dedispersion tile configuration of its direct-dedispersion files
 *          (they share one: at creation the first such file's); files in the
 *          sub-band variant keep their own stage-1 tile shape. */
typedef struct hp_batch hp_batch;
#define HP_BATCH_MAX_FILES 32

int hp_batch_create(hp_batch** out, hp_plan* const* plans, int nfiles);
int hp_batch_destroy(hp_batch* batch);

/* Use tile configuration `config` for every direct-dedispersion file (drops a
 * captured graph). */
int hp_batch_set_config(hp_batch* batch, int config);

/* Time every dedispersion tile shape (the configurations that
 * HP_PARAM_DEDISP_CONFIG selects) on these inputs, one timed pass each after
 * one warm-up pass (synchronising), and keep the fastest for the batch and its plans.
 * Inputs as for hp_batch_search. */
int hp_batch_autotune(hp_batch* batch, const uint8_t* const* filterbanks_dev,
                      const int64_t* nsamps, void* stream, int* best_config, float* best_ms);

/* Search every file: filterbanks_dev / nsamps are host arrays of nfiles device
 * pointers and lengths; cand_out a host array of nfiles output buffers.  The
 * first call with a given set of arguments runs directly, the second captures
 * a CUDA graph, later identical calls replay it.  Asynchronous on `stream`. */
int hp_batch_search(hp_batch* batch, const uint8_t* const* filterbanks_dev, const int64_t* nsamps,
                    void* stream, hp_cand_buf* cand_out);

/* Wait for `stream`, then return (and clear) the first device-side status of
 * any of the batch's plans (see hp_plan_sync_status). */
int hp_batch_sync_status(hp_batch* batch, void* stream);

/* Kernel launches enqueued per hp_batch_search call (graph nodes when replayed). */
int hp_batch_kernels_per_call(const hp_batch* batch, int64_t* kernels);

/* Per-stage timing and launch accounting (no counterpart in the paper, whose
 * Fig. 2 reports per-stage times of Heimdall).  With HP_PARAM_STAGE_TIMING = 1
 * every stage launch is bracketed by CUDA events recorded on the launching
 * stream (up to 4096 launches per stage are kept).  Kernel launches are
 * counted always. */
#define HP_STAGE_TRANSPOSE 0    /* time-major -> channel-major copy of the input */
#define HP_STAGE_DEDISP 1       /* dedispersion kernel */
#define HP_STAGE_SEARCH 2       /* baseline, sigma, boxcars, peaks */
#define HP_STAGE_MERGE 3        /* sort + friends-of-friends */
#define HP_STAGE_RFI 4          /* RFI mitigation (when HP_PARAM_RFI = 1) */
#define HP_STAGE_SUBBAND_SUM 5  /* sub-band variant, stage 2 (stage 1 counts as HP_STAGE_DEDISP) */
#define HP_NUM_STAGES 6
typedef struct {
    double stage_ms[HP_NUM_STAGES];      /* summed event time of the recorded launches */
    int64_t stage_calls[HP_NUM_STAGES];  /* launches whose events were summed */
    int64_t kernel_launches;             /* CUDA kernels launched by the library */
    int64_t device_allocs;               /* device allocations the plan made since it was
                                            created (its allocator or cudaMalloc); the
                                            paper's Table II counts the same for Heimdall */
} hp_stats;

/* Synchronise on the recorded events, write the totals since the last reset
 * into *out (host), then reset them if `reset` is non-zero (device_allocs is
 * never reset). */
int hp_plan_stats(hp_plan* plan, hp_stats* out, int reset);

/* Candidate merging that allocates nothing (the paper has no counterpart).
 * Some callers cannot allocate device memory when they merge: a real-time
 * pipeline that forbids allocation after start-up (cudaMalloc can block and can
 * fail on a full device), or code inside a framework that owns all device
 * memory.  This call runs the same kernels as hp_merge, with the same result,
 * but keeps all of their scratch in one fixed device array built into the
 * library (about 5.3 MB, reserved on every GPU that loads the library until the
 * process exits), and it calls no cudaMalloc, cudaFree or allocating library
 * routine.  No plan is needed:
 *   raw_dev / nraw_dev  device raw candidates and their device count
 *   raw_capacity        entries of raw_dev, at most HP_MERGE_STATIC_MAX_RAW;
 *                       larger values are rejected with HP_ERR_INVALID_ARG
 *   sigma_dev           device double [ndm], per-trial sigma (as hp_detect writes)
 *   boxcar_widths       host, nw (1..32) strictly increasing widths (as in the plan)
 *   dm_tol, t_gap, w_tol  merge tolerances, within the bounds that
 *                       HP_PARAM_DM_TOL / T_GAP / W_TOL accept (else HP_ERR_INVALID_ARG)
 *   cand_out            merged clusters (see hp_cand_buf)
 *   status_dev          optional device int32, caller-owned: when the device count
 *                       *nraw_dev exceeds raw_capacity, only the first raw_capacity
 *                       entries (in buffer order, which for hp_detect output is
 *                       arbitrary) are merged and HP_ERR_CAND_OVERFLOW is written
 *                       here if it still holds HP_OK (0); the caller sets it to 0
 *                       beforehand and reads it once the stream has completed.
 *                       With NULL such a truncation is not reported.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture, and do not call
 * this after resetting the device (cudaDeviceReset), which moves the array.
 * All calls share the one array, and its contents persist from call to call
 * (every word the kernels read is rewritten first, so nothing has to be
 * cleared); calls whose work overlaps on the GPU, e.g. on two streams at once,
 * race on it and must be ordered by the caller. */
#define HP_MERGE_STATIC_MAX_RAW 65536
int hp_merge_static(const hp_raw_cand* raw_dev, const int64_t* nraw_dev, int64_t raw_capacity,
                    const double* sigma_dev, const int* boxcar_widths, int nw, int dm_tol,
                    int64_t t_gap, int w_tol, void* stream, hp_cand_buf* cand_out,
                    int32_t* status_dev);

/* Device memory of the plan (its tables and, unless a workspace is bound, its
 * search workspace) from a caller's allocator instead of cudaMalloc/cudaFree,
 * e.g. a framework's caching allocator.  alloc returns a device pointer
 * aligned to 256 bytes or NULL; free gets back the pointer and its size.  The
 * plan synchronises the device before it frees anything, so the memory is idle
 * when free is called.  Both NULL restores cudaMalloc.  Memory obtained from
 * the previous allocator is returned to it first.  Not thread-safe with
 * concurrent calls on the same plan. */
typedef void* (*hp_alloc_fn)(size_t bytes, void* ctx);
typedef void (*hp_free_fn)(void* ptr, size_t bytes, void* ctx);
int hp_plan_set_allocator(hp_plan* plan, hp_alloc_fn alloc, hp_free_fn free_fn, void* ctx);

/* Wait for the plan's enqueued work on `stream` and return (then clear) the
 * first device-side status latched since the last call: HP_OK,
 * HP_ERR_CAND_OVERFLOW or HP_ERR_TIMEOUT.  Synchronises the stream. */
int hp_plan_sync_status(hp_plan* plan, void* stream);

/* ----------------------------------------------------------- streaming */
/* Many beams searched as their data arrive, gulp by gulp.  Sections III-B and
 * V-C of the paper search long observations in chunks whose time segments
 * overlap so that a dispersed pulse stays whole across a chunk boundary, and
 * overlap transfers with computation by double buffering (Section IV-C); the
 * paper gives the overlap only in words.  The rule used here, for gulps of G
 * samples and H = max_delay + widest boxcar - 1:
 *   - gulp g of a beam (input samples [g G, (g+1) G)) is searched as one
 *     series over input [B0, E), E = (g+1) G, B0 = max(0, g G - H): the last
 *     H samples of earlier gulps stay resident on the device (the tail);
 *     baseline and sigma are those of a plain search of that buffer;
 *   - its window is dedispersed samples [B0, B0 + nwin), nwin = E - H - B0;
 *     the Wmax - 1 samples after it are look-ahead.  A gulp with E <= H has
 *     no window (nwin <= 0) and only fills the tail;
 *   - a run of above-threshold boxcar starts is reported by the gulp whose
 *     window holds its first start, its peak taken inside that buffer; a run
 *     that the previous window ended inside is not reported again;
 *   - each gulp's raw candidates are merged on their own (as hp_merge), with
 *     samples in the beam's dedispersed time (window start + offset).
 * Continuous batching: a native scheduler thread takes the gulps that have
 * arrived from every admitted beam (at most one per beam) into one step --
 * one transpose and one dedispersion launch over all of them, then per gulp
 * the search and merge on side streams and the copy of its candidates to host
 * memory -- and keeps up to two steps in flight, so gulps that arrive while a
 * step runs join the next.  Beams are admitted in order of their first push
 * while the device budget has room for their tails; the others wait until an
 * admitted beam ends.  A beam's results do not depend on the other beams. */
typedef struct hp_stream hp_stream;
#define HP_STREAM_MAX_BEAMS 1024
#define HP_STREAM_EMPTY 1   /* hp_stream_poll: no result within the timeout */

typedef struct {
    int32_t nbeams;          /* beam ids 0 .. nbeams-1 (1..HP_STREAM_MAX_BEAMS) */
    int32_t max_batch;       /* gulps per step, 1..HP_BATCH_MAX_FILES (0: min(nbeams, 32)) */
    int64_t gulp;            /* samples per gulp, >= 64 and >= H / 62 */
    int64_t hbm_budget;      /* device bytes the stream may allocate (0: no limit) */
    int64_t cand_capacity;   /* merged candidates kept per gulp, >= 1 */
    int64_t raw_capacity;    /* raw candidates per gulp, >= 1024 */
} hp_stream_config;

typedef struct {
    int32_t beam;
    int32_t status;          /* HP_OK or the device-side status of the gulp's step */
    int64_t gulp_index;      /* 0, 1, ... in push order of the beam */
    int64_t window_start;    /* B0: first dedispersed sample of the window */
    int64_t window_len;      /* nwin, 0 when the gulp had no window */
    int64_t ncand;           /* merged candidates of the gulp (may exceed what is kept) */
    double latency_s;        /* hp_stream_push -> candidates in host memory */
    int32_t batch_size;      /* gulps in the step that searched it */
    int32_t pad_;
} hp_gulp_result;

typedef struct {
    int64_t steps;           /* batched steps completed */
    int64_t gulps;           /* gulps completed */
    int32_t beam_slots;      /* beams the budget holds at once */
    int32_t max_batch;
    int32_t admitted;        /* beams holding a slot now */
    int32_t waiting;         /* beams waiting for a slot */
    int64_t device_bytes;    /* bytes allocated by the stream */
    int64_t tail_samples;    /* H */
    int64_t max_batch_seen;
    int64_t device_allocs;   /* device allocations made since hp_stream_open (all at open) */
} hp_stream_stats;

/* Open a stream.  The plan (caller-owned, not used by the stream afterwards)
 * supplies the band, trials, widths, threshold and parameters; the stream
 * keeps its own copy.  Allocates everything it will use: per step slot a
 * search workspace for G + H samples and a candidate buffer, per beam slot a
 * ring of ceil(H/G) + 2 gulps and two [ndm][nw] carry arrays.  HP_ERR_OOM when
 * the budget does not hold one beam slot and one step slot. */
int hp_stream_open(hp_stream** out, const hp_plan* plan, const hp_stream_config* config);

/* Queue the next gulp of `beam`: nsamps == gulp samples of nchans bytes each
 * ([nsamps][nchans], host memory, pinned for asynchronous copies).  The
 * memory must stay valid and unchanged until hp_stream_poll has returned
 * this gulp's result.  Returns at once (HP_ERR_INVALID_ARG for an ended beam
 * or a wrong size; the stream's first CUDA error once one occurred). */
int hp_stream_push(hp_stream* s, int beam, const uint8_t* gulp_host, int64_t nsamps);

/* No more gulps for `beam`: its slot is released once its queued gulps are
 * done, and the longest-waiting beam takes it. */
int hp_stream_end_beam(hp_stream* s, int beam);

/* Wait up to timeout_ms (< 0: forever) for the next finished gulp, in order
 * of completion: fills *result and copies min(ncand, cand_cap, cand_capacity)
 * candidates to host memory `cands`.  HP_STREAM_EMPTY when none finished. */
int hp_stream_poll(hp_stream* s, hp_gulp_result* result, hp_cand* cands, int64_t cand_cap,
                   int timeout_ms);

int hp_stream_get_stats(hp_stream* s, hp_stream_stats* out);

/* Stop the stream: queued gulps that no step has taken are dropped, the steps
 * in flight are waited for, unread results are discarded and everything the
 * stream allocated is freed.  (To finish a stream, poll until every pushed
 * gulp's result has arrived, then close.) */
int hp_stream_close(hp_stream* s);

#ifdef __cplusplus
}
#endif
#endif /* HP_H */
