/*
 * hp_bench.h -- measurement helpers of the search library (no counterpart in
 * the paper).  They measure the issue rates that bound the dedispersion
 * kernel, which is limited by integer-ALU and shared-memory throughput, not by
 * HBM bandwidth or tensor cores.
 */
#ifndef HP_BENCH_H
#define HP_BENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double int_add_ops_per_s;   /* 32-bit integer adds (lane operations) per second */
    double prmt_ops_per_s;      /* byte-permute lane operations per second */
    double lds32_bytes_per_s;   /* conflict-free 32-bit shared-memory load bytes per second */
    int sm_count;               /* multiprocessors of the current device */
    int reserved;
} hp_peaks;

/* Run the microbenchmarks on the current device (synchronous, about a
 * second).  Each kernel fills every SM with independent dependency chains,
 * is timed with CUDA events after a warm-up launch, and the rate is the best
 * of three launches.  *out is host memory.  Returns HP_OK or HP_ERR_CUDA. */
int hp_measure_peaks(hp_peaks* out);

/* The shape of dedispersion tile shape `config` (HP_PARAM_DEDISP_CONFIG), for
 * rooflines: out[0..7] = trials per warp, 4-sample words per lane, warps along
 * the trials, warps along time (plus one producer warp), shared-memory bytes
 * per stage buffer, stage buffers, channel-pair loop unroll, threads per
 * block.  A lane loads words + 1 row words per channel and trial and spends
 * two PRMTs per word (alignment, odd bytes).  out is host memory.  Returns
 * HP_OK or HP_ERR_INVALID_ARG for an unknown config. */
int hp_dedisp_config(int config, int32_t out[8]);

/* Self-test of the bounded device waits that every staged kernel uses (its
 * barrier waits give up after HP_PARAM_TIMEOUT_S and latch HP_ERR_TIMEOUT, so
 * a stalled copy ends the launch with a status instead of a hang).  One block
 * of two warps on the current device: barrier A is initialised for one arrival
 * that nobody makes; warp 0 waits on it (the wait runs out after limit_ns,
 * latches HP_ERR_TIMEOUT and raises the block's abort flag) and warp 1 waits
 * on it too (it leaves on that flag, or runs out itself).  Barrier B gets its
 * one arrival and its wait must succeed.  Synchronous.  out (host memory):
 * out[0] = the latched status (HP_ERR_TIMEOUT expected), out[1] = 1 if warp
 * 0's wait ran out, out[2] = 1 if warp 1's wait gave up, out[3] = 1 if the
 * wait on the completed barrier succeeded.  Returns HP_OK, HP_ERR_INVALID_ARG
 * (null out, limit_ns outside (0, 10 s]) or HP_ERR_CUDA. */
int hp_selftest_bounded_wait(int64_t limit_ns, int32_t out[4]);

#ifdef __cplusplus
}
#endif
#endif /* HP_BENCH_H */
