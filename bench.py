#!/usr/bin/env python3
"""Benchmark of the GB300 single-pulse search (one JSON line on rank 0).

A step is one whole search (dedispersion, per-trial baseline / sigma /
boxcars / peaks, merge) of one synthetic filterbank shaped like the paper's
single-file FAST workload: 4096 channels over 1000-1500 MHz, 2^20 samples of
49.152 us (51.5 s), ~1500 trials on DM 0-2000, boxcars 1..4096, S/N 6.
The 4.3 GB input is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank searches its own file
(weak scaling, no collective on the data path); the time is the max over ranks.
``--impl reference`` times the CPU oracle on the host cores instead, on a
bounded sample of trials of the same workload.
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DM-trial·samples/s"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dedispersion kernel on this workload and tile configuration: an ncu capture of the
# same kernel on the 2^18-sample case (nout 168 628, profiles/dedisp_rows_kernel_fast_4096ch.md)
# scaled by the number of time tiles to the full nout of 955 060.  Keyed by the kernel
# source it was measured on; a changed kernel, another workload or another
# configuration reports null until it is captured again.
DEDISP_TRAFFIC = {"source_sha256_16": "0e82e2697ab3fb83", "bytes": (6.095e9 + 1.010e9) * 955060 / 168628,
                  "ndm": 1500, "nchans": 4096, "nsamps": 1 << 20, "config": 17}
# The same for the two stages of the sub-band variant (64-channel sub-bands, groups
# of 8 trials): DRAM bytes of one step, captured on the 2^18-sample case
# (profiles/subband_fast_4096ch.md).  Stage 1's traffic grows with its byte-adds
# (scaled by 7.445e11 / 1.389e11 to the full file, within 0.5% of an earlier full-size
# capture); stage 2's partial-sum rows do not scale with the file length, so it stays null.
SUBBAND_TRAFFIC = {"source_sha256_16": "0e82e2697ab3fb83+6752b94441917dc0",
                   "stage1": (6.036e9 + 8.660e9) * 7.445e11 / 1.389e11, "stage2": None,
                   "ndm": 1500, "nchans": 4096, "nsamps": 1 << 20, "config": 12, "S": 64, "G": 8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dedisp-config", type=int, default=None)
    ap.add_argument("--nsamps", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fused", action="store_true",
                    help="skip the search with the remedian levels fused into dedispersion")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 16-file batched-vs-plain measurement")
    ap.add_argument("--batch-files", type=int, default=16)
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the 19-beam streamed (serving) measurement")
    ap.add_argument("--no-subband", action="store_true",
                    help="skip the sub-band dedispersion variant's line")
    ap.add_argument("--subband", default="64,8",
                    help="channels per sub-band and trials per group of the variant")
    ap.add_argument("--no-width-sigma", action="store_true",
                    help="skip the per-width normalisation variant's line")
    ap.add_argument("--no-decimate", action="store_true",
                    help="skip the decimated-boxcar variant's line")
    ap.add_argument("--decimate", type=int, default=16,
                    help="R of the decimated-boxcar variant")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the tiny and stress recipes' lines")
    ap.add_argument("--serve-beams", type=int, default=19)
    ap.add_argument("--serve-seconds", type=float, default=40.0,
                    help="seconds of real-time stream per beam")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------- ranks (weak scaling)
def rank_workload(rank, world, nsamps):
    """One file per rank: the FAST shape, a different seed on every rank when
    there are several (the path shards by file, nothing is exchanged)."""
    if world == 1:
        return workload(nsamps)
    from paper_2512_00398_gb300 import workloads
    return workloads.fast(nsamps=nsamps, seed=2 + rank)


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the time)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def aggregate(world, units_per_rank, seconds):
    """Whole-job throughput: every rank processed `units_per_rank` in `seconds`."""
    return world * units_per_rank / seconds


def recovery_rates(w, pulses, cands):
    """Injected pulses found among the merged candidates (the criterion of
    workloads.recovered), for matched S/N >= 10 and for 6-10."""
    from paper_2512_00398_gb300.workloads import recovered
    out = {}
    if all(p.snr != p.snr for p in pulses):
        # amplitudes given per channel (the tiny recipe): no nominal S/N
        found = sum(1 for p in pulses if recovered(p, cands, w, snr_min=w.threshold))
        return {"all": f"{found}/{len(pulses)}"}
    for name, lo, hi in (("snr>=10", 10.0, float("inf")), ("snr 6-10", 6.0, 10.0)):
        sel = [p for p in pulses if lo <= p.snr < hi]
        found = sum(1 for p in sel if recovered(p, cands, w, snr_min=w.threshold))
        out[name] = f"{found}/{len(sel)}"
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of one GPU during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- workload
def workload(nsamps):
    from paper_2512_00398_gb300 import workloads
    return workloads.fast(nsamps=nsamps)


def describe(w, nout):
    o = w.obs
    return {"workload": f"single FAST-like filterbank: {o.nchans} ch x {o.nsamps} samples "
                        f"({o.duration:.1f} s at {o.tsamp * 1e6:.3f} us), {w.ndm} trials on "
                        f"DM 0-{float(w.dm_list[-1]):.0f}, boxcars 1..{int(w.widths[-1])}, S/N "
                        f"{w.threshold:g}, 20 injected pulses",
            "nchans": o.nchans, "nsamps": o.nsamps, "tsamp_s": o.tsamp, "ndm": w.ndm,
            "nout": nout, "nw": w.nw, "l2": "inputs larger than L2 (no flush)"}


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0   # earlier GB300 measurement, used only when the file is absent


def source_sha(name):
    import hashlib
    src = os.path.join(ROOT, "paper_2512_00398_gb300", "csrc", name)
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def subband_traffic(w, config, S, G):
    t = SUBBAND_TRAFFIC
    sha = source_sha("dedisp.cu") + "+" + source_sha("subband.cu")
    if (sha != t["source_sha256_16"] or w.ndm != t["ndm"] or w.obs.nchans != t["nchans"]
            or w.obs.nsamps != t["nsamps"] or config != t["config"] or (S, G) != (t["S"], t["G"])):
        return None, None
    return t["stage1"], t["stage2"]


# ALU-pipe PRMTs per aligned 4-sample word: the alignment and the odd bytes
PRMT_PER_WORD = 2.0


def dedisp_traffic(w, config):
    sha = source_sha("dedisp.cu")
    t = DEDISP_TRAFFIC
    if (sha != t["source_sha256_16"] or w.ndm != t["ndm"] or w.obs.nchans != t["nchans"]
            or w.obs.nsamps != t["nsamps"] or config != t["config"]):
        return None
    return t["bytes"]


# ------------------------------------------------------------ CPU oracle
def oracle_sample(s, w, ntrials, d0=None):
    """Time the oracle on `ntrials` consecutive trials of the full input."""
    import oracle
    o = w.obs
    tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list)
    nout = o.nsamps - int(tab.max())
    if d0 is None:
        d0 = max(0, w.ndm // 2 - ntrials // 2)
    t = time.perf_counter()
    D = oracle.dedisperse(s.data, tab, rows=(d0, d0 + ntrials), nout=nout)
    raw, _, _ = oracle.search_trials(D, d0, o.tsamp, w.widths, w.threshold)
    oracle.merge(raw, w.widths)
    dt = time.perf_counter() - t
    return dt, ntrials * nout, nout


def cpu_baseline(s, w, budget_s=15.0):
    import oracle
    dt1, units1, nout = oracle_sample(s, w, 1)
    k = int(max(1, min(64, budget_s / max(dt1, 1e-3))))
    dt, units, _ = oracle_sample(s, w, k)
    return {"value": units / dt, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{k} consecutive trials (of {w.ndm}) around the middle of the DM range, "
                      f"full {w.obs.nsamps} samples: dedispersion + per-trial stages + merge, "
                      f"{dt:.1f} s"}


# -------------------------------------------------------------- our path
def run_ours(args):
    import torch
    import paper_2512_00398_gb300 as hp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = rank_workload(rank, world, args.nsamps)
    s = w.generate(threads=min(16, os.cpu_count() or 8))
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    if args.dedisp_config is not None:
        plan.set_param("dedisp_config", args.dedisp_config)
    nout = plan.nout(o.nsamps)
    plan.bind_workspace(o.nsamps)
    fb = torch.from_numpy(s.data).cuda()
    out = hp.new_cand_buf(1 << 16)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        hp.hp_search(plan, fb, stream, out=out)
    st = hp.hp_plan_sync_status(plan, stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "warm-up")
    ncl = int(out[1].item())
    cands = hp.cands_to_numpy(*out)
    recovery = recovery_rates(w, s.pulses, cands)
    hp.hp_plan_stats(plan, reset=True)
    plan.set_param("stage_timing", 1)

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            hp.hp_search(plan, fb, stream, out=out)
        e1.record(stream)
        barrier()
    dev_ms = e0.elapsed_time(e1) / args.steps
    st = hp.hp_plan_sync_status(plan, stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "timed region")
    stats = hp.hp_plan_stats(plan, reset=True)
    # the same search with the RFI stage on (two more steps, not part of `value`)
    plan.set_param("rfi", 1)
    for _ in range(3):
        hp.hp_search(plan, fb, stream, out=out)
    st = hp.hp_plan_sync_status(plan, stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "search with RFI stage")
    rstats = hp.hp_plan_stats(plan, reset=True)
    rfi_ms = rstats["stage_ms"]["rfi"] / max(1, rstats["stage_calls"]["rfi"])
    plan.set_param("rfi", 0)
    # the same search with the second remedian level formed in the dedispersion
    # epilogue (HP_PARAM_FUSE_LEVELS = 1, not the default): stage times and step
    # time over `steps` searches, candidates identical to the default path's
    fused = None
    if not args.no_fused:
        plan.set_param("fuse_levels", 1)
        plan.bind_workspace(o.nsamps)
        for _ in range(2):
            hp.hp_search(plan, fb, stream, out=out)
        hp.hp_plan_stats(plan, reset=True)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            hp.hp_search(plan, fb, stream, out=out)
        f1.record(stream)
        torch.cuda.synchronize()
        fst_code = hp.hp_plan_sync_status(plan, stream)
        if fst_code != hp.HP_OK:
            raise hp.HPError(fst_code, "fused search")
        fst = hp.hp_plan_stats(plan, reset=True)
        fused = {"ms_per_step": f0.elapsed_time(f1) / args.steps,
                 "stages_ms": {k: v / max(1, fst["stage_calls"][k])
                               for k, v in fst["stage_ms"].items() if v},
                 "identical_candidates": bool(np.array_equal(hp.cands_to_numpy(*out), cands))}
        plan.set_param("fuse_levels", 0)
    plan.set_param("stage_timing", 0)

    # end to end through the public call: every step copies its 4.3 GB input from
    # pinned host memory to the device, searches it and reads the count and the
    # candidate records back.  Two device input buffers: the copy of the next
    # step's input (on a copy stream) overlaps this step's search; the timed
    # region holds exactly `steps` copies, searches and reads (the copy for the
    # first timed step is issued before it, one for the step after the last inside).
    e2e = None
    if not args.no_e2e:
        host = torch.from_numpy(s.data).pin_memory()
        res = torch.empty(out[0].numel(), dtype=torch.uint8).pin_memory()
        cnt_h = torch.empty(1, dtype=torch.int64).pin_memory()
        bufs = [fb, torch.empty_like(fb)]
        cs = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]
        used_rec = [False, False]

        def upload(k):
            b = k % 2
            if used_rec[b]:
                cs.wait_event(used[b])       # the search that last read this buffer
            with torch.cuda.stream(cs):
                bufs[b].copy_(host, non_blocking=True)
            copied[b].record(cs)

        upload(0)
        d2h = []
        total = args.warmup + args.steps
        for it in range(total):
            if it == args.warmup:
                barrier()
                t0 = time.perf_counter()
            b = it % 2
            stream.wait_event(copied[b])
            hp.hp_search(plan, bufs[b], stream, out=out)
            used[b].record(stream)
            used_rec[b] = True
            upload(it + 1)
            cnt_h.copy_(out[1], non_blocking=True)
            stream.synchronize()
            n = min(int(cnt_h.item()), out[0].numel() // hp.CAND_DTYPE.itemsize)
            nb = n * hp.CAND_DTYPE.itemsize
            if nb:
                res[:nb].copy_(out[0][:nb], non_blocking=True)
            stream.synchronize()
            if it >= args.warmup:
                d2h.append(8 + nb)
        cs.synchronize()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = [e2e_s, float(np.mean(d2h))]
        del bufs

    dev_ms, e2e_s = max_over_ranks([dev_ms, e2e[0] if e2e else 0.0], dist, "cuda")
    units = w.ndm * nout
    line = None
    if rank == 0:
        value = aggregate(world, units, dev_ms * 1e-3)
        clocks = clk.summary()
        adds = float(w.ndm) * o.nchans * nout
        dd_ms = stats["stage_ms"]["dedisp"] / max(1, stats["stage_calls"]["dedisp"])
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded noise + dispersed pulses, shaped like a FAST file)",
            "config": describe(w, nout),
            "rtf": world * o.duration / (dev_ms * 1e-3),
            "clusters": ncl,
            "recovery": recovery,
            "stages_ms": {k: v / max(1, stats["stage_calls"][k])
                          for k, v in stats["stage_ms"].items()},
            "gpu_launches": stats["kernel_launches"],
            "rfi_stage_ms": rfi_ms,
        }
        if fused is not None:
            fused["unfused_ms_per_step"] = dev_ms
            fused["unfused_stages_ms"] = line["stages_ms"]
            fused["note"] = ("HP_PARAM_FUSE_LEVELS = 1: the dedispersion epilogue forms the "
                             "second remedian level, the remedian no longer reads D; off by "
                             "default (the fused kernel instance's summation loop is slower)")
            line["fused_levels"] = fused
        peaks = hp.hp_measure_peaks()
        sm_mhz = clocks["sm_mhz"] or 0.0
        # ALU roofline: 16-bit x 2 SWAR lanes give two byte-adds per 32-bit lane
        # operation, so the add peak is twice the measured 32-bit add issue rate
        peak_adds = 2.0 * peaks["int_add_ops_per_s"]
        achieved = adds / (dd_ms * 1e-3)
        cfg = int(plan.get_param("dedisp_config"))
        traffic = dedisp_traffic(w, cfg)
        alg_bytes = float(o.nchans) * o.nsamps + 4.0 * w.ndm * nout
        hbm_peak = measured_hbm_gbs()
        line["roofline"] = {
            "bound": "alu", "kernel": "dedisp_rows_kernel", "achieved": achieved / 1e12,
            "peak": peak_adds / 1e12, "unit": "Tadd/s", "frac": achieved / peak_adds,
            "traffic": traffic,
            "algorithmic": f"{w.ndm} trials x {o.nchans} ch x {nout} samples = {adds:.3e} "
                           f"byte-adds per launch; {alg_bytes:.3e} algorithmic bytes (input "
                           f"once + int32 output)",
            "traffic_over_algorithmic": traffic / alg_bytes if traffic else None,
            "hbm": {"achieved_gbs": traffic / (dd_ms * 1e-3) / 1e9 if traffic else None,
                    "peak_gbs": hbm_peak, "basis": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            # each 4-sample word costs prmt_per_word ALU-pipe PRMTs (align, then
            # one or two splits); the measured PRMT rate is the ALU pipe's rate
            "frac_vs_alu_design_ceiling": achieved / (peaks["prmt_ops_per_s"] * 4.0
                                                      / PRMT_PER_WORD),
            "config": cfg,
            "peak_basis": "measured int32 add issue rate x 2 (16-bit SWAR lanes); "
                          f"int32 {peaks['int_add_ops_per_s'] / 1e12:.2f} Tops/s, PRMT "
                          f"{peaks['prmt_ops_per_s'] / 1e12:.2f} Tops/s, LDS.32 "
                          f"{peaks['lds32_bytes_per_s'] / 1e12:.2f} TB/s, "
                          f"{peaks['sm_count']} SMs",
            "frac_vs_int32_rate": achieved / peaks["int_add_ops_per_s"],
        }
        # shared-memory loads: NW + 1 row words per lane, channel and trial for NW
        # words of 4 samples (byte-row kernels), against the measured LDS.32 rate
        shape = hp.hp_dedisp_config(cfg)
        if True:
            lds_bytes = adds * (shape["NW"] + 1) / shape["NW"]
            line["roofline"]["lds"] = {
                "achieved_tbs": lds_bytes / (dd_ms * 1e-3) / 1e12,
                "peak_tbs": peaks["lds32_bytes_per_s"] / 1e12,
                "frac": lds_bytes / (dd_ms * 1e-3) / peaks["lds32_bytes_per_s"],
                "basis": f"{shape['NW'] + 1} LDS.32 per {shape['NW']} words of 4 samples per "
                         "(trial, channel); measured conflict-free LDS.32 rate"}
        # the per-trial stages: the histogram pass reads D and writes y, the
        # detect pass reads y (the remedian reads D once more at 1/5 of the
        # rate it walks); per (trial, sample) nw threshold tests + 1 prefix add
        se_ms = stats["stage_ms"]["search"] / max(1, stats["stage_calls"]["search"])
        se_bytes = 4.0 * w.ndm * nout * 3
        se_ops = float(w.ndm) * nout * (w.nw + 1)
        line["search_roofline"] = {
            "bound": "hbm", "kernels": "remedian, mad_hist, refine, sigma, detect, tail",
            "frac": se_bytes / (se_ms * 1e-3) / 1e9 / hbm_peak,
            "achieved_gbs": se_bytes / (se_ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm_peak,
            "hbm_frac": se_bytes / (se_ms * 1e-3) / 1e9 / hbm_peak,
            "achieved_tops": se_ops / (se_ms * 1e-3) / 1e12,
            "int32_peak_tops": peaks["int_add_ops_per_s"] / 1e12,
            "alu_frac": se_ops / (se_ms * 1e-3) / peaks["int_add_ops_per_s"],
            "algorithmic": f"{se_bytes:.3e} B (D read, y written, y read) and {se_ops:.3e} "
                           f"integer ops ((nw + 1) per trial-sample) per search",
        }
        line["clocks"] = clocks
        if e2e:
            line["e2e"] = {"value": world * units / e2e_s, "unit": METRIC,
                           "h2d_bytes_per_step": int(s.data.nbytes), "d2h_bytes_per_step": int(e2e[1]),
                           "ms_per_step": e2e_s * 1e3,
                           "copies": "pinned host -> device every step, overlapped with the "
                                     "previous step's search (two input buffers)"}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(s, w)
    if world == 1 and not args.no_subband:
        line["subband"] = run_subband(args, hp, torch, stream, w, s, fb, cands, peaks, hbm_peak,
                                      dev_ms)
    if world == 1 and not args.no_width_sigma:
        line["width_sigma"] = run_width_sigma(args, hp, torch, stream, w, s, fb, cands, peaks,
                                              hbm_peak, dev_ms, stats)
    if world == 1 and not args.no_decimate:
        line["decimate"] = run_decimate(args, hp, torch, stream, w, s, fb, cands, dev_ms, stats)
    if world == 1 and not args.no_batch:
        del fb
        plan.close()
        torch.cuda.empty_cache()
        line["batch"] = run_batch(args, hp, torch, stream)
    if world == 1 and not args.no_configs:
        line["configs"] = run_configs(args, hp, torch, stream, peaks, hbm_peak)
    if world == 1 and not args.no_serve:
        line["serve"] = run_serve(args, hp, torch)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return line


# ------------------------------------------------ sub-band dedispersion
def best_match_snr(pulse, cands, w):
    """Largest S/N among the clusters that match an injected pulse (the
    position, DM and width criteria of workloads.recovered, any S/N)."""
    from paper_2512_00398_gb300.workloads import recovered
    best = 0.0
    for c in cands:
        if recovered(pulse, [c], w, snr_min=0.0):
            best = max(best, float(c["snr"]))
    return best


def run_subband(args, hp, torch, stream, w, s, fb, direct_cands, peaks, hbm_peak, direct_ms):
    """The sub-band variant (not the paper's method) on the same file: its
    throughput in the headline's units, its two stages against their rooflines,
    and what it costs in sensitivity: recovery and each injected pulse's best
    matched S/N against the direct search's."""
    S, G = (int(v) for v in args.subband.split(","))
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    plan.set_param("subband_chans", S)
    plan.set_param("subband_group", G)
    plan.bind_workspace(o.nsamps)
    nout = plan.nout(o.nsamps)
    out = hp.new_cand_buf(1 << 16)
    for _ in range(max(3, args.warmup)):
        hp.hp_search(plan, fb, stream, out=out)
    st = hp.hp_plan_sync_status(plan, stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "sub-band warm-up")
    cands = hp.cands_to_numpy(*out)
    hp.hp_plan_stats(plan, reset=True)
    plan.set_param("stage_timing", 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hp.hp_search(plan, fb, stream, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if hp.hp_plan_sync_status(plan, stream) != hp.HP_OK:
        raise hp.HPError(hp.hp_plan_sync_status(plan, stream), "sub-band timed region")
    stats = hp.hp_plan_stats(plan, reset=True)
    per = {k: v / args.steps for k, v in stats["stage_ms"].items()}   # summed over launches
    ratios = []
    for p in s.pulses:
        d0 = best_match_snr(p, direct_cands, w)
        if d0 > 0:
            ratios.append(best_match_snr(p, cands, w) / d0)
    nsub = -(-o.nchans // S)
    ngrp = -(-w.ndm // G)
    eff = plan.delays()
    top = eff[:, ::S].astype(np.int64)               # delay of each sub-band's first channel
    sb_len = nout + int(top.max())
    # stage 1: byte-adds at the nominal trials, each sub-band of each chunk of groups
    # over the samples stage 2 reads from it (nout + its largest first-channel delay)
    shape = hp.hp_dedisp_config(int(plan.get_param("dedisp_config")))
    gchunk = shape["RD"] * shape["WD"]                 # nominal trials per chunk
    widths_s = np.minimum(S, o.nchans - np.arange(nsub) * S)
    adds1 = 0.0
    for g0 in range(0, ngrp, gchunk):
        nd = min(gchunk, ngrp - g0)
        d_last = min((g0 + nd) * G, w.ndm) - 1
        adds1 += float(nd) * float(np.sum(widths_s * (nout + top[d_last])))
    adds2 = float(w.ndm) * nsub * nout               # stage 2: int32 adds of partial sums
    bytes2 = 4.0 * nsub * ngrp * sb_len + 4.0 * w.ndm * nout
    peak_adds = 2.0 * peaks["int_add_ops_per_s"]
    t1, t2 = per["dedisp"], per["subband_sum"]
    tr1, tr2 = subband_traffic(w, int(plan.get_param("dedisp_config")), S, G)
    plan.close()
    return {
        "what": "two-stage sub-band dedispersion (not the paper's method): identical to direct "
                "dedispersion with the effective delay table, bit-exact with the oracle's",
        "S": S, "G": G, "value": w.ndm * nout / (ms * 1e-3), "unit": METRIC,
        "ms_per_step": ms, "speedup_vs_direct": direct_ms / ms, "nout": nout,
        "stages_ms": per, "gpu_launches_per_step": stats["kernel_launches"] / args.steps,
        "recovery": recovery_rates(w, s.pulses, cands),
        "snr_vs_direct": {"min": min(ratios) if ratios else None,
                          "median": float(np.median(ratios)) if ratios else None,
                          "pulses": len(ratios)},
        "stage1_roofline": {"bound": "alu", "kernel": "dedisp_rows_kernel (segmented)",
                            "achieved": adds1 / (t1 * 1e-3) / 1e12, "peak": peak_adds / 1e12,
                            "unit": "Tadd/s", "frac": adds1 / (t1 * 1e-3) / peak_adds,
                            "traffic": tr1,
                            "algorithmic": f"{o.nchans} ch x {ngrp} nominal trials x (nout + the "
                                           f"sub-band's largest first-channel delay in its "
                                           f"chunk, at most {sb_len}) samples = {adds1:.3e} "
                                           f"byte-adds per step"},
        "stage2_roofline": {"bound": "hbm", "kernel": "subband_sum_kernel",
                            "achieved": bytes2 / (t2 * 1e-3) / 1e9, "peak": hbm_peak,
                            "unit": "GB/s", "frac": bytes2 / (t2 * 1e-3) / 1e9 / hbm_peak,
                            "traffic": tr2,
                            "traffic_over_algorithmic": tr2 / bytes2 if tr2 else None,
                            "adds_tops": adds2 / (t2 * 1e-3) / 1e12,
                            "algorithmic": f"partial sums read once ({nsub} x {ngrp} x {sb_len} "
                                           f"int32) + series written ({w.ndm} x {nout} int32) "
                                           f"= {bytes2:.3e} B per step; {adds2:.3e} adds"},
    }


# ------------------------------------------- per-width normalisation
def run_width_sigma(args, hp, torch, stream, w, s, fb, direct_cands, peaks, hbm_peak, direct_ms,
                    direct_stats):
    """The per-width normalisation variant (not the paper's reading) on the
    same file: throughput, the cost of the exact per-width medians, and what it
    changes: clusters, recovery and the injected pulses' matched S/N."""
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    plan.set_param("width_sigma", 1)
    plan.bind_workspace(o.nsamps)
    nout = plan.nout(o.nsamps)
    out = hp.new_cand_buf(1 << 16)
    for _ in range(max(3, args.warmup)):
        hp.hp_search(plan, fb, stream, out=out)
    if hp.hp_plan_sync_status(plan, stream) != hp.HP_OK:
        raise hp.HPError(hp.hp_plan_sync_status(plan, stream), "per-width warm-up")
    cands = hp.cands_to_numpy(*out)
    hp.hp_plan_stats(plan, reset=True)
    plan.set_param("stage_timing", 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hp.hp_search(plan, fb, stream, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    stats = hp.hp_plan_stats(plan, reset=True)
    per = {k: v / args.steps for k, v in stats["stage_ms"].items()}
    ratios = []
    for p in s.pulses:
        d0 = best_match_snr(p, direct_cands, w)
        if d0 > 0:
            ratios.append(best_match_snr(p, cands, w) / d0)
    direct_search = direct_stats["stage_ms"]["search"] / max(1, direct_stats["stage_calls"]["search"])
    extra = per["search"] - direct_search
    # the selection passes: every (trial, width, start) boxcar sum rebuilt and
    # counted once per histogram level (two levels on this data), y read per pass
    evals = 2.0 * w.ndm * nout * w.nw
    plan.close()
    return {
        "what": "per-width normalisation (not the paper's reading): sigma_k from the exact "
                "median of |S_k| per trial and width; threshold thr*sigma_k, S/N S/sigma_k",
        "value": w.ndm * nout / (ms * 1e-3), "unit": METRIC, "ms_per_step": ms,
        "vs_direct_ms_per_step": direct_ms, "stages_ms": per,
        "per_width_median_ms": extra,
        "gpu_launches_per_step": stats["kernel_launches"] / args.steps,
        "clusters": int(len(cands)), "clusters_direct": int(len(direct_cands)),
        "recovery": recovery_rates(w, s.pulses, cands),
        "snr_vs_direct": {"min": min(ratios) if ratios else None,
                          "median": float(np.median(ratios)) if ratios else None,
                          "pulses": len(ratios)},
        "median_passes": {"boxcar_evaluations": evals,
                          "achieved_gevals_per_s": evals / (extra * 1e-3) / 1e9 if extra > 0 else None,
                          "int32_peak_tops": peaks["int_add_ops_per_s"] / 1e12,
                          "note": "two histogram levels of exact radix selection per "
                                  "(trial, width): each rebuilds nw boxcar sums per sample "
                                  "from a shared-memory prefix and counts one digit"},
    }


# ------------------------------------------------ decimated boxcars
def run_decimate(args, hp, torch, stream, w, s, fb, direct_cands, direct_ms, direct_stats):
    """The decimated-boxcar variant (not the paper's method) on the same file:
    widths W > R that are multiples of R tested on the start grid W / R only."""
    o = w.obs
    R = int(args.decimate)
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    plan.set_param("decimate", R)
    plan.bind_workspace(o.nsamps)
    nout = plan.nout(o.nsamps)
    out = hp.new_cand_buf(1 << 16)
    for _ in range(max(3, args.warmup)):
        hp.hp_search(plan, fb, stream, out=out)
    if hp.hp_plan_sync_status(plan, stream) != hp.HP_OK:
        raise hp.HPError(hp.hp_plan_sync_status(plan, stream), "decimated warm-up")
    cands = hp.cands_to_numpy(*out)
    hp.hp_plan_stats(plan, reset=True)
    plan.set_param("stage_timing", 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hp.hp_search(plan, fb, stream, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    stats = hp.hp_plan_stats(plan, reset=True)
    per = {k: v / args.steps for k, v in stats["stage_ms"].items()}
    ratios = []
    for p in s.pulses:
        d0 = best_match_snr(p, direct_cands, w)
        if d0 > 0:
            ratios.append(best_match_snr(p, cands, w) / d0)
    direct_search = direct_stats["stage_ms"]["search"] / max(1, direct_stats["stage_calls"]["search"])
    plan.close()
    return {
        "what": "decimated boxcars (not the paper's method): widths W > R, multiples of R, "
                "tested on the start grid m*W/R (boxcars of R samples on the series summed "
                "in blocks of W/R)",
        "R": R, "value": w.ndm * nout / (ms * 1e-3), "unit": METRIC, "ms_per_step": ms,
        "vs_direct_ms_per_step": direct_ms, "search_ms": per["search"],
        "search_ms_direct": direct_search,
        "gpu_launches_per_step": stats["kernel_launches"] / args.steps,
        "clusters": int(len(cands)), "clusters_direct": int(len(direct_cands)),
        "recovery": recovery_rates(w, s.pulses, cands),
        "snr_vs_direct": {"min": min(ratios) if ratios else None,
                          "median": float(np.median(ratios)) if ratios else None,
                          "pulses": len(ratios)},
    }


# ------------------------------------------- the tiny and stress recipes
def time_plan(hp, torch, plan, fb, stream, steps, warmup, capacity=1 << 16):
    """ms per hp_search step (events around `steps` steps after `warmup`), then
    per-stage ms from `steps` more with stage timing; returns the candidates."""
    out = hp.new_cand_buf(capacity)
    for _ in range(warmup):
        hp.hp_search(plan, fb, stream, out=out)
    st = hp.hp_plan_sync_status(plan, stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "warm-up")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        hp.hp_search(plan, fb, stream, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    hp.hp_plan_stats(plan, reset=True)
    plan.set_param("stage_timing", 1)
    for _ in range(steps):
        hp.hp_search(plan, fb, stream, out=out)
    st = hp.hp_plan_sync_status(plan, stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "timed steps")
    stats = hp.hp_plan_stats(plan, reset=True)
    plan.set_param("stage_timing", 0)
    stages = {k: v / max(1, stats["stage_calls"][k]) for k, v in stats["stage_ms"].items()}
    return ms, stages, hp.cands_to_numpy(*out)


def config_line(w, ms, stages, cands, s, peaks, hbm_peak, nout):
    """Throughput, real-time factor, rooflines and recovery of one recipe."""
    o = w.obs
    adds = float(w.ndm) * o.nchans * nout
    se_bytes = 4.0 * w.ndm * nout * 3
    peak_adds = 2.0 * peaks["int_add_ops_per_s"]
    return {
        "value": w.ndm * nout / (ms * 1e-3), "unit": METRIC, "ms_per_step": ms,
        "rtf": o.duration / (ms * 1e-3), "stages_ms": stages,
        "roofline": {"bound": "alu", "kernel": "dedisp_rows_kernel",
                     "achieved": adds / (stages["dedisp"] * 1e-3) / 1e12,
                     "peak": peak_adds / 1e12, "unit": "Tadd/s",
                     "frac": adds / (stages["dedisp"] * 1e-3) / peak_adds},
        "search_roofline": {"bound": "hbm",
                            "achieved_gbs": se_bytes / (stages["search"] * 1e-3) / 1e9,
                            "peak_gbs": hbm_peak,
                            "frac": se_bytes / (stages["search"] * 1e-3) / 1e9 / hbm_peak},
        "clusters": int(len(cands)),
        "recovery": recovery_rates(w, s.pulses, cands),
    }


def run_configs(args, hp, torch, stream, peaks, hbm_peak):
    """The tiny recipe (128 ch, 32 768 samples, 100 trials) with the oracle timed
    on the whole file and its clusters compared, and the stress recipe (4096 ch,
    2^21 samples, ~4000 trials on DM 0-5000, boxcars to 8192, broadband spikes,
    narrowband tones and drift), searched plain and with RFI mitigation, the
    oracle timed on a sample of its trials."""
    import oracle
    from paper_2512_00398_gb300 import workloads
    res = {}
    # tiny: many steps (a search takes well under a millisecond)
    w = workloads.tiny()
    s = w.generate()
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    nout = plan.nout(o.nsamps)
    fb = torch.from_numpy(s.data).cuda()
    ms, stages, cands = time_plan(hp, torch, plan, fb, stream, 200, 20)
    line = config_line(w, ms, stages, cands, s, peaks, hbm_peak, nout)
    t = time.perf_counter()
    want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    dt = time.perf_counter() - t
    key = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
    line["oracle_equal"] = bool([key(c) for c in cands] == [key(c) for c in want.clusters] and
                                np.abs(cands["snr"].astype(np.float64)
                                       - want.clusters["snr"]).max() <= 1e-4)
    line["cpu_baseline"] = {"value": w.ndm * nout / dt, "unit": METRIC,
                            "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"the whole file (all {w.ndm} trials), {dt:.2f} s"}
    line["workload"] = (f"tiny: {o.nchans} ch, {o.nsamps} samples at {o.tsamp * 1e6:.0f} us, "
                        f"{w.ndm} trials on DM 0-400, boxcars 1..64, 3 pulses")
    res["tiny"] = line
    plan.close()
    del fb
    # stress: the raw list reaches ~6e7 (the drift's long-boxcar residuals)
    w = workloads.stress()
    s = w.generate(threads=min(16, os.cpu_count() or 8))
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                   raw_capacity=1 << 26)
    nout = plan.nout(o.nsamps)
    plan.bind_workspace(o.nsamps)
    fb = torch.from_numpy(s.data).cuda()
    ms, stages, cands = time_plan(hp, torch, plan, fb, stream, 2, 1, capacity=1 << 24)
    line = config_line(w, ms, stages, cands, s, peaks, hbm_peak, nout)
    plan.set_param("rfi", 1)
    ms_r, stages_r, cands_r = time_plan(hp, torch, plan, fb, stream, 2, 1, capacity=1 << 24)
    line["with_rfi_mitigation"] = {"value": w.ndm * nout / (ms_r * 1e-3), "ms_per_step": ms_r,
                                   "rfi_stage_ms": stages_r["rfi"], "clusters": int(len(cands_r)),
                                   "recovery": recovery_rates(w, s.pulses, cands_r)}
    plan.close()
    del fb
    torch.cuda.empty_cache()
    dt1, units1, _ = oracle_sample(s, w, 1)
    k = int(max(1, min(8, 12.0 / max(dt1, 1e-3))))
    dtk, unitsk, _ = oracle_sample(s, w, k)
    line["cpu_baseline"] = {"value": unitsk / dtk, "unit": METRIC, "cores": oracle.num_threads(),
                            "kind": "oracle",
                            "sample": f"{k} consecutive trials (of {w.ndm}) around the middle of "
                                      f"the DM range, full {o.nsamps} samples, {dtk:.1f} s "
                                      "(extrapolated to the whole file)"}
    line["workload"] = (f"stress: {o.nchans} ch, {o.nsamps} samples ({o.duration:.1f} s), "
                        f"{w.ndm} trials on DM 0-{float(w.dm_list[-1]):.0f}, boxcars 1..8192, "
                        f"{len(s.pulses)} pulses, spikes, tones and drift")
    res["stress"] = line
    del s
    return res


# ------------------------------------------------------ batched vs plain
def run_batch(args, hp, torch, stream):
    """The multi-file workload: 16 files of uneven length, channel count and
    sampling time, searched once file by file with hp_search and once as one
    autotuned, graph-captured hp_batch; both timed with events over the same
    number of passes, candidates compared file by file."""
    from paper_2512_00398_gb300 import workloads
    files = workloads.batch(nfiles=args.batch_files)
    fbs, plans, units, dur, nbytes = [], [], 0, 0.0, 0
    for w in files:
        o = w.obs
        s = w.generate(threads=min(16, os.cpu_count() or 8))
        fbs.append(torch.from_numpy(s.data).cuda())
        del s
        p = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
        p.bind_workspace(o.nsamps)
        plans.append(p)
        units += w.ndm * p.nout(o.nsamps)
        dur += o.duration
        nbytes += o.nchans * o.nsamps
    steps = max(1, args.steps)
    outs = [hp.new_cand_buf(1 << 16) for _ in files]

    def plain_pass():
        for p, fb, out in zip(plans, fbs, outs):
            hp.hp_search(p, fb, stream, out=out)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    plain_cfg = plans[0].get_param("dedisp_config")
    plain_ms = timed(plain_pass)
    for p in plans:
        st = hp.hp_plan_sync_status(p, stream)
        if st != hp.HP_OK:
            raise hp.HPError(st, "plain pass")
    want = [hp.cands_to_numpy(d, c) for d, c in outs]

    b = hp.Batch(plans)
    t = time.perf_counter()
    cfg, tune_ms = b.autotune(fbs, stream)
    tune_s = time.perf_counter() - t
    for p in plans:                                  # the plain path with the same tile shape
        p.set_param("dedisp_config", cfg)
    bouts = [hp.new_cand_buf(1 << 16) for _ in files]
    batch_ms = timed(lambda: b.search_async(fbs, stream, outs=bouts))
    st = b.sync_status(stream)
    if st != hp.HP_OK:
        raise hp.HPError(st, "batched pass")
    got = [hp.cands_to_numpy(d, c) for d, c in bouts]
    identical = all(np.array_equal(g, w_) for g, w_ in zip(got, want))
    # the spread: plain and batched passes alternated, each timed over `steps` passes
    reps = []
    for _ in range(5):
        pm = timed(plain_pass)
        bm = timed(lambda: b.search_async(fbs, stream, outs=bouts))
        reps.append((pm, bm))
    gains = sorted(pm / bm for pm, bm in reps)
    kernels = b.kernels_per_call()
    b.close()
    res = {
        "workload": f"{len(files)} files, {min(w.obs.nsamps for w in files)}-"
                    f"{max(w.obs.nsamps for w in files)} samples, 1024/2048/4096 ch, "
                    f"49.152/64 us, {files[0].ndm} trials on DM 0-1000 each, boxcars 1..4096, "
                    f"{nbytes / 1e9:.1f} GB input (larger than L2, no flush)",
        "units_per_pass": units, "duration_s": dur,
        "plain": {"value": units / (plain_ms * 1e-3), "ms_per_pass": plain_ms,
                  "rtf": dur / (plain_ms * 1e-3), "dedisp_config": plain_cfg},
        "batched": {"value": units / (batch_ms * 1e-3), "ms_per_pass": batch_ms,
                    "rtf": dur / (batch_ms * 1e-3), "dedisp_config": cfg,
                    "autotune_s": tune_s, "kernels_per_call": kernels, "cuda_graph": True},
        "gain": plain_ms / batch_ms,
        "gain_repeats": {"n": len(gains), "median": gains[len(gains) // 2], "min": gains[0],
                         "max": gains[-1],
                         "plain_ms": [pm for pm, _ in reps], "batched_ms": [bm for _, bm in reps],
                         "basis": "plain and batched passes alternated, same tile shape"},
        "identical_candidates": bool(identical),
        "clusters": int(sum(len(x) for x in want)),
        "steps": steps,
    }
    del fbs
    for p in plans:
        p.close()
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------- serving
class GulpMaker:
    """Every beam's gulps drawn on the device as they are needed: radiometer
    noise from torch's generator seeded per (beam, gulp), the beam's dispersed
    Gaussian pulses added (the signal model of synth: cold-plasma delays in
    continuous time, signal added before quantisation), rounded and clipped
    to uint8 and copied into a pinned host slot.  The serving measurement needs
    19 independent beams at the real-time rate (1.6 GB/s of data), more than the
    host generator makes; the device does it on a side stream in a few ms per
    gulp."""

    def __init__(self, torch, beams, G, slots_per_beam):
        self.torch = torch
        self.beams = beams
        self.G = G
        o = beams[0].obs
        self.nch = o.nchans
        self.stream = torch.cuda.Stream()
        self.spb = slots_per_beam
        self.slots = [[torch.empty((G, o.nchans), dtype=torch.uint8, pin_memory=True)
                       for _ in range(slots_per_beam)] for _ in beams]
        self.ready = [[None] * slots_per_beam for _ in beams]
        self.freqs = o.freqs()

    def make(self, b, g):
        """Start gulp g of beam b; returns its slot index."""
        torch = self.torch
        w = self.beams[b]
        o = w.obs
        G = self.G
        k = g % self.spb
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1000003 * (b + 1) + g)
        with torch.cuda.stream(self.stream):
            x = torch.randn((G, self.nch), generator=gen, device="cuda", dtype=torch.float32)
            x.mul_(o.sigma).add_(o.mean)
            t0 = g * G * o.tsamp
            t1 = (g + 1) * G * o.tsamp
            for p in w.pulses:
                tau = p.t0 + 4148.808 * p.dm * (self.freqs ** -2 - o.f_top ** -2)
                half = 4.0 * p.fwhm
                if tau.max() + half < t0 or tau.min() - half > t1:
                    continue
                rel = torch.from_numpy((tau - t0).astype(np.float32)).cuda()
                tt = torch.arange(G, device="cuda", dtype=torch.float32) * o.tsamp
                dt = (tt[:, None] - rel[None, :]) / p.fwhm
                x.add_(torch.exp(dt.square_().mul_(-4.0 * math.log(2.0))).mul_(p.amp))
            q = x.round_().clamp_(0, 255).to(torch.uint8)
            self.slots[b][k].copy_(q, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.ready[b][k] = ev
        return k

    def get(self, b, g):
        k = g % self.spb
        self.ready[b][k].synchronize()
        return self.slots[b][k]


def run_serve(args, hp, torch):
    """The 19-beam stream: 4096 ch, 49.152 us, DM 0-2000, gulps of 65 536
    samples (3.22 s), every beam its own data (GulpMaker) with about one
    injected pulse per beam-minute.  Phase 1 pushes every beam's gulps at the
    real-time rate (one gulp per beam every 3.22 s, each beam's arrival jittered
    by 0-20 ms) and reports the gulp latency (push -> candidates in host
    memory) and the injection recovery; phase 2 pushes a backlog of gulps at
    once and reports the sustained throughput."""
    import threading
    from paper_2512_00398_gb300 import workloads
    from paper_2512_00398_gb300.workloads import recovered
    G = 65536
    nb = args.serve_beams
    nb2 = 6                                           # backlog gulps per beam (phase 2)
    beams = workloads.serve(nbeams=nb, gulp=G, seconds=args.serve_seconds)
    w = beams[0]
    o = w.obs
    tg = G * o.tsamp
    ng = max(1, int(round(args.serve_seconds / tg)))
    maker = GulpMaker(torch, beams, G, slots_per_beam=nb2 + 2)
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    budget = 120 * (1 << 30)
    st = hp.Stream(plan, nbeams=nb, gulp=G, hbm_budget=budget, cand_capacity=4096)
    info0 = st.stats()
    H = info0["tail_samples"]
    done = [set() for _ in range(nb)]                 # gulps whose result came back
    lock = threading.Lock()
    cands = [[] for _ in range(nb)]

    def collect(n, out):
        while len(out) < n:
            r = st.poll(timeout_ms=600000)
            if r is None:
                raise RuntimeError("stream stalled")
            info, c = r
            if info["status"] != hp.HP_OK:
                raise hp.HPError(info["status"], "stream gulp")
            out.append(info)
            with lock:
                done[info["beam"]].add(info["gulp_index"])
            if len(c):
                cands[info["beam"]].append(c)

    def wait_slot(b, g):
        """Slot g % slots may be reused once gulp g - slots has come back."""
        old = g - maker.spb
        while old >= 0:
            with lock:
                if old in done[b]:
                    return
            time.sleep(0.001)

    # phase 1: real time, data made one gulp ahead
    rng = np.random.default_rng(17)
    jit = rng.uniform(0.0, 0.020, size=(ng, nb))
    for b in range(nb):
        maker.make(b, 0)
    res1 = []
    t0 = time.perf_counter() + 0.5

    def producer():
        for g in range(ng):
            for b in np.argsort(jit[g]):
                b = int(b)
                t = t0 + (g + 1) * tg + jit[g, b]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                st.push(b, maker.get(b, g))
            if g + 1 < ng:
                for b in range(nb):
                    wait_slot(b, g + 1)
                    maker.make(b, g + 1)

    th = threading.Thread(target=producer)
    th.start()
    collect(ng * nb, res1)
    th.join()
    searched = [r for r in res1 if r["window_len"] > 0]
    lat = np.array([r["latency_s"] for r in searched])
    units1 = sum(r["window_len"] for r in searched) * w.ndm
    # injection recovery over the real-time phase (pulses fully inside it)
    pulses, found = 0, 0
    for b in range(nb):
        cb = np.concatenate(cands[b]) if cands[b] else np.zeros(0, hp.CAND_DTYPE)
        for p in beams[b].pulses:
            if p.t0 + 5.0 > ng * tg or p.snr < 10.0:
                continue
            pulses += 1
            found += recovered(p, cb, beams[b], snr_min=w.threshold)
    # phase 2: a backlog of nb2 gulps per beam pushed at once
    res2 = []
    for g in range(ng, ng + nb2):
        for b in range(nb):
            wait_slot(b, g)
            maker.make(b, g)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for g in range(ng, ng + nb2):
        for b in range(nb):
            st.push(b, maker.get(b, g))
    collect(nb2 * nb, res2)
    wall2 = time.perf_counter() - t
    units2 = sum(r["window_len"] for r in res2) * w.ndm
    stats = st.stats()
    st.close()
    plan.close()
    del maker
    return {
        "workload": f"{nb} beams x {o.nchans} ch, {o.tsamp * 1e6:.3f} us, gulps of {G} samples "
                    f"({tg:.3f} s), {w.ndm} trials on DM 0-{float(w.dm_list[-1]):.0f}, boxcars "
                    f"1..{int(w.widths[-1])}, tail {H} samples, budget {budget >> 30} GiB; "
                    f"data: every beam and gulp drawn separately on the device (seeded "
                    f"noise + ~1 dispersed pulse per beam-minute), pinned host memory",
        "realtime": {"seconds": ng * tg, "gulps": len(res1), "searched": len(searched),
                     "latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                     "latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                     "latency_max_s": float(lat.max()) if lat.size else None,
                     "gulp_s": tg,
                     "rtf_p99": float(tg / np.percentile(lat, 99)) if lat.size else None,
                     "value": units1 / (ng * tg), "unit": METRIC,
                     "recovery_snr_ge_10": f"{found}/{pulses}"},
        "saturated": {"gulps": len(res2), "wall_s": wall2, "value": units2 / wall2,
                      "unit": METRIC, "rtf": len(res2) * tg / wall2},
        "steps": stats["steps"], "max_batch_seen": stats["max_batch_seen"],
        "beam_slots": stats["beam_slots"], "device_gib": stats["device_bytes"] / (1 << 30),
        "device_allocs_after_open": stats["device_allocs"] - info0["device_allocs"],
    }


# --------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import oracle
    w = workload(args.nsamps)
    s = w.generate(threads=min(16, os.cpu_count() or 8))
    dt1, _, nout = oracle_sample(s, w, 1)
    k = int(max(1, min(64, 8.0 / max(dt1, 1e-3))))
    for i in range(args.warmup):
        oracle_sample(s, w, k, d0=(i * k) % max(1, w.ndm - k))
    times = []
    for i in range(args.steps):
        dt, units, _ = oracle_sample(s, w, k, d0=((args.warmup + i) * k) % max(1, w.ndm - k))
        times.append(dt)
    step = float(np.mean(times))
    value = k * nout / step
    sample = (f"{k} consecutive trials (of {w.ndm}) per step, full {w.obs.nsamps} samples: "
              f"dedispersion + per-trial stages + merge")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": describe(w, nout),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
