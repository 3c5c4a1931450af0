"""GB300-native single-pulse search: the data-parallel hot path of Heimdall++
(arXiv 2512.00398) as hand-written sm_103a CUDA behind a small C ABI.

Python names mirror ``include/hp.h``.  Device buffers are torch CUDA tensors,
streams are torch CUDA streams (default: the current stream).  The functions
prefixed ``hp_`` are asynchronous like their C counterparts; ``search``,
``dedisperse``, ``detect`` and ``merge`` are conveniences that synchronise
and return host arrays.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import (CAND_DTYPE, EXPORTS, HP_ERR_CAND_OVERFLOW, HP_ERR_CUDA, HP_ERR_INVALID_ARG,
                   HP_ERR_NSAMPS_TOO_SHORT, HP_ERR_OOM, HP_ERR_TIMEOUT, HP_NUM_DEDISP_CONFIGS,
                   HP_NUM_STAGES, HP_OK, HP_PARAM_BASELINE_MODE, HP_PARAM_BASELINE_S,
                   HP_PARAM_DEDISP_CONFIG, HP_PARAM_DM_TOL, HP_PARAM_RAW_CAPACITY,
                   HP_PARAM_STAGE_TIMING, HP_PARAM_T_GAP, HP_PARAM_TIMEOUT_S, HP_PARAM_W_TOL,
                   HP_PARAM_RFI, HP_PARAM_RFI_NB_K, HP_PARAM_RFI_BB_K, HP_STAGE_RFI,
                   HP_PARAM_SUBBAND_CHANS, HP_PARAM_SUBBAND_GROUP, HP_PARAM_WIDTH_SIGMA,
                   HP_PARAM_DECIMATE, HP_PARAM_FUSE_LEVELS,
                   HP_STAGE_DEDISP, HP_STAGE_MERGE, HP_STAGE_SEARCH, HP_STAGE_TRANSPOSE, RAW_DTYPE,
                   STAGE_NAMES, HP_BATCH_MAX_FILES, HP_MERGE_STATIC_MAX_RAW, CandBuf, HPError, Peaks,
                   Stats, HP_STREAM_EMPTY, HP_STREAM_MAX_BEAMS, check, lib, status_str)
from . import _lib as _lib_mod

_PARAMS = {"baseline_mode": HP_PARAM_BASELINE_MODE, "baseline_s": HP_PARAM_BASELINE_S,
           "dm_tol": HP_PARAM_DM_TOL, "t_gap": HP_PARAM_T_GAP, "w_tol": HP_PARAM_W_TOL,
           "raw_capacity": HP_PARAM_RAW_CAPACITY, "dedisp_config": HP_PARAM_DEDISP_CONFIG,
           "stage_timing": HP_PARAM_STAGE_TIMING, "timeout_s": HP_PARAM_TIMEOUT_S,
           "rfi": HP_PARAM_RFI, "rfi_nb_k": HP_PARAM_RFI_NB_K, "rfi_bb_k": HP_PARAM_RFI_BB_K,
           "subband_chans": HP_PARAM_SUBBAND_CHANS, "subband_group": HP_PARAM_SUBBAND_GROUP,
           "width_sigma": HP_PARAM_WIDTH_SIGMA, "decimate": HP_PARAM_DECIMATE,
           "fuse_levels": HP_PARAM_FUSE_LEVELS}


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


class Plan:
    """Owning handle of an ``hp_plan`` (see ``hp_plan_create``)."""

    def __init__(self, nchans, f_top, chan_bw, tsamp, dm_list, widths, snr_threshold, **params):
        self.dm_list = np.ascontiguousarray(dm_list, dtype=np.float32)
        self.widths = np.ascontiguousarray(widths, dtype=np.int32)
        self.nchans = int(nchans)
        self.f_top, self.chan_bw, self.tsamp = float(f_top), float(chan_bw), float(tsamp)
        self.threshold = float(snr_threshold)
        h = C.c_void_p()
        check(lib().hp_plan_create(C.byref(h), self.nchans, self.f_top, self.chan_bw,
                                   self.tsamp, self.dm_list.ctypes.data_as(C.c_void_p),
                                   int(self.dm_list.size), self.widths.ctypes.data_as(C.c_void_p),
                                   int(self.widths.size), C.c_float(self.threshold)),
              "hp_plan_create")
        self._h = h
        self._ws = None
        for k, v in params.items():
            self.set_param(k, v)

    # -- handle ----------------------------------------------------------
    @property
    def handle(self):
        if self._h is None:
            raise HPError(HP_ERR_INVALID_ARG, "plan already destroyed")
        return self._h

    def use_allocator(self, alloc=None, free=None):
        """Take the plan's device memory from Python callables alloc(nbytes) ->
        int pointer and free(ptr, nbytes) (both None: cudaMalloc again)."""
        if (alloc is None) != (free is None):
            raise HPError(HP_ERR_INVALID_ARG, "alloc and free go together")
        if alloc is None:
            a, f = _lib_mod.ALLOC_FN(), _lib_mod.FREE_FN()
        else:
            a = _lib_mod.ALLOC_FN(lambda n, ctx: int(alloc(int(n))) or None)
            f = _lib_mod.FREE_FN(lambda ptr, n, ctx: free(int(ptr), int(n)))
        check(lib().hp_plan_set_allocator(self.handle, a, f, None), "hp_plan_set_allocator")
        self._alloc_cbs = (a, f)        # the library calls them until replaced

    def use_torch_allocator(self):
        """The plan's tables and workspace from torch's caching allocator."""
        import torch

        def alloc(n):
            return torch.cuda.caching_allocator_alloc(n)

        def free(ptr, n):
            torch.cuda.caching_allocator_delete(ptr)

        self.use_allocator(alloc, free)

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().hp_plan_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- parameters ------------------------------------------------------
    @property
    def ndm(self) -> int:
        return int(self.dm_list.size)

    @property
    def nw(self) -> int:
        return int(self.widths.size)

    def set_param(self, name, value):
        pid = _PARAMS[name] if isinstance(name, str) else int(name)
        check(lib().hp_plan_set_param(self.handle, pid, float(value)), f"hp_plan_set_param({name})")

    def get_param(self, name) -> float:
        pid = _PARAMS[name] if isinstance(name, str) else int(name)
        v = C.c_double()
        check(lib().hp_plan_get_param(self.handle, pid, C.byref(v)), f"hp_plan_get_param({name})")
        return v.value

    def delays(self) -> np.ndarray:
        out = np.empty((self.ndm, self.nchans), dtype=np.int32)
        check(lib().hp_plan_delays(self.handle, out.ctypes.data_as(C.c_void_p)), "hp_plan_delays")
        return out

    @property
    def max_delay(self) -> int:
        v = C.c_int32()
        check(lib().hp_plan_max_delay(self.handle, C.byref(v)), "hp_plan_max_delay")
        return int(v.value)

    def nout(self, nsamps: int) -> int:
        return int(nsamps) - self.max_delay

    def workspace_bytes(self, nsamps: int) -> int:
        v = C.c_size_t()
        check(lib().hp_plan_workspace_bytes(self.handle, int(nsamps), C.byref(v)),
              "hp_plan_workspace_bytes")
        return int(v.value)

    def bind_workspace(self, nsamps: int, device=None):
        """Allocate the scratch for inputs of ``nsamps`` samples as a torch
        tensor and bind it, so the library itself allocates nothing."""
        torch = _torch()
        need = self.workspace_bytes(nsamps)
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
            self._ws = torch.empty(need, dtype=torch.uint8, device=dev)
        check(lib().hp_plan_bind_workspace(self.handle, C.c_void_p(self._ws.data_ptr()),
                                           self._ws.numel()), "hp_plan_bind_workspace")
        return self._ws


# ------------------------------------------------------------------ C names
def hp_plan_create(nchans, f_top_MHz, chan_bw_MHz, tsamp_s, dm_list, boxcar_widths,
                   snr_threshold, **params) -> Plan:
    return Plan(nchans, f_top_MHz, chan_bw_MHz, tsamp_s, dm_list, boxcar_widths, snr_threshold,
                **params)


def hp_plan_destroy(plan: Plan):
    plan.close()


def _check_fb(plan: Plan, fb):
    torch = _torch()
    if not (isinstance(fb, torch.Tensor) and fb.is_cuda and fb.dtype == torch.uint8
            and fb.dim() == 2 and fb.shape[1] == plan.nchans and fb.is_contiguous()):
        raise HPError(HP_ERR_INVALID_ARG, "filterbank must be a contiguous CUDA uint8 "
                                          "tensor [nsamps, nchans]")


def new_cand_buf(capacity: int, device=None):
    """Device storage for ``capacity`` hp_cand records plus their count."""
    torch = _torch()
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    data = torch.empty(max(1, capacity) * CAND_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    return data, count


def _buf(data, count, capacity) -> CandBuf:
    return CandBuf(C.c_void_p(data.data_ptr()), int(capacity), C.c_void_p(count.data_ptr()))


def hp_search(plan: Plan, filterbank, stream=None, out=None, capacity: int = 1 << 16):
    """Enqueue the whole search; returns the device (data, count) pair."""
    _check_fb(plan, filterbank)
    data, count = out if out is not None else new_cand_buf(capacity, filterbank.device)
    cap = data.numel() // CAND_DTYPE.itemsize
    b = _buf(data, count, cap)
    check(lib().hp_search(plan.handle, C.c_void_p(filterbank.data_ptr()), int(filterbank.shape[0]),
                          _stream_ptr(stream), C.byref(b)), "hp_search")
    return data, count


def hp_dedisperse(plan: Plan, filterbank, stream=None, out=None):
    """Enqueue dedispersion; returns an int32 [ndm, pitch] tensor (nout valid)."""
    torch = _torch()
    _check_fb(plan, filterbank)
    nout = plan.nout(filterbank.shape[0])
    if nout <= int(plan.widths[-1]):
        raise HPError(HP_ERR_NSAMPS_TOO_SHORT, "hp_dedisperse")
    if out is None:
        pitch = (nout + 3) // 4 * 4
        out = torch.empty((plan.ndm, pitch), dtype=torch.int32, device=filterbank.device)
    check(lib().hp_dedisperse(plan.handle, C.c_void_p(filterbank.data_ptr()),
                              int(filterbank.shape[0]), C.c_void_p(out.data_ptr()),
                              int(out.stride(0)), _stream_ptr(stream)), "hp_dedisperse")
    return out


def hp_detect(plan: Plan, series, nout: int, stream=None, capacity: int = 1 << 20):
    """Enqueue the per-trial stages on dedispersed rows; returns
    (raw data, raw count, sigma, mad) device tensors."""
    torch = _torch()
    dev = series.device
    raw = torch.empty(max(1, capacity) * RAW_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    sigma = torch.empty(plan.ndm, dtype=torch.float64, device=dev)
    mad = torch.empty(plan.ndm, dtype=torch.int64, device=dev)
    b = CandBuf(C.c_void_p(raw.data_ptr()), int(capacity), C.c_void_p(cnt.data_ptr()))
    check(lib().hp_detect(plan.handle, C.c_void_p(series.data_ptr()), int(nout),
                          int(series.stride(0)), _stream_ptr(stream), C.byref(b),
                          C.c_void_p(sigma.data_ptr()), C.c_void_p(mad.data_ptr())), "hp_detect")
    return raw, cnt, sigma, mad


def hp_merge(plan: Plan, raw, raw_count, sigma, stream=None, out=None, capacity: int = 1 << 16):
    """Enqueue merging of device raw candidates; returns (data, count)."""
    data, count = out if out is not None else new_cand_buf(capacity, raw.device)
    cap = data.numel() // CAND_DTYPE.itemsize
    b = _buf(data, count, cap)
    raw_cap = raw.numel() // RAW_DTYPE.itemsize
    check(lib().hp_merge(plan.handle, C.c_void_p(raw.data_ptr()), C.c_void_p(raw_count.data_ptr()),
                         int(raw_cap), C.c_void_p(sigma.data_ptr()), _stream_ptr(stream),
                         C.byref(b)), "hp_merge")
    return data, count


def hp_merge_static(raw, raw_count, sigma, widths, dm_tol=1, t_gap=0, w_tol=None, stream=None,
                    out=None, capacity: int = 1 << 16, status=None):
    """Merge device raw candidates without any device allocation by the
    library (its scratch is a fixed array built into the library); for
    callers that must not allocate.  ``status``: optional device int32 tensor
    (set to 0 by the caller) in which a raw count beyond the buffer is
    reported.  Returns the device (data, count) pair."""
    data, count = out if out is not None else new_cand_buf(capacity, raw.device)
    cap = data.numel() // CAND_DTYPE.itemsize
    b = _buf(data, count, cap)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    raw_cap = raw.numel() // RAW_DTYPE.itemsize
    check(lib().hp_merge_static(C.c_void_p(raw.data_ptr()), C.c_void_p(raw_count.data_ptr()),
                                int(raw_cap), C.c_void_p(sigma.data_ptr()),
                                w.ctypes.data_as(C.c_void_p), int(w.size), int(dm_tol), int(t_gap),
                                int(w.size if w_tol is None else w_tol), _stream_ptr(stream),
                                C.byref(b),
                                C.c_void_p(status.data_ptr() if status is not None else None)),
          "hp_merge_static")
    return data, count


def hp_rfi_clean(plan: Plan, filterbank, stream=None, cleaned: bool = True):
    """RFI mitigation alone: returns (cleaned uint8 [nsamps][nchans] or None,
    channel flags, sample flags, channel medians) as device tensors."""
    import torch
    _check_fb(plan, filterbank)
    n = int(filterbank.shape[0])
    dev = filterbank.device
    out = torch.empty_like(filterbank) if cleaned else None
    cf = torch.empty(plan.nchans, dtype=torch.uint8, device=dev)
    sf = torch.empty(n, dtype=torch.uint8, device=dev)
    med = torch.empty(plan.nchans, dtype=torch.int32, device=dev)
    check(lib().hp_rfi_clean(plan.handle, C.c_void_p(filterbank.data_ptr()), n, _stream_ptr(stream),
                             C.c_void_p(out.data_ptr()) if out is not None else None,
                             C.c_void_p(cf.data_ptr()), C.c_void_p(sf.data_ptr()),
                             C.c_void_p(med.data_ptr())), "hp_rfi_clean")
    return out, cf, sf, med


def hp_width_sigmas(plan: Plan, stream=None):
    """Per-width sigmas and MADs ([ndm][nw] device tensors) of the plan's last
    search in the per-width mode."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    sg = torch.empty((plan.ndm, plan.nw), dtype=torch.float64, device=dev)
    md = torch.empty((plan.ndm, plan.nw), dtype=torch.int64, device=dev)
    check(lib().hp_width_sigmas(plan.handle, C.c_void_p(sg.data_ptr()), C.c_void_p(md.data_ptr()),
                                _stream_ptr(stream)), "hp_width_sigmas")
    return sg, md


def hp_plan_autotune(plan: Plan, filterbank, stream=None):
    """Time every dedispersion tile shape on this input and keep the fastest;
    returns (config, ms)."""
    _check_fb(plan, filterbank)
    cfg, ms = C.c_int(0), C.c_float(0.0)
    check(lib().hp_plan_autotune(plan.handle, C.c_void_p(filterbank.data_ptr()),
                                 int(filterbank.shape[0]), _stream_ptr(stream), C.byref(cfg),
                                 C.byref(ms)), "hp_plan_autotune")
    return int(cfg.value), float(ms.value)


class Batch:
    """Owning handle of an ``hp_batch``: several files searched as one launch
    sequence (captured into a CUDA graph after the first call)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = C.c_void_p()
        check(lib().hp_batch_create(C.byref(h), arr, len(self.plans)), "hp_batch_create")
        self._h = h
        self._bufs = None

    @property
    def handle(self):
        if self._h is None:
            raise HPError(HP_ERR_INVALID_ARG, "batch already destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().hp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, config: int):
        check(lib().hp_batch_set_config(self.handle, int(config)), "hp_batch_set_config")

    @staticmethod
    def _arrays(filterbanks):
        fbs = (C.c_void_p * len(filterbanks))(*[fb.data_ptr() for fb in filterbanks])
        ns = (C.c_int64 * len(filterbanks))(*[int(fb.shape[0]) for fb in filterbanks])
        return fbs, ns

    def autotune(self, filterbanks, stream=None):
        fbs, ns = self._arrays(filterbanks)
        cfg, ms = C.c_int(0), C.c_float(0.0)
        check(lib().hp_batch_autotune(self.handle, fbs, ns, _stream_ptr(stream), C.byref(cfg),
                                      C.byref(ms)), "hp_batch_autotune")
        return int(cfg.value), float(ms.value)

    def search_async(self, filterbanks, stream=None, outs=None, capacity: int = 1 << 16):
        """Enqueue the batch; returns the list of device (data, count) pairs."""
        if len(filterbanks) != len(self.plans):
            raise HPError(HP_ERR_INVALID_ARG, "one filterbank per plan")
        for p, fb in zip(self.plans, filterbanks):
            _check_fb(p, fb)
        if outs is None:
            outs = [new_cand_buf(capacity, fb.device) for fb in filterbanks]
        bufs = (CandBuf * len(outs))(*[_buf(d, c, d.numel() // CAND_DTYPE.itemsize)
                                       for d, c in outs])
        fbs, ns = self._arrays(filterbanks)
        check(lib().hp_batch_search(self.handle, fbs, ns, _stream_ptr(stream), bufs),
              "hp_batch_search")
        return outs

    def sync_status(self, stream=None) -> int:
        return int(lib().hp_batch_sync_status(self.handle, _stream_ptr(stream)))

    def kernels_per_call(self) -> int:
        k = C.c_int64(0)
        check(lib().hp_batch_kernels_per_call(self.handle, C.byref(k)), "hp_batch_kernels_per_call")
        return int(k.value)

    def search(self, filterbanks, stream=None, capacity: int = 1 << 16):
        """Search every file and return one merged-candidate array per file."""
        outs = self.search_async(filterbanks, stream, capacity=capacity)
        st = self.sync_status(stream)
        if st != HP_OK:
            raise HPError(st, "hp_batch_search (device)")
        return [cands_to_numpy(d, c) for d, c in outs]


class Stream:
    """Owning handle of an ``hp_stream``: beams pushed gulp by gulp, searched in
    batched steps by the library's scheduler thread, results polled back.

    A pushed gulp's host array is kept referenced here until its result has
    been polled (the library copies from it asynchronously)."""

    def __init__(self, plan: Plan, nbeams: int, gulp: int, hbm_budget: int = 0,
                 max_batch: int = 0, cand_capacity: int = 4096, raw_capacity: int = 1 << 18):
        cfg = _lib_mod.StreamConfig(int(nbeams), int(max_batch), int(gulp), int(hbm_budget),
                                    int(cand_capacity), int(raw_capacity))
        h = C.c_void_p()
        check(lib().hp_stream_open(C.byref(h), plan.handle, C.byref(cfg)), "hp_stream_open")
        self._h = h
        self.nchans = plan.nchans
        self.gulp = int(gulp)
        self.cand_capacity = int(cand_capacity)
        self._held = {}
        self._next = [0] * int(nbeams)

    @property
    def handle(self):
        if self._h is None:
            raise HPError(HP_ERR_INVALID_ARG, "stream already closed")
        return self._h

    def push(self, beam: int, gulp):
        """gulp: uint8 [gulp][nchans], a numpy array or a (pinned) CPU tensor."""
        if hasattr(gulp, "data_ptr"):
            ptr, n = gulp.data_ptr(), gulp.shape[0]
            ok = gulp.is_contiguous() and gulp.numel() == self.gulp * self.nchans
        else:
            gulp = np.ascontiguousarray(gulp, dtype=np.uint8)
            ptr, n = gulp.ctypes.data, gulp.shape[0]
            ok = gulp.size == self.gulp * self.nchans
        if not ok:
            raise HPError(HP_ERR_INVALID_ARG, "gulp must be [gulp][nchans] contiguous uint8")
        check(lib().hp_stream_push(self.handle, int(beam), C.c_void_p(ptr), int(n)),
              "hp_stream_push")
        self._held[(int(beam), self._next[beam])] = gulp
        self._next[beam] += 1

    def end_beam(self, beam: int):
        check(lib().hp_stream_end_beam(self.handle, int(beam)), "hp_stream_end_beam")

    def poll(self, timeout_ms: int = -1):
        """Next finished gulp as (info dict, candidates), or None on timeout."""
        r = _lib_mod.GulpResult()
        out = np.empty(self.cand_capacity, dtype=CAND_DTYPE)
        rc = lib().hp_stream_poll(self.handle, C.byref(r), out.ctypes.data_as(C.c_void_p),
                                  self.cand_capacity, int(timeout_ms))
        if rc == HP_STREAM_EMPTY:
            return None
        check(rc, "hp_stream_poll")
        self._held.pop((int(r.beam), int(r.gulp_index)), None)
        info = {f: getattr(r, f) for f, _ in _lib_mod.GulpResult._fields_ if f != "pad_"}
        n = min(int(r.ncand), self.cand_capacity)
        return info, out[:n].copy()

    def stats(self) -> dict:
        st = _lib_mod.StreamStats()
        check(lib().hp_stream_get_stats(self.handle, C.byref(st)), "hp_stream_get_stats")
        return {f: getattr(st, f) for f, _ in _lib_mod.StreamStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().hp_stream_close(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def hp_plan_sync_status(plan: Plan, stream=None) -> int:
    return int(lib().hp_plan_sync_status(plan.handle, _stream_ptr(stream)))


def hp_plan_stats(plan: Plan, reset: bool = True) -> dict:
    """Per-stage event times (ms, summed) and launch counts since the last reset."""
    st = Stats()
    check(lib().hp_plan_stats(plan.handle, C.byref(st), int(bool(reset))), "hp_plan_stats")
    return {"stage_ms": {n: st.stage_ms[i] for i, n in enumerate(STAGE_NAMES)},
            "stage_calls": {n: int(st.stage_calls[i]) for i, n in enumerate(STAGE_NAMES)},
            "kernel_launches": int(st.kernel_launches), "device_allocs": int(st.device_allocs)}


def hp_dedisp_config(config: int) -> dict:
    """The shape of a dedispersion tile shape (no GPU needed)."""
    out = (C.c_int32 * 8)()
    check(lib().hp_dedisp_config(int(config), out), "hp_dedisp_config")
    keys = ("RD", "NW", "WD", "WT", "stage_bytes", "stages", "unroll", "threads")
    return dict(zip(keys, (int(v) for v in out)))


def hp_selftest_bounded_wait(limit_ns: int) -> dict:
    """Run the bounded-wait self-test on the current GPU (synchronous)."""
    out = (C.c_int32 * 4)()
    check(lib().hp_selftest_bounded_wait(int(limit_ns), out), "hp_selftest_bounded_wait")
    return {"status": int(out[0]), "warp0_ran_out": bool(out[1]), "warp1_gave_up": bool(out[2]),
            "completed_wait_ok": bool(out[3])}


def hp_measure_peaks() -> dict:
    """Integer-add, byte-permute and shared-memory load rates of the current GPU."""
    pk = Peaks()
    check(lib().hp_measure_peaks(C.byref(pk)), "hp_measure_peaks")
    return {"int_add_ops_per_s": pk.int_add_ops_per_s, "prmt_ops_per_s": pk.prmt_ops_per_s,
            "lds32_bytes_per_s": pk.lds32_bytes_per_s, "sm_count": int(pk.sm_count)}


# ------------------------------------------------------- host conveniences
def cands_to_numpy(data, count, dtype=CAND_DTYPE) -> np.ndarray:
    n = int(count.item())
    cap = data.numel() // dtype.itemsize
    m = min(n, cap)
    host = data[: m * dtype.itemsize].cpu().numpy()
    return host.view(dtype).copy()


def search(plan: Plan, filterbank, stream=None, capacity: int = 1 << 16) -> np.ndarray:
    """Search and return the merged candidates (synchronises)."""
    data, count = hp_search(plan, filterbank, stream, capacity=capacity)
    st = hp_plan_sync_status(plan, stream)
    if st != HP_OK:
        raise HPError(st, "hp_search (device)")
    n = int(count.item())
    if n > capacity:
        raise HPError(HP_ERR_CAND_OVERFLOW, f"hp_search: {n} clusters > capacity {capacity}")
    return cands_to_numpy(data, count)


def dedisperse(plan: Plan, filterbank, stream=None) -> np.ndarray:
    out = hp_dedisperse(plan, filterbank, stream)
    st = hp_plan_sync_status(plan, stream)
    if st != HP_OK:
        raise HPError(st, "hp_dedisperse (device)")
    return out[:, : plan.nout(filterbank.shape[0])].cpu().numpy()


def detect(plan: Plan, series, nout: int, stream=None, capacity: int = 1 << 20):
    raw, cnt, sigma, mad = hp_detect(plan, series, nout, stream, capacity)
    st = hp_plan_sync_status(plan, stream)
    if st != HP_OK:
        raise HPError(st, "hp_detect (device)")
    n = int(cnt.item())
    if n > capacity:
        raise HPError(HP_ERR_CAND_OVERFLOW, f"hp_detect: {n} raw candidates > {capacity}")
    return cands_to_numpy(raw, cnt, RAW_DTYPE), sigma.cpu().numpy(), mad.cpu().numpy()
