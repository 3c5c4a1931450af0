"""ctypes binding of the C ABI in ``include/hp.h`` (argument marshalling only).

Every step of the search runs in the CUDA library ``_build/libhp.so``; this
module only converts arguments, owns nothing but handles, and uses PyTorch
for device memory and streams.  There is no CPU fallback: if the library is
missing and cannot be built, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

HP_OK = 0
HP_ERR_INVALID_ARG = -1
HP_ERR_CUDA = -2
HP_ERR_OOM = -3
HP_ERR_CAND_OVERFLOW = -4
HP_ERR_TIMEOUT = -5
HP_ERR_NSAMPS_TOO_SHORT = -6

HP_PARAM_BASELINE_MODE = 0
HP_PARAM_BASELINE_S = 1
HP_PARAM_DM_TOL = 2
HP_PARAM_T_GAP = 3
HP_PARAM_W_TOL = 4
HP_PARAM_RAW_CAPACITY = 5
HP_PARAM_DEDISP_CONFIG = 6
HP_PARAM_STAGE_TIMING = 7
HP_PARAM_TIMEOUT_S = 8
HP_PARAM_RFI = 9
HP_PARAM_RFI_NB_K = 10
HP_PARAM_RFI_BB_K = 11
HP_PARAM_SUBBAND_CHANS = 12
HP_PARAM_SUBBAND_GROUP = 13
HP_PARAM_WIDTH_SIGMA = 14
HP_PARAM_DECIMATE = 15
HP_PARAM_FUSE_LEVELS = 16
HP_NUM_DEDISP_CONFIGS = 20

HP_STAGE_TRANSPOSE, HP_STAGE_DEDISP, HP_STAGE_SEARCH, HP_STAGE_MERGE, HP_STAGE_RFI = 0, 1, 2, 3, 4
HP_STAGE_SUBBAND_SUM = 5
HP_NUM_STAGES = 6
STAGE_NAMES = ("transpose", "dedisp", "search", "merge", "rfi", "subband_sum")

#: hp_cand (48 bytes)
CAND_DTYPE = np.dtype([("dm_idx", "<i4"), ("width_idx", "<i4"), ("sample", "<i8"),
                       ("snr", "<f4"), ("members", "<i4"), ("dm_lo", "<i4"), ("dm_hi", "<i4"),
                       ("t_lo", "<i8"), ("t_hi", "<i8")])
#: hp_raw_cand (24 bytes)
RAW_DTYPE = np.dtype([("dm_idx", "<i4"), ("width_idx", "<i4"), ("sample", "<i8"), ("S", "<i8")])
assert CAND_DTYPE.itemsize == 48 and RAW_DTYPE.itemsize == 24

#: every symbol include/hp.h and include/hp_bench.h declare
EXPORTS = ("hp_status_str", "hp_plan_create", "hp_plan_destroy", "hp_plan_set_param",
           "hp_plan_get_param", "hp_plan_delays", "hp_plan_max_delay", "hp_plan_workspace_bytes",
           "hp_plan_bind_workspace", "hp_search", "hp_dedisperse", "hp_detect", "hp_merge",
           "hp_plan_sync_status", "hp_plan_stats", "hp_measure_peaks", "hp_dedisp_config",
           "hp_selftest_bounded_wait", "hp_merge_static",
           "hp_plan_autotune", "hp_batch_create", "hp_batch_destroy", "hp_batch_set_config",
           "hp_batch_autotune", "hp_batch_search", "hp_batch_sync_status",
           "hp_batch_kernels_per_call", "hp_stream_open", "hp_stream_push", "hp_stream_end_beam",
           "hp_stream_poll", "hp_stream_get_stats", "hp_stream_close", "hp_plan_set_allocator", "hp_rfi_clean",
           "hp_width_sigmas")

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)

HP_STREAM_MAX_BEAMS = 1024
HP_STREAM_EMPTY = 1

HP_BATCH_MAX_FILES = 32

#: raw-candidate limit of hp_merge_static
HP_MERGE_STATIC_MAX_RAW = 65536


class HPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} ({code})")


class CandBuf(C.Structure):
    _fields_ = [("data", C.c_void_p), ("capacity", C.c_int64), ("count", C.c_void_p)]


class Peaks(C.Structure):
    _fields_ = [("int_add_ops_per_s", C.c_double), ("prmt_ops_per_s", C.c_double),
                ("lds32_bytes_per_s", C.c_double), ("sm_count", C.c_int), ("reserved", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("stage_ms", C.c_double * HP_NUM_STAGES), ("stage_calls", C.c_int64 * HP_NUM_STAGES),
                ("kernel_launches", C.c_int64), ("device_allocs", C.c_int64)]


class StreamConfig(C.Structure):
    _fields_ = [("nbeams", C.c_int32), ("max_batch", C.c_int32), ("gulp", C.c_int64),
                ("hbm_budget", C.c_int64), ("cand_capacity", C.c_int64),
                ("raw_capacity", C.c_int64)]


class GulpResult(C.Structure):
    _fields_ = [("beam", C.c_int32), ("status", C.c_int32), ("gulp_index", C.c_int64),
                ("window_start", C.c_int64), ("window_len", C.c_int64), ("ncand", C.c_int64),
                ("latency_s", C.c_double), ("batch_size", C.c_int32), ("pad_", C.c_int32)]


class StreamStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("gulps", C.c_int64), ("beam_slots", C.c_int32),
                ("max_batch", C.c_int32), ("admitted", C.c_int32), ("waiting", C.c_int32),
                ("device_bytes", C.c_int64), ("tail_samples", C.c_int64),
                ("max_batch_seen", C.c_int64), ("device_allocs", C.c_int64)]


_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
            L.hp_status_str.argtypes = [i32]
            L.hp_status_str.restype = C.c_char_p
            L.hp_plan_create.argtypes = [C.POINTER(vp), i32, dbl, dbl, dbl, vp, i32, vp, i32,
                                         C.c_float]
            L.hp_plan_destroy.argtypes = [vp]
            L.hp_plan_set_param.argtypes = [vp, i32, dbl]
            L.hp_plan_get_param.argtypes = [vp, i32, C.POINTER(dbl)]
            L.hp_plan_delays.argtypes = [vp, vp]
            L.hp_plan_max_delay.argtypes = [vp, C.POINTER(C.c_int32)]
            L.hp_plan_workspace_bytes.argtypes = [vp, i64, C.POINTER(C.c_size_t)]
            L.hp_plan_bind_workspace.argtypes = [vp, vp, C.c_size_t]
            L.hp_search.argtypes = [vp, vp, i64, vp, C.POINTER(CandBuf)]
            L.hp_dedisperse.argtypes = [vp, vp, i64, vp, i64, vp]
            L.hp_detect.argtypes = [vp, vp, i64, i64, vp, C.POINTER(CandBuf), vp, vp]
            L.hp_merge.argtypes = [vp, vp, vp, i64, vp, vp, C.POINTER(CandBuf)]
            L.hp_plan_sync_status.argtypes = [vp, vp]
            L.hp_plan_stats.argtypes = [vp, C.POINTER(Stats), i32]
            L.hp_measure_peaks.argtypes = [C.POINTER(Peaks)]
            L.hp_dedisp_config.argtypes = [C.c_int, C.c_void_p]
            L.hp_selftest_bounded_wait.argtypes = [C.c_int64, C.c_void_p]
            L.hp_merge_static.argtypes = [vp, vp, i64, vp, vp, i32, i32, i64, i32, vp,
                                          C.POINTER(CandBuf), vp]
            L.hp_plan_autotune.argtypes = [vp, vp, i64, vp, C.POINTER(i32), C.POINTER(C.c_float)]
            L.hp_batch_create.argtypes = [C.POINTER(vp), vp, i32]
            L.hp_batch_destroy.argtypes = [vp]
            L.hp_batch_set_config.argtypes = [vp, i32]
            L.hp_batch_autotune.argtypes = [vp, vp, vp, vp, C.POINTER(i32), C.POINTER(C.c_float)]
            L.hp_batch_search.argtypes = [vp, vp, vp, vp, vp]
            L.hp_batch_sync_status.argtypes = [vp, vp]
            L.hp_batch_kernels_per_call.argtypes = [vp, C.POINTER(i64)]
            L.hp_stream_open.argtypes = [C.POINTER(vp), vp, C.POINTER(StreamConfig)]
            L.hp_stream_push.argtypes = [vp, i32, vp, i64]
            L.hp_stream_end_beam.argtypes = [vp, i32]
            L.hp_stream_poll.argtypes = [vp, C.POINTER(GulpResult), vp, i64, i32]
            L.hp_stream_get_stats.argtypes = [vp, C.POINTER(StreamStats)]
            L.hp_stream_close.argtypes = [vp]
            L.hp_plan_set_allocator.argtypes = [vp, ALLOC_FN, FREE_FN, vp]
            L.hp_rfi_clean.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
            L.hp_width_sigmas.argtypes = [vp, vp, vp, vp]
            for name in EXPORTS:
                if name != "hp_status_str":
                    getattr(L, name).restype = i32
            _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().hp_status_str(int(code)).decode()


def check(code: int, where: str):
    if code != HP_OK:
        raise HPError(code, where)
