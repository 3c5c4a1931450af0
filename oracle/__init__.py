"""CPU oracle of the single-pulse search hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
(and its reference arm) may import this package.  The CUDA library under
``paper_2512_00398_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``hp_oracle.c`` (plain C, exact integers, FP64
statistics); this module compiles it with gcc and wraps it with ctypes and
numpy.  Each wrapper names the step of the pipeline (Section II-B and
Algorithm 1 of arXiv 2512.00398) that it defines.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhp_oracle.so")
_lock = threading.Lock()
_lib = None

RAW_DTYPE = np.dtype([("dm_idx", "<i4"), ("width_idx", "<i4"), ("sample", "<i8"),
                      ("S", "<i8"), ("snr", "<f8")])
CLUSTER_DTYPE = np.dtype([("dm_idx", "<i4"), ("width_idx", "<i4"), ("sample", "<i8"),
                          ("snr", "<f8"), ("members", "<i4"), ("dm_lo", "<i4"),
                          ("dm_hi", "<i4"), ("pad_", "<i4"), ("t_lo", "<i8"), ("t_hi", "<i8")])

OK, ERR_ARG, ERR_OVERFLOW, ERR_SHORT = 0, -1, -4, -6


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _P(t):
    return C.POINTER(t)


class _Params(C.Structure):
    _fields_ = [("nchans", C.c_int), ("f_top", C.c_double), ("chan_bw", C.c_double),
                ("tsamp", C.c_double), ("dm_list", _P(C.c_float)), ("ndm", C.c_int),
                ("widths", _P(C.c_int32)), ("nw", C.c_int), ("thr", C.c_float),
                ("baseline_mode", C.c_int), ("baseline_s", C.c_double), ("dm_tol", C.c_int),
                ("t_gap", C.c_int64), ("w_tol", C.c_int), ("subband_chans", C.c_int),
                ("subband_group", C.c_int), ("width_sigma", C.c_int), ("decimate", C.c_int)]


def lib():
    """The compiled oracle.  ``HPO_ORACLE_LIB`` may name another build of the
    same source (the mutation test loads deliberately broken copies this way)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("HPO_ORACLE_LIB") or build()
            L = C.CDLL(path)
            vp = C.c_void_p
            L.hpo_num_threads.restype = C.c_int
            L.hpo_delays.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, vp, C.c_int, vp]
            L.hpo_max_delay.argtypes = [vp, C.c_int, C.c_int]
            L.hpo_max_delay.restype = C.c_int32
            L.hpo_dedisperse_rows.argtypes = [vp, C.c_int64, C.c_int, vp, C.c_int, C.c_int,
                                              C.c_int64, vp]
            L.hpo_subband_delays.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]
            L.hpo_width_sigma.argtypes = [vp, C.c_int64, vp, C.c_int, vp, vp]
            L.hpo_dedisperse_point.argtypes = [vp, C.c_int, vp, C.c_int64]
            L.hpo_dedisperse_point.restype = C.c_int64
            L.hpo_remedian_levels.argtypes = [C.c_int64]
            L.hpo_remedian.argtypes = [vp, C.c_int64, C.c_int, vp]
            L.hpo_remedian.restype = C.c_int64
            L.hpo_baseline_median.argtypes = [vp, C.c_int64, C.c_int, vp]
            L.hpo_baseline_mean.argtypes = [vp, C.c_int64, C.c_int64, vp]
            L.hpo_mad.argtypes = [vp, C.c_int64]
            L.hpo_mad.restype = C.c_int64
            L.hpo_sigma_from_mad.argtypes = [C.c_int64]
            L.hpo_sigma_from_mad.restype = C.c_double
            L.hpo_detect_trial.argtypes = [vp, C.c_int64, C.c_int, C.c_double, vp, C.c_int,
                                           C.c_float, vp, C.c_int64, vp]
            L.hpo_sort_raw.argtypes = [vp, C.c_int64]
            L.hpo_raw_snr.argtypes = [vp, C.c_int64, vp, vp]
            L.hpo_merge.argtypes = [vp, C.c_int64, vp, C.c_int, C.c_int64, C.c_int, vp,
                                    C.c_int64, vp]
            L.hpo_baseline_window.argtypes = [C.c_double, C.c_double]
            L.hpo_baseline_window.restype = C.c_int64
            L.hpo_subtract_baseline.argtypes = [vp, C.c_int64, C.c_int, C.c_int64, vp]
            L.hpo_search_trials.argtypes = [vp, C.c_int64, C.c_int, C.c_int, _P(_Params), vp,
                                            C.c_int64, vp, vp, vp]
            L.hpo_search.argtypes = [vp, C.c_int64, _P(_Params), vp, C.c_int64, vp, vp,
                                     C.c_int64, vp, vp, vp]
            L.hpo_detect_window.argtypes = [vp, C.c_int64, C.c_int, C.c_double, vp, C.c_int,
                                            C.c_float, C.c_int64, vp, vp, C.c_int64, vp,
                                            C.c_int64, vp]
            L.hpo_search_window.argtypes = [vp, C.c_int64, _P(_Params), C.c_int64, C.c_int64,
                                            vp, vp, vp, C.c_int64, vp, vp, C.c_int64, vp]
            L.hpo_rfi_clean.argtypes = [vp, C.c_int64, C.c_int, C.c_int, C.c_float, C.c_int,
                                        C.c_double, C.c_double, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().hpo_num_threads())


# ---------------------------------------------------------------- c1 delays
def delays(nchans, f_top, chan_bw, tsamp, dm_list) -> np.ndarray:
    """Delay table int32[ndm][nchans] (cold-plasma law, rint)."""
    dm = np.ascontiguousarray(dm_list, dtype=np.float32)
    out = np.empty((dm.size, nchans), dtype=np.int32)
    rc = lib().hpo_delays(int(nchans), float(f_top), float(chan_bw), float(tsamp), _ptr(dm),
                          int(dm.size), _ptr(out))
    if rc:
        raise ValueError(f"hpo_delays rc={rc}")
    return out


def subband_delays(delay_table: np.ndarray, S: int, G: int) -> np.ndarray:
    """Effective table of two-stage (sub-band) dedispersion: sub-bands of S
    channels, groups of G trials with nominal trial g*G + (len-1)//2;
    e[d][c] = delay[d][top] + delay[n][c] - delay[n][top] (top = c//S*S,
    n = the nominal trial of d's group).  A variant of step c2."""
    dt = np.ascontiguousarray(delay_table, dtype=np.int32)
    ndm, nch = dt.shape
    out = np.empty_like(dt)
    rc = lib().hpo_subband_delays(_ptr(dt), int(ndm), int(nch), int(S), int(G), _ptr(out))
    if rc:
        raise ValueError(f"hpo_subband_delays rc={rc}")
    return out


# ---------------------------------------------------------- c2 dedispersion
def dedisperse(x: np.ndarray, delay_table: np.ndarray, rows=None, nout=None) -> np.ndarray:
    """D[d][t] = sum_c x[t + delay[d][c]][c] for the requested trial rows."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    dt = np.ascontiguousarray(delay_table, dtype=np.int32)
    nsamps, nch = x.shape
    ndm = dt.shape[0]
    if nout is None:
        nout = nsamps - int(dt.max(initial=0))
    d0, d1 = (0, ndm) if rows is None else rows
    out = np.empty((d1 - d0, nout), dtype=np.int32)
    rc = lib().hpo_dedisperse_rows(_ptr(x), int(nsamps), int(nch), _ptr(dt), int(d0), int(d1),
                                   int(nout), _ptr(out))
    if rc:
        raise ValueError(f"hpo_dedisperse_rows rc={rc}")
    return out


def dedisperse_point(x: np.ndarray, delay_row: np.ndarray, t: int) -> int:
    row = np.ascontiguousarray(delay_row, dtype=np.int32)
    return int(lib().hpo_dedisperse_point(_ptr(x), int(x.shape[1]), _ptr(row), int(t)))


# ------------------------------------------------------------- c3 baseline
def remedian_levels(win: int) -> int:
    return int(lib().hpo_remedian_levels(int(win)))


def baseline_window(baseline_s: float, tsamp: float) -> int:
    return int(lib().hpo_baseline_window(float(baseline_s), float(tsamp)))


def remedian(D: np.ndarray, L: int) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.int32)
    m = np.empty(max(1, -(-D.size // (5 ** L))), dtype=np.int64)
    n = lib().hpo_remedian(_ptr(D), int(D.size), int(L), _ptr(m))
    return m[:n]


def baseline_median(D: np.ndarray, L: int) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.int32)
    b = np.empty(D.size, dtype=np.int64)
    rc = lib().hpo_baseline_median(_ptr(D), int(D.size), int(L), _ptr(b))
    if rc:
        raise ValueError(rc)
    return b


def baseline_mean(D: np.ndarray, H: int) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.int32)
    b = np.empty(D.size, dtype=np.int64)
    rc = lib().hpo_baseline_mean(_ptr(D), int(D.size), int(H), _ptr(b))
    if rc:
        raise ValueError(rc)
    return b


def subtract_baseline(D: np.ndarray, mode: int, win: int) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.int32)
    y = np.empty(D.size, dtype=np.int64)
    rc = lib().hpo_subtract_baseline(_ptr(D), int(D.size), int(mode), int(win), _ptr(y))
    if rc:
        raise ValueError(rc)
    return y


# -------------------------------------------------------- c4 normalisation
def width_sigma(y: np.ndarray, widths):
    """Per-width MAD_k = lower median of |S_k(t)| over all starts and
    sigma_k = 1.482602218505602 * MAD_k (a variant of step c4)."""
    y = np.ascontiguousarray(y, dtype=np.int64)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    m = np.empty(w.size, np.int64)
    sg = np.empty(w.size, np.float64)
    rc = lib().hpo_width_sigma(_ptr(y), int(y.size), _ptr(w), int(w.size), _ptr(m), _ptr(sg))
    if rc:
        raise ValueError(f"hpo_width_sigma rc={rc}")
    return m, sg


def mad(y: np.ndarray) -> int:
    y = np.ascontiguousarray(y, dtype=np.int64)
    return int(lib().hpo_mad(_ptr(y), int(y.size)))


def sigma_from_mad(m: int) -> float:
    return float(lib().hpo_sigma_from_mad(int(m)))


# ------------------------------------------------- c5 + c6 boxcar + peaks
def detect_trial(y: np.ndarray, d: int, sigma: float, widths, thr: float,
                 cap: int = 1 << 20) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.int64)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    out = np.empty(cap, dtype=RAW_DTYPE)
    n = C.c_int64(0)
    rc = lib().hpo_detect_trial(_ptr(y), int(y.size), int(d), float(sigma), _ptr(w), int(w.size),
                                float(thr), _ptr(out), int(cap), C.byref(n))
    if rc:
        raise ValueError(f"hpo_detect_trial rc={rc} n={n.value}")
    return out[: n.value].copy()


# ---------------------------------------------------------------- c7 merge
def sort_raw(c: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=RAW_DTYPE).copy()
    lib().hpo_sort_raw(_ptr(c), int(c.size))
    return c


def raw_with_snr(raw, sigma, widths) -> np.ndarray:
    """Raw candidates given as (dm_idx, width_idx, sample, S) with their S/N
    filled in from the per-trial sigmas (step c5): snr = S / (sigma_d sqrt(W))."""
    raw = np.asarray(raw)
    c = np.zeros(raw.size, dtype=RAW_DTYPE)
    for f in ("dm_idx", "width_idx", "sample", "S"):
        c[f] = raw[f]
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    if c.size:
        if c["dm_idx"].min() < 0 or c["dm_idx"].max() >= sg.size:
            raise ValueError("dm_idx outside the sigma array")
        if c["width_idx"].min() < 0 or c["width_idx"].max() >= w.size:
            raise ValueError("width_idx outside the width list")
    lib().hpo_raw_snr(_ptr(c), int(c.size), _ptr(sg), _ptr(w))
    return c


def merge(raw: np.ndarray, widths, dm_tol: int = 1, t_gap: int = 0, w_tol: int | None = None):
    c = np.ascontiguousarray(raw, dtype=RAW_DTYPE).copy()
    w = np.ascontiguousarray(widths, dtype=np.int32)
    if w_tol is None:
        w_tol = int(w.size)
    out = np.empty(max(1, c.size), dtype=CLUSTER_DTYPE)
    n = C.c_int64(0)
    rc = lib().hpo_merge(_ptr(c), int(c.size), _ptr(w), int(dm_tol), int(t_gap), int(w_tol),
                         _ptr(out), int(out.size), C.byref(n))
    if rc:
        raise ValueError(rc)
    return out[: n.value].copy()


# ------------------------------------------------------------ whole path
@dataclass
class SearchResult:
    raw: np.ndarray          # RAW_DTYPE, sorted by (dm_idx, sample, width_idx)
    clusters: np.ndarray     # CLUSTER_DTYPE
    sigma: np.ndarray        # float64 [ndm]
    mad: np.ndarray          # int64 [ndm]


def _params(nchans, f_top, chan_bw, tsamp, dm_list, widths, thr, baseline_mode, baseline_s,
            dm_tol, t_gap, w_tol, subband=None, width_sigma=False, decimate=0):
    dm = np.ascontiguousarray(dm_list, dtype=np.float32)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p = _Params(int(nchans), float(f_top), float(chan_bw), float(tsamp),
                dm.ctypes.data_as(_P(C.c_float)), int(dm.size), w.ctypes.data_as(_P(C.c_int32)),
                int(w.size), float(thr), int(baseline_mode), float(baseline_s), int(dm_tol),
                int(t_gap), int(w.size if w_tol is None else w_tol),
                int(subband[0]) if subband else 0, int(subband[1]) if subband else 1,
                int(bool(width_sigma)), int(decimate))
    return p, (dm, w)


def search(x: np.ndarray, f_top, chan_bw, tsamp, dm_list, widths, thr, baseline_mode=0,
           baseline_s=2.0, dm_tol=1, t_gap=0, w_tol=None, cap=1 << 22,
           subband=None, width_sigma=False, decimate=0) -> SearchResult:
    """The whole hot path on a uint8[nsamps][nchans] filterbank.  subband=(S, G)
    dedisperses with the sub-band variant's effective table (subband_delays);
    width_sigma=True normalises every width by its own sigma (width_sigma());
    decimate=R evaluates widths W > R that are multiples of R only at the starts
    m * W / R (decimated boxcars)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    nsamps, nch = x.shape
    p, keep = _params(nch, f_top, chan_bw, tsamp, dm_list, widths, thr, baseline_mode,
                      baseline_s, dm_tol, t_gap, w_tol, subband, width_sigma, decimate)
    ndm = keep[0].size
    raw = np.empty(cap, dtype=RAW_DTYPE)
    cl = np.empty(cap, dtype=CLUSTER_DTYPE)
    sig = np.empty(ndm, dtype=np.float64)
    md = np.empty(ndm, dtype=np.int64)
    nr, nc = C.c_int64(0), C.c_int64(0)
    rc = lib().hpo_search(_ptr(x), int(nsamps), C.byref(p), _ptr(raw), int(cap), C.byref(nr),
                          _ptr(cl), int(cap), C.byref(nc), _ptr(sig), _ptr(md))
    if rc:
        raise ValueError(f"hpo_search rc={rc}")
    return SearchResult(raw[: nr.value].copy(), cl[: nc.value].copy(), sig, md)


def search_trials(D: np.ndarray, d_begin: int, tsamp, widths, thr, baseline_mode=0,
                  baseline_s=2.0, cap=1 << 22, width_sigma=False, decimate=0):
    """Per-trial stages (baseline, sigma, boxcars, peaks) on dedispersed rows."""
    D = np.ascontiguousarray(D, dtype=np.int32)
    nrows, nout = D.shape
    p, keep = _params(1, 1500.0, -1.0, tsamp, np.zeros(1, np.float32), widths, thr,
                      baseline_mode, baseline_s, 1, 0, None, None, width_sigma, decimate)
    raw = np.empty(cap, dtype=RAW_DTYPE)
    sig = np.empty(nrows, dtype=np.float64)
    md = np.empty(nrows, dtype=np.int64)
    nr = C.c_int64(0)
    rc = lib().hpo_search_trials(_ptr(D), int(nout), int(d_begin), int(nrows), C.byref(p),
                                 _ptr(raw), int(cap), C.byref(nr), _ptr(sig), _ptr(md))
    if rc:
        raise ValueError(f"hpo_search_trials rc={rc}")
    return raw[: nr.value].copy(), sig, md


# ----------------------------------------------------- c9 streamed search
def detect_window(y: np.ndarray, d: int, sigma: float, widths, thr: float, nwin: int,
                  carry_in=None, t_offset: int = 0, cap: int = 1 << 20):
    """Runs of one series reported by the window rule (Sections III-B, V-C;
    reading in hp_oracle.c).  Returns (raw candidates, carry_out[nw])."""
    y = np.ascontiguousarray(y, dtype=np.int64)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    cin = None if carry_in is None else np.ascontiguousarray(carry_in, dtype=np.uint8)
    cout = np.zeros(w.size, dtype=np.uint8)
    out = np.empty(cap, dtype=RAW_DTYPE)
    n = C.c_int64(0)
    rc = lib().hpo_detect_window(_ptr(y), int(y.size), int(d), float(sigma), _ptr(w),
                                 int(w.size), float(thr), int(nwin),
                                 None if cin is None else _ptr(cin), _ptr(cout), int(t_offset),
                                 _ptr(out), int(cap), C.byref(n))
    if rc:
        raise ValueError(f"hpo_detect_window rc={rc}")
    return out[: n.value].copy(), cout


def search_window(x: np.ndarray, f_top, chan_bw, tsamp, dm_list, widths, thr, nwin: int,
                  t_offset: int, carry_in=None, baseline_mode=0, baseline_s=2.0, dm_tol=1,
                  t_gap=0, w_tol=None, cap=1 << 22, width_sigma=False, subband=None):
    """One gulp's buffer searched with the window rule; returns (raw, clusters,
    carry_out[ndm][nw]).  width_sigma=True: per-width sigmas of the buffer;
    subband=(S, G): the sub-band variant's effective table."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    nsamps, nch = x.shape
    p, keep = _params(nch, f_top, chan_bw, tsamp, dm_list, widths, thr, baseline_mode,
                      baseline_s, dm_tol, t_gap, w_tol, subband, width_sigma)
    ndm, nw = keep[0].size, keep[1].size
    cin = None if carry_in is None else np.ascontiguousarray(carry_in, dtype=np.uint8)
    cout = np.zeros((ndm, nw), dtype=np.uint8)
    raw = np.empty(cap, dtype=RAW_DTYPE)
    cl = np.empty(cap, dtype=CLUSTER_DTYPE)
    nr, nc = C.c_int64(0), C.c_int64(0)
    rc = lib().hpo_search_window(_ptr(x), int(nsamps), C.byref(p), int(nwin), int(t_offset),
                                 None if cin is None else _ptr(cin), _ptr(cout), _ptr(raw),
                                 int(cap), C.byref(nr), _ptr(cl), int(cap), C.byref(nc))
    if rc:
        raise ValueError(f"hpo_search_window rc={rc}")
    return raw[: nr.value].copy(), cl[: nc.value].copy(), cout


def gulp_geometry(g: int, gulp: int, maxd: int, wmax: int):
    """Buffer of gulp g (Sections III-B, V-C; reading in hp_oracle.c):
    (B0, E, nwin) with input samples [B0, E) searched and boxcar starts
    [0, nwin) its window; nwin <= 0 means the gulp is not searched."""
    H = maxd + wmax - 1
    E = (g + 1) * gulp
    B0 = max(0, g * gulp - H)
    return B0, E, E - H - B0


def stream_search(x: np.ndarray, gulp: int, f_top, chan_bw, tsamp, dm_list, widths, thr,
                  baseline_mode=0, baseline_s=2.0, dm_tol=1, t_gap=0, w_tol=None, rfi=None,
                  width_sigma=False, subband=None):
    """A beam's whole series x[nsamps][nchans] searched gulp by gulp; the last
    partial gulp is dropped.  Returns one dict per gulp: g, B0, nwin, raw,
    clusters (samples in the beam's dedispersed time).  rfi=(nb_k, bb_k) cleans
    each searched buffer first (its own statistics, step c0); width_sigma=True
    normalises every width by its own sigma over the searched buffer;
    subband=(S, G) dedisperses with the sub-band variant (the gulp geometry then
    follows its effective table)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    nch = x.shape[1]
    tab = delays(nch, f_top, chan_bw, tsamp, dm_list)
    if subband:
        tab = subband_delays(tab, subband[0], subband[1])
    maxd = int(tab.max())
    wmax = int(np.max(widths))
    out, carry = [], None
    for g in range(x.shape[0] // gulp):
        B0, E, nwin = gulp_geometry(g, gulp, maxd, wmax)
        if nwin <= 0:
            out.append({"g": g, "B0": B0, "nwin": 0, "raw": np.empty(0, RAW_DTYPE),
                        "clusters": np.empty(0, CLUSTER_DTYPE)})
            continue
        buf = x[B0:E]
        if rfi is not None:
            buf = rfi_clean(buf, tsamp, rfi[0], rfi[1], baseline_mode, baseline_s).cleaned
        raw, cl, carry = search_window(buf, f_top, chan_bw, tsamp, dm_list, widths, thr,
                                       nwin, B0, carry, baseline_mode, baseline_s, dm_tol, t_gap,
                                       w_tol, width_sigma=width_sigma, subband=subband)
        out.append({"g": g, "B0": B0, "nwin": nwin, "raw": raw, "clusters": cl})
    return out


# ------------------------------------------------------------ c0 RFI mitigation
@dataclass
class RfiResult:
    cleaned: np.ndarray       # uint8 [nsamps][nchans]
    chan_flag: np.ndarray     # bool [nchans] narrowband channels
    samp_flag: np.ndarray     # bool [nsamps] broadband samples
    chan_median: np.ndarray   # int32 [nchans]
    sigma_z: float


def rfi_clean(x: np.ndarray, tsamp: float, nb_k: int = 5, bb_k: float = 5.0,
              baseline_mode: int = 0, baseline_s: float = 2.0) -> RfiResult:
    """Narrowband channel masking and zero-DM broadband excision (Sections
    II-B and III-C; reading in hp_oracle.c)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    nsamps, nch = x.shape
    out = np.empty_like(x)
    cf = np.zeros(nch, np.uint8)
    sf = np.zeros(nsamps, np.uint8)
    med = np.zeros(nch, np.int32)
    sg = C.c_double(0.0)
    rc = lib().hpo_rfi_clean(_ptr(x), int(nsamps), int(nch), int(nb_k), float(bb_k),
                             int(baseline_mode), float(baseline_s), float(tsamp), _ptr(out),
                             _ptr(cf), _ptr(sf), _ptr(med), C.byref(sg))
    if rc:
        raise ValueError(f"hpo_rfi_clean rc={rc}")
    return RfiResult(out, cf.astype(bool), sf.astype(bool), med, float(sg.value))
