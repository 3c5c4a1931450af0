"""Pins of the streamed (gulp-by-gulp) oracle.

Sections III-B and V-C search long observations chunk by chunk with
overlapping time segments; the rule used for the overlap (each gulp searches
[tail | gulp] with a tail of maxd + Wmax - 1 samples, reports the runs whose
first start lies in its window and carries a per-(trial, width) "run open"
flag to the next gulp) is written out in hp_oracle.c.  These tests tie it to
an independent brute-force enumeration of runs, to the plain search (pinned
elsewhere) and to the injected signal.
"""
import math

import numpy as np
import pytest

import oracle

from test_oracle_pins import recovered


def _runs_brute(y, sigma, W, thr):
    """Maximal runs of above-threshold boxcar starts as (first, last, peak, S)."""
    S = np.convolve(y, np.ones(W, np.int64), mode="valid")
    lim = float(thr) * sigma * math.sqrt(W)
    above = [float(s) >= lim for s in S]
    runs, t = [], 0
    while t < len(S):
        if not above[t]:
            t += 1
            continue
        a = t
        while t < len(S) and above[t]:
            t += 1
        seg = S[a:t]
        p = a + int(np.argmax(seg))            # first maximum
        runs.append((a, t - 1, p, int(S[p])))
    return runs, above


def _window_brute(y, sigma, widths, thr, nwin, carry_in, t_offset):
    out, cout = [], []
    for k, W in enumerate(widths):
        if W > len(y) or not sigma > 0:
            cout.append(0)
            continue
        runs, above = _runs_brute(y, sigma, int(W), thr)
        cout.append(int(1 <= nwin <= len(above) and above[nwin - 1]))
        for a, _, p, s in runs:
            if a >= nwin or (a == 0 and carry_in is not None and carry_in[k]):
                continue
            out.append((k, p + t_offset, s))
    return sorted(out), cout


@pytest.mark.parametrize("seed", range(8))
def test_detect_window_bruteforce(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(40, 400))
    y = rng.integers(-30, 30, size=n).astype(np.int64)
    for _ in range(4):
        a = int(rng.integers(0, n - 5))
        y[a:a + int(rng.integers(1, 12))] += int(rng.integers(40, 150))
    y[0:3] += 120                                 # a run at start 0 for the carry rule
    widths = np.array([1, 2, 4, 8, 16], np.int32)
    sigma = float(rng.uniform(8, 30))
    thr = float(np.float32(rng.uniform(1.5, 4)))
    nwin = int(rng.integers(1, n - 15))
    cin = rng.integers(0, 2, size=widths.size).astype(np.uint8)
    off = int(rng.integers(0, 10 ** 6))
    for carry in (None, cin):
        raw, cout = oracle.detect_window(y, 3, sigma, widths, thr, nwin, carry, off)
        got = sorted((int(z["width_idx"]), int(z["sample"]), int(z["S"])) for z in raw)
        want, wcout = _window_brute(y, sigma, widths, thr, nwin, carry, off)
        assert got == want
        assert list(cout) == wcout
        assert (raw["dm_idx"] == 3).all()


def test_detect_window_whole_series_is_plain_detection():
    rng = np.random.default_rng(7)
    y = rng.integers(-40, 40, size=3000).astype(np.int64)
    y[[100, 1500, 2990]] += 400
    widths = np.array([1, 2, 4, 8, 64], np.int32)
    plain = oracle.detect_trial(y, 1, 20.0, widths, 4.0)
    raw, _ = oracle.detect_window(y, 1, 20.0, widths, 4.0, nwin=y.size)
    assert np.array_equal(np.sort(plain, order=["width_idx", "sample"]),
                          np.sort(raw, order=["width_idx", "sample"]))
    assert oracle.detect_window(y, 1, 0.0, widths, 4.0, nwin=10)[0].size == 0   # sigma 0


def test_carry_suppresses_a_continued_run_and_chains_across_gulps():
    # one long series, fixed sigma, windows of G starts with Wmax - 1 look-ahead
    rng = np.random.default_rng(11)
    G, widths = 50, np.array([1, 2, 4], np.int32)
    wmax = int(widths.max())
    y = rng.integers(-5, 5, size=8 * G + wmax - 1).astype(np.int64)
    y[G - 2:G + 1] += 100           # a run across the first boundary (starts 48..50)
    y[3 * G:3 * G + 2] += 100       # a run at the very start of window 3
    carry, got = None, []
    for g in range(8):
        buf = y[g * G:(g + 1) * G + wmax - 1]
        raw, carry = oracle.detect_window(buf, 0, 10.0, widths, 5.0, G, carry, g * G)
        got += [(int(z["width_idx"]), int(z["sample"]), int(z["S"])) for z in raw]
    # every run of the whole series whose first start is < 8 G appears once,
    # with the peak found inside the window's own buffer
    for k, W in enumerate(widths):
        runs, _ = _runs_brute(y, 10.0, int(W), 5.0)
        mine = sorted((s, S) for kk, s, S in got if kk == k)
        want = []
        for a, b, p, S in runs:
            if a >= 8 * G:
                continue
            g = a // G
            stop = min(b, (g + 1) * G + wmax - int(W) - 1 + 0)   # buffer end for width W
            seg = [int(np.sum(y[t:t + W])) for t in range(a, stop + 1)]
            q = a + int(np.argmax(seg))
            want.append((q, seg[q - a]))
        assert mine == sorted(want), k
    # the boundary run is reported by gulp 0 only; gulp 1 saw start 0 above with carry set
    assert sum(1 for k, s, _ in got if k == 0 and G - 3 <= s <= G + 1) == 1


def test_gulp_windows_partition_the_time_axis():
    for maxd, wmax, G in [(5019, 64, 4096), (93745, 4096, 65536), (10, 4, 1000), (0, 1, 7)]:
        H = maxd + wmax - 1
        nxt = 0
        for g in range(40):
            B0, E, nwin = oracle.gulp_geometry(g, G, maxd, wmax)
            if nwin <= 0:
                assert E <= H
                continue
            assert B0 == nxt                          # windows abut, starting at 0
            assert nwin == min(G, E - H)
            assert (E - B0) - maxd == nwin + wmax - 1  # look-ahead of Wmax - 1
            nxt = B0 + nwin


def test_single_gulp_is_plain_search_restricted_to_the_window(tiny_workload):
    w, s = tiny_workload
    o = w.obs
    tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list)
    maxd, wmax = int(tab.max()), int(w.widths.max())
    N = 3 * 4096
    x = s.data[:N]
    nwin = N - maxd - wmax + 1
    raw, cl, cout = oracle.search_window(x, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                                         w.threshold, nwin, 0)
    # expected: plain per-trial stages, runs kept by first start < nwin
    D = oracle.dedisperse(x, tab)
    win = oracle.baseline_window(2.0, o.tsamp)
    want = []
    for d in range(D.shape[0]):
        y = oracle.subtract_baseline(D[d], 0, win)
        sig = oracle.sigma_from_mad(oracle.mad(y))
        for k, W in enumerate(w.widths):
            runs, above = _runs_brute(y, sig, int(W), w.threshold)
            assert cout[d, k] == int(above[nwin - 1])
            want += [(d, k, p, S) for a, _, p, S in runs if a < nwin]
    got = sorted((int(z["dm_idx"]), int(z["width_idx"]), int(z["sample"]), int(z["S"]))
                 for z in raw)
    assert got == sorted(want) and len(got) > 0
    assert np.array_equal(cl, oracle.merge(raw, w.widths))


def test_stream_recovers_injected_pulses():
    from paper_2512_00398_gb300 import workloads
    beams = workloads.stream_tiny(nbeams=2, ngulps=8, gulp=4096)
    for w in beams:
        o = w.obs
        s = w.generate()
        res = oracle.stream_search(s.data, 4096, o.f_top, o.chan_bw, o.tsamp, w.dm_list,
                                   w.widths, w.threshold)
        cl = np.concatenate([r["clusters"] for r in res])
        tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list)
        end = oracle.gulp_geometry(7, 4096, int(tab.max()), int(w.widths.max()))
        searched_to = end[0] + end[2]
        for p in s.pulses:
            if p.t0 / o.tsamp + 64 < searched_to:      # fully inside the searched windows
                assert recovered(p, cl, w), p
        # every reported start lies in its own gulp's window
        for r in res:
            for c in r["raw"]:
                W = int(w.widths[c["width_idx"]])
                assert r["B0"] <= c["sample"] <= r["B0"] + r["nwin"] - 1 + (w.widths.max() - W)
