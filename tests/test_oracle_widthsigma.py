"""Pins of the oracle's per-width normalisation (a variant of step c4).

MAD_k is the lower median of |S_k(t)| over every start; these tests check it
against a numpy brute force, the W = 1 reduction to the plain MAD, the sqrt(W)
law on white noise and its failure on a random walk, and the detections of the
search in this mode against candidate lists built independently in numpy.
"""
import numpy as np
import pytest

import oracle


def _brute_mad(y, W):
    c = np.concatenate([[0], np.cumsum(y.astype(np.int64))])
    S = c[W:] - c[:-W]
    a = np.sort(np.abs(S))
    return int(a[(a.size - 1) // 2])


@pytest.mark.parametrize("seed", range(4))
def test_bruteforce(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(50, 3000))
    y = rng.integers(-500, 500, n).astype(np.int64)
    y[rng.integers(0, n, 5)] += 20000
    widths = np.array(sorted({1, 2, 3, 7, int(rng.integers(1, n)), n - 1, n}), np.int32)
    m, s = oracle.width_sigma(y, widths)
    for k, W in enumerate(widths):
        assert m[k] == _brute_mad(y, int(W)), W
        assert s[k] == 1.482602218505602 * float(m[k])


def test_width_one_is_the_mad():
    rng = np.random.default_rng(3)
    y = rng.integers(-1000, 1000, 12345).astype(np.int64)
    m, _ = oracle.width_sigma(y, [1])
    assert m[0] == oracle.mad(y)


def test_sqrt_law_on_white_noise_and_growth_on_red_noise():
    rng = np.random.default_rng(8)
    widths = np.array([1, 4, 16, 64, 256], np.int32)
    y = np.rint(rng.normal(0, 1000, 400000)).astype(np.int64)
    _, s = oracle.width_sigma(y, widths)
    ratio = s / (s[0] * np.sqrt(widths))
    assert np.all(np.abs(ratio - 1) < 0.03), ratio
    # a random walk: wide boxcars see far more than sqrt(W) times the single-sample spread
    walk = y + np.cumsum(np.rint(rng.normal(0, 300, y.size))).astype(np.int64)
    walk -= int(np.median(walk))
    _, s2 = oracle.width_sigma(np.diff(np.concatenate([[0], walk])), widths)   # increments: white
    _, s3 = oracle.width_sigma(walk - np.convolve(walk, np.ones(4001) / 4001, "same").astype(np.int64),
                               widths)
    assert s3[-1] / (s3[0] * np.sqrt(256)) > 1.5
    assert np.all(s2 > 0)


def _expected_raw(y, widths, thr):
    """Runs of S_k >= thr * sigma_k, one candidate per run at its largest S
    (ties: the earliest), snr = S / sigma_k -- written out in numpy."""
    out = []
    c = np.concatenate([[0], np.cumsum(y.astype(np.int64))])
    for k, W in enumerate(widths):
        S = c[W:] - c[:-W]
        sk = 1.482602218505602 * float(_brute_mad(y, int(W)))
        if not sk > 0:
            continue
        above = S.astype(np.float64) >= float(np.float32(thr)) * sk
        t = 0
        while t < S.size:
            if above[t]:
                e = t
                while e < S.size and above[e]:
                    e += 1
                j = t + int(np.argmax(S[t:e]))
                out.append((k, j, int(S[j]), float(S[j]) / sk))
                t = e
            else:
                t += 1
    return sorted(out)


@pytest.mark.parametrize("seed", range(3))
def test_search_trials_detections_bruteforce(seed):
    """The per-trial stages in this mode: the baseline and y come from the
    pinned baseline step; the detections are checked against numpy."""
    rng = np.random.default_rng(40 + seed)
    n = 6000
    widths = np.array([1, 2, 4, 8, 16, 64], np.int32)
    D = np.rint(rng.normal(20000, 40, (2, n))).astype(np.int32)
    D[0, 1000:1010] += 200
    D[1, 3000:3064] += 60
    D[1, 5000:5001] += 400
    tsamp, thr = 1e-3, 6.0
    raw, _, _ = oracle.search_trials(D, 0, tsamp, widths, thr, width_sigma=True)
    win = oracle.baseline_window(2.0, tsamp)
    for d in range(2):
        y = oracle.subtract_baseline(D[d], 0, win)
        want = _expected_raw(y, widths, thr)
        got = sorted((int(r["width_idx"]), int(r["sample"]), int(r["S"]), float(r["snr"]))
                     for r in raw[raw["dm_idx"] == d])
        assert [g[:3] for g in got] == [w[:3] for w in want]
        assert np.allclose([g[3] for g in got], [w[3] for w in want], rtol=0, atol=1e-12)
        assert len(want) > 0


def test_search_mode_off_is_the_paper_reading(tiny_workload):
    w, s = tiny_workload
    o = w.obs
    a = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    b = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                      width_sigma=False)
    assert np.array_equal(a.clusters, b.clusters)
    # in the per-width mode the injected pulses are still found (white noise:
    # sigma_k close to sigma sqrt(W))
    from paper_2512_00398_gb300 import workloads
    c = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                      width_sigma=True)
    for p in s.pulses:
        assert workloads.recovered(p, c.clusters, w), p


def test_stream_window_with_width_sigma(tiny_workload):
    """One gulp's buffer in the per-width mode: runs of S_k >= thr * sigma_k with
    sigma_k from the buffer, kept when their first start lies in the window;
    carry flags = start nwin - 1 above threshold."""
    w, s = tiny_workload
    o = w.obs
    tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list)
    maxd, wmax = int(tab.max()), int(w.widths.max())
    N = 3 * 4096
    x = s.data[:N]
    nwin = N - maxd - wmax + 1
    raw, cl, cout = oracle.search_window(x, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                                         w.threshold, nwin, 0, width_sigma=True)
    D = oracle.dedisperse(x, tab)
    win = oracle.baseline_window(2.0, o.tsamp)
    thr = float(np.float32(w.threshold))
    want = []
    for d in range(D.shape[0]):
        y = oracle.subtract_baseline(D[d], 0, win)
        c = np.concatenate([[0], np.cumsum(y)])
        for k, W in enumerate(w.widths):
            S = c[W:] - c[:-W]
            sk = 1.482602218505602 * float(_brute_mad(y, int(W)))
            above = S.astype(np.float64) >= thr * sk if sk > 0 else np.zeros(S.size, bool)
            assert cout[d, k] == int(above[nwin - 1])
            t = 0
            while t < S.size:
                if not above[t]:
                    t += 1
                    continue
                e = t
                while e < S.size and above[e]:
                    e += 1
                if t < nwin:
                    j = t + int(np.argmax(S[t:e]))
                    want.append((d, k, j, int(S[j])))
                t = e
    got = sorted((int(z["dm_idx"]), int(z["width_idx"]), int(z["sample"]), int(z["S"]))
                 for z in raw)
    assert got == sorted(want) and len(got) > 0
