"""Pins of the oracle's decimated boxcars (a variant the paper does not use).

With a decimation R, a width W > R that is a multiple of R is evaluated only at
the starts m * q, q = W / R: the boxcar of R samples on the series summed in
blocks of q.  These tests build that scrunched series in numpy and find the
runs on it, and check the reduction to every start when R is at least the
widest boxcar.
"""
import numpy as np
import pytest

import oracle


def _runs(S, lim):
    out, t = [], 0
    while t < S.size:
        if S[t] >= lim:
            e = t
            while e < S.size and S[e] >= lim:
                e += 1
            j = t + int(np.argmax(S[t:e]))
            out.append((j, int(S[j])))
            t = e
        else:
            t += 1
    return out


def _expected(y, widths, thr, sigma, R):
    got = []
    for k, W in enumerate(widths):
        W = int(W)
        q = W // R if (R > 0 and W > R and W % R == 0) else 1
        m = y.size // q
        ys = y[: m * q].reshape(m, q).sum(axis=1)          # the series scrunched by q
        L = W // q
        c = np.concatenate([[0], np.cumsum(ys)])
        S = c[L:] - c[:-L]                                   # boxcar of W / q on it
        lim = float(np.float32(thr)) * sigma * np.sqrt(float(W))
        got += [(k, j * q, s) for j, s in _runs(S.astype(np.float64), lim)
                if j * q <= y.size - W]
    return sorted(got)


@pytest.mark.parametrize("R", [2, 4, 16])
def test_decimated_detections_bruteforce(R):
    rng = np.random.default_rng(60 + R)
    n = 20000
    widths = np.array([1, 2, 4, 8, 16, 32, 64, 256], np.int32)
    D = np.rint(rng.normal(30000, 50, (2, n))).astype(np.int32)
    D[0, 4000:4040] += 120
    D[1, 9000:9300] += 40
    D[1, 15000:15003] += 500
    tsamp, thr = 1e-3, 6.0
    raw, sig, _ = oracle.search_trials(D, 0, tsamp, widths, thr, decimate=R)
    win = oracle.baseline_window(2.0, tsamp)
    for d in range(2):
        y = oracle.subtract_baseline(D[d], 0, win)
        want = _expected(y, widths, thr, sig[d], R)
        got = sorted((int(r["width_idx"]), int(r["sample"]), int(r["S"]))
                     for r in raw[raw["dm_idx"] == d])
        assert got == want
        assert len(want) > 0
    # the decimated widths report only grid starts
    for r in raw:
        W = int(widths[r["width_idx"]])
        if W > R and W % R == 0:
            assert int(r["sample"]) % (W // R) == 0


def test_decimation_at_least_the_widest_boxcar_is_every_start(tiny_workload):
    w, s = tiny_workload
    o = w.obs
    a = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    b = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                      decimate=int(w.widths.max()))
    assert np.array_equal(a.clusters, b.clusters)
    # a coarse grid still finds the injected pulses
    from paper_2512_00398_gb300 import workloads
    c = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                      decimate=8)
    for p in s.pulses:
        assert workloads.recovered(p, c.clusters, w, snr_min=w.threshold), p
