"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle step (Section II-B stages, Algorithm 1) to a closed
form, a hand-worked example (tests/golden), an invariant, a textbook or library
routine, or an independent brute-force formulation on tiny inputs, chosen so
that a dropped term, a wrong sign or index, a wrong rounding or an
off-by-one fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ---------------------------------------------------------------- c1 delays

def test_delay_worked_example():
    rows = _rows("delay_worked_example.txt")
    dms = np.array([float(r[0]) for r in rows], np.float32)
    want = np.array([int(r[2]) for r in rows])
    exact = np.array([float(r[1]) for r in rows])
    # the fixture's exact column is the closed form 4148.808 * 5/9 * 1e-6 / 1e-3 per DM unit
    assert np.allclose(exact, dms.astype(np.float64) * 4148.808 * 5.0 / 9.0 * 1e-3, rtol=1e-9)
    tab = oracle.delays(2, 1500.0, -500.0, 1e-3, dms)
    assert (tab[:, 0] == 0).all()
    assert (tab[:, 1] == want).all()


def test_delay_textbook_magnitude():
    # Lorimer & Kramer: dt ~= 4.15 ms * DM * (f_lo,GHz^-2 - f_hi,GHz^-2).  The 4.15
    # approximation differs from 4148.808 s MHz^2 by 0.03 %.
    nch, f_top, bw, ts = 128, 1500.0, -1.953125, 64e-6
    tab = oracle.delays(nch, f_top, bw, ts, np.array([400.0], np.float32))
    f_lo = (f_top + (nch - 1) * bw) / 1000.0
    approx = 4.15e-3 * 400 * (f_lo ** -2 - 1.5 ** -2) / ts
    assert abs(tab[0, -1] - approx) / approx < 1e-3
    assert tab[0, -1] == 5019


def test_delay_invariants():
    dms = np.concatenate([[0.0], np.sort(np.random.default_rng(3).uniform(0, 3000, 40))])
    tab = oracle.delays(512, 1500.0, -500.0 / 512, 49.152e-6, dms.astype(np.float32))
    assert (tab[0] == 0).all()                      # DM 0: no delay anywhere
    assert (tab[:, 0] == 0).all()                   # reference channel is f_top
    assert (np.diff(tab, axis=0) >= 0).all()        # non-decreasing in DM
    assert (np.diff(tab, axis=1) >= 0).all()        # non-decreasing as frequency falls
    # proportional to DM before rounding: |rint(a) - DM_ratio*rint(b)| stays within rounding
    r = tab[-1].astype(float) / max(float(dms[-1]), 1.0)
    r2 = tab[-2].astype(float) / float(dms[-2])
    assert np.all(np.abs(r - r2) <= 1.0 / float(dms[-2]) + 1.0 / float(dms[-1]) + 1e-12)


# --------------------------------------------------------- c2 dedispersion

def _tiny_band(nch=8):
    return dict(nchans=nch, f_top=1500.0, chan_bw=-40.0, tsamp=1e-3)


def test_dedisp_impulse_response():
    b = _tiny_band()
    dms = np.array([0.0, 5.0, 20.0, 50.0], np.float32)
    tab = oracle.delays(b["nchans"], b["f_top"], b["chan_bw"], b["tsamp"], dms)
    nsamps = 256
    nout = nsamps - int(tab.max())
    for c in range(b["nchans"]):
        for t0 in (nsamps - 1, int(tab.max()) + 3, 40):
            x = np.zeros((nsamps, b["nchans"]), np.uint8)
            x[t0, c] = 7
            D = oracle.dedisperse(x, tab)
            for d in range(dms.size):
                want = np.zeros(nout, np.int64)
                t = t0 - tab[d, c]
                if 0 <= t < nout:
                    want[t] = 7
                assert (D[d] == want).all(), (c, t0, d)


def test_dedisp_dm0_is_channel_sum_and_linear_shift():
    rng = np.random.default_rng(5)
    b = _tiny_band(16)
    dms = np.array([0.0, 3.0, 9.0, 31.0, 60.0], np.float32)
    tab = oracle.delays(b["nchans"], b["f_top"], b["chan_bw"], b["tsamp"], dms)
    x1 = rng.integers(0, 120, size=(300, 16), dtype=np.uint8)
    x2 = rng.integers(0, 120, size=(300, 16), dtype=np.uint8)
    D1, D2 = oracle.dedisperse(x1, tab), oracle.dedisperse(x2, tab)
    nout = D1.shape[1]
    assert (D1[0] == x1[:nout].astype(np.int64).sum(axis=1)).all()
    assert (oracle.dedisperse(x1 + x2, tab) == D1.astype(np.int64) + D2).all()
    k = 17
    xs = np.zeros_like(x1)
    xs[k:] = x1[:-k]
    Ds = oracle.dedisperse(xs, tab)
    assert (Ds[:, k:] == D1[:, : nout - k]).all()


def test_dedisp_bruteforce_gather():
    rng = np.random.default_rng(6)
    b = _tiny_band(8)
    dms = np.linspace(0, 80, 7).astype(np.float32)
    tab = oracle.delays(b["nchans"], b["f_top"], b["chan_bw"], b["tsamp"], dms)
    x = rng.integers(0, 256, size=(256, 8), dtype=np.uint8)
    D = oracle.dedisperse(x, tab)
    nout = 256 - int(tab.max())
    t = np.arange(nout)[:, None]
    for d in range(dms.size):
        brute = x[t + tab[d][None, :], np.arange(8)[None, :]].astype(np.int64).sum(axis=1)
        assert (D[d] == brute).all()
    assert oracle.dedisperse_point(x, tab[3], 11) == int(D[3, 11])


# ------------------------------------------------------------- c3 baseline

def test_remedian_levels():
    for win, L in [(0, 0), (1, 0), (4, 0), (5, 1), (24, 1), (25, 2), (124, 2), (125, 3),
                   (15624, 5), (15625, 6), (31250, 6), (78124, 6), (78125, 7)]:
        assert oracle.remedian_levels(win) == L, win
    assert oracle.baseline_window(2.0, 64e-6) == 31250


def test_baseline_worked_example():
    for row in _rows("baseline_worked_example.txt"):
        bar = row.index("|")
        L = int(row[1])
        series = np.array([int(v) for v in row[2:bar]], np.int32)
        want = np.array([int(v) for v in row[bar + 1:]])
        assert (oracle.baseline_median(series, L) == want).all(), row[0]


def _remedian_brute(vals, L):
    """Recursive remedian on Python lists (independent formulation)."""
    if L == 0:
        return list(vals)
    groups = [sorted(vals[i:i + 5]) for i in range(0, len(vals), 5)]
    return _remedian_brute([g[(len(g) - 1) // 2] for g in groups], L - 1)


def _baseline_brute(vals, L):
    m = _remedian_brute(vals, L)
    P = 5 ** L
    cen = [P * j + (P - 1) // 2 for j in range(len(m))]
    out = []
    for t in range(len(vals)):
        if t <= cen[0]:
            out.append(m[0])
        elif t >= cen[-1]:
            out.append(m[-1])
        else:
            j = max(i for i in range(len(cen)) if cen[i] <= t)
            out.append(m[j] + math.floor(Fraction((m[j + 1] - m[j]) * (t - cen[j]), P)))
    return out


@pytest.mark.parametrize("n,L", [(1, 1), (4, 1), (5, 1), (7, 1), (26, 2), (124, 2), (126, 2),
                                 (631, 3), (700, 4), (3000, 2)])
def test_baseline_median_bruteforce(n, L):
    rng = np.random.default_rng(n * 31 + L)
    D = rng.integers(-5000, 5000, size=n).astype(np.int32)
    assert (oracle.baseline_median(D, L) == np.array(_baseline_brute(D.tolist(), L))).all()
    assert (oracle.remedian(D, L) == np.array(_remedian_brute(D.tolist(), L))).all()


@pytest.mark.parametrize("n", [1, 24, 25, 26, 3124, 3125, 3126, 15625 + 17, 40000])
def test_remedian_levels_compose(n):
    """The remedian's levels compose: L levels over D equal L - 2 levels over the
    second-level values (medians of five medians of five, over groups of 25
    aligned samples, the trailing partial groups by their lower medians); the
    fused search forms those values first and runs the remaining levels on them."""
    rng = np.random.default_rng(n)
    D = rng.integers(0, 1 << 20, size=n).astype(np.int32)
    lv2 = oracle.remedian(D, 2)
    assert lv2.size == -(-n // 25)
    for g in (0, lv2.size - 1):
        grp = D[25 * g:25 * g + 25].tolist()
        meds = [sorted(grp[i:i + 5])[(len(grp[i:i + 5]) - 1) // 2] for i in range(0, len(grp), 5)]
        assert lv2[g] == sorted(meds)[(len(meds) - 1) // 2]
    for L in range(2, 7):
        assert np.array_equal(oracle.remedian(D, L), oracle.remedian(lv2.astype(np.int32), L - 2)), L


def test_baseline_median_monotone_and_ramp():
    L, P = 3, 125
    n = 8 * P
    # a non-decreasing series: each group median is its middle element, so the
    # level-L value of block j is the sample at its centre c_j
    D = np.sort(np.random.default_rng(2).integers(0, 10 ** 6, size=n)).astype(np.int32)
    m = oracle.remedian(D, L)
    assert (m == D[P * np.arange(8) + (P - 1) // 2]).all()
    # an integer ramp is reproduced exactly between the first and last centres
    for slope in (3, -7):
        D = (1000 + slope * np.arange(n)).astype(np.int32)
        b = oracle.baseline_median(D, L)
        c0, c1 = (P - 1) // 2, 7 * P + (P - 1) // 2
        assert (b[c0:c1 + 1] == D[c0:c1 + 1]).all()
        assert (b[:c0] == D[c0]).all() and (b[c1:] == D[c1]).all()


def test_baseline_median_constant_and_spike():
    D = np.full(3000, 424242, np.int32)
    assert (oracle.baseline_median(D, 3) == 424242).all()
    D2 = D.copy()
    D2[1234] += 10 ** 6
    assert (oracle.baseline_median(D2, 3) == 424242).all()


@pytest.mark.parametrize("n,H", [(1, 0), (10, 3), (257, 20), (1000, 999)])
def test_baseline_mean_bruteforce(n, H):
    D = np.random.default_rng(n + H).integers(-9000, 9000, size=n).astype(np.int32)
    want = [sum(D[max(0, t - H): t + H + 1].tolist()) // len(D[max(0, t - H): t + H + 1])
            for t in range(n)]
    assert (oracle.baseline_mean(D, H) == np.array(want)).all()


# -------------------------------------------------------- c4 normalisation

def test_mad_matches_sort_median():
    rng = np.random.default_rng(8)
    for n in (1, 2, 3, 10, 11, 1000, 1001):
        y = rng.integers(-10 ** 6, 10 ** 6, size=n)
        assert oracle.mad(y) == int(np.sort(np.abs(y))[(n - 1) // 2])
    assert oracle.sigma_from_mad(100) == pytest.approx(148.2602218505602, rel=0, abs=1e-12)


def test_sigma_unit_rms_on_gaussian():
    rng = np.random.default_rng(9)
    for s in (50.0, 768.0):
        y = np.rint(rng.normal(0, s, size=400_000)).astype(np.int64)
        sig = oracle.sigma_from_mad(oracle.mad(y))
        assert abs(np.std(y / sig) - 1.0) < 0.02


# --------------------------------------------------- c5 + c6 boxcar + peaks

def test_boxcar_worked_example():
    y = np.zeros(256, np.int64)
    y[100:108] = 10
    rows = _rows("boxcar_worked_example.txt")
    widths = np.array([int(r[0]) for r in rows], np.int32)
    c = oracle.detect_trial(y, 4, 1.0, widths, 6.0)
    assert c.size == len(rows)
    for r, cand in zip(rows, sorted(c, key=lambda z: z["width_idx"])):
        assert widths[cand["width_idx"]] == int(r[0])
        assert cand["sample"] == int(r[1]) and cand["S"] == int(r[2]) and cand["dm_idx"] == 4
        assert cand["snr"] == pytest.approx(float(r[3]), abs=1e-8)


def _detect_brute(y, sigma, widths, thr):
    out = []
    n = len(y)
    for k, W in enumerate(widths):
        if W > n:
            continue
        S = np.convolve(y, np.ones(W, np.int64), mode="valid")        # S[t] = sum y[t:t+W]
        lim = float(thr) * sigma * math.sqrt(W)
        above = np.array([float(s) >= lim for s in S])
        edges = np.diff(np.concatenate([[0], above.astype(int), [0]]))
        for a, b in zip(np.flatnonzero(edges == 1), np.flatnonzero(edges == -1)):
            t = a + int(np.argmax(S[a:b]))
            out.append((k, t, int(S[t])))
    return sorted(out)


@pytest.mark.parametrize("seed", range(6))
def test_detect_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(50, 600))
    y = rng.integers(-40, 40, size=n).astype(np.int64)
    for _ in range(3):
        a = int(rng.integers(0, n - 10))
        y[a:a + int(rng.integers(1, 10))] += int(rng.integers(30, 200))
    widths = np.array([1, 2, 3, 4, 8, 16, 64, 1000], np.int32)
    sigma = float(rng.uniform(10, 40))
    thr = float(np.float32(rng.uniform(1.5, 5)))
    c = oracle.detect_trial(y, 0, sigma, widths, thr)
    got = sorted((int(z["width_idx"]), int(z["sample"]), int(z["S"])) for z in c)
    assert got == _detect_brute(y, sigma, widths, thr)
    for z in c:
        assert z["snr"] == z["S"] / (sigma * math.sqrt(widths[z["width_idx"]]))


def test_detect_threshold_is_inclusive_and_sigma_zero():
    y = np.zeros(16, np.int64)
    y[5] = 4
    c = oracle.detect_trial(y, 0, 1.0, np.array([1], np.int32), 4.0)    # limit exactly 4.0
    assert c.size == 1 and c[0]["sample"] == 5
    y[5] = 3
    assert oracle.detect_trial(y, 0, 1.0, np.array([1], np.int32), 4.0).size == 0
    y[5] = 10 ** 6
    assert oracle.detect_trial(y, 0, 0.0, np.array([1], np.int32), 4.0).size == 0


def test_detect_ties_go_to_smallest_t():
    y = np.zeros(64, np.int64)
    y[[10, 20]] = 50                   # one run for W=16 covering both, two equal maxima
    c = oracle.detect_trial(y, 0, 1.0, np.array([16], np.int32), 2.0)
    assert c.size == 1 and c[0]["S"] == 100 and c[0]["sample"] == 5


# ---------------------------------------------------------------- c7 merge

def _merge_brute(raw, widths, dm_tol, t_gap, w_tol):
    n = len(raw)
    key = sorted(range(n), key=lambda i: (raw[i]["dm_idx"], raw[i]["sample"], raw[i]["width_idx"]))
    r = [raw[i] for i in key]
    lab = list(range(n))

    def friends(a, b):
        ta, ea = int(a["sample"]), int(a["sample"]) + int(widths[a["width_idx"]])
        tb, eb = int(b["sample"]), int(b["sample"]) + int(widths[b["width_idx"]])
        return (abs(int(a["dm_idx"]) - int(b["dm_idx"])) <= dm_tol
                and abs(int(a["width_idx"]) - int(b["width_idx"])) <= w_tol
                and max(ta, tb) - min(ea, eb) <= t_gap)

    changed = True
    while changed:                                   # label propagation to the minimum
        changed = False
        for i in range(n):
            for j in range(n):
                if i != j and friends(r[i], r[j]) and lab[j] < lab[i]:
                    lab[i] = lab[j]
                    changed = True
    out = []
    for root in sorted(set(lab)):
        mem = [i for i in range(n) if lab[i] == root]
        best = mem[0]
        for i in mem:
            if r[i]["snr"] > r[best]["snr"]:
                best = i
        out.append((int(r[best]["dm_idx"]), int(r[best]["width_idx"]), int(r[best]["sample"]),
                    float(r[best]["snr"]), len(mem), min(int(r[i]["dm_idx"]) for i in mem),
                    max(int(r[i]["dm_idx"]) for i in mem), min(int(r[i]["sample"]) for i in mem),
                    max(int(r[i]["sample"]) + int(widths[r[i]["width_idx"]]) for i in mem)))
    return out


def _random_raw(rng, n, ndm=12, nw=4, tmax=400):
    raw = np.zeros(n, oracle.RAW_DTYPE)
    keys = set()
    i = 0
    while i < n:
        k = (int(rng.integers(0, ndm)), int(rng.integers(0, tmax)), int(rng.integers(0, nw)))
        if k in keys:
            continue
        keys.add(k)
        raw[i] = (k[0], k[2], k[1], 0, float(rng.integers(6, 12)))   # few snr values: ties
        i += 1
    return raw


@pytest.mark.parametrize("seed", range(8))
def test_merge_bruteforce(seed):
    rng = np.random.default_rng(200 + seed)
    widths = np.array([1, 2, 4, 8], np.int32)
    raw = _random_raw(rng, int(rng.integers(1, 120)))
    dm_tol, t_gap, w_tol = [(1, 0, 4), (2, 3, 1), (0, 0, 0), (1, -1, 4)][seed % 4]
    got = oracle.merge(raw, widths, dm_tol, t_gap, w_tol)
    want = _merge_brute(raw, widths, dm_tol, t_gap, w_tol)
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert (int(g["dm_idx"]), int(g["width_idx"]), int(g["sample"]), float(g["snr"]),
                int(g["members"]), int(g["dm_lo"]), int(g["dm_hi"]), int(g["t_lo"]),
                int(g["t_hi"])) == w


def test_merge_permutation_invariant_and_touching_windows():
    rng = np.random.default_rng(7)
    widths = np.array([1, 2, 4, 8], np.int32)
    raw = _random_raw(rng, 300, ndm=30, tmax=2000)
    a = oracle.merge(raw, widths)
    b = oracle.merge(raw[rng.permutation(raw.size)], widths)
    assert (a == b).all()
    two = np.zeros(2, oracle.RAW_DTYPE)
    two[0] = (0, 2, 10, 0, 7.0)          # window [10, 14)
    two[1] = (0, 0, 14, 0, 8.0)          # window [14, 15): touches -> gap 0
    assert len(oracle.merge(two, widths, 1, 0)) == 1
    two[1]["sample"] = 15                # gap 1
    assert len(oracle.merge(two, widths, 1, 0)) == 2
    assert len(oracle.merge(two, widths, 1, 1)) == 1


def test_raw_snr_hand_values_and_search_consistency(tiny_workload):
    """S/N of raw candidates from their sums: hand-worked values (sigma 2,
    W 4: S 120 -> 30; sigma 0.5, W 1: S -3 -> -6; sigma 3, W 16: S 84 -> 7),
    and on a whole search every raw candidate's S/N is reproduced from its S,
    its trial's sigma and its width."""
    widths = np.array([1, 4, 16], np.int32)
    raw = np.zeros(3, oracle.RAW_DTYPE)
    raw[0] = (0, 1, 5, 120, 0.0)
    raw[1] = (1, 0, 9, -3, 0.0)
    raw[2] = (2, 2, 0, 84, 0.0)
    got = oracle.raw_with_snr(raw, np.array([2.0, 0.5, 3.0]), widths)
    assert list(got["snr"]) == [30.0, -6.0, 7.0]
    w, s = tiny_workload
    o = w.obs
    r = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    assert r.raw.size > 0
    again = oracle.raw_with_snr(r.raw, r.sigma, w.widths)
    assert np.array_equal(again["snr"], r.raw["snr"])


# ------------------------------------------------------- whole-path pins

from paper_2512_00398_gb300.workloads import recovered  # noqa: E402  (the recovery criterion)


def test_injection_recovery_tiny(tiny_workload):
    w, s = tiny_workload
    o = w.obs
    r = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    for p in s.pulses:
        assert recovered(p, r.clusters, w), p


def test_unit_rms_on_pure_noise():
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    w.pulses = []
    s = w.generate()
    o = w.obs
    tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list[::20])
    D = oracle.dedisperse(s.data, tab)
    win = oracle.baseline_window(2.0, o.tsamp)
    for row in D:
        y = oracle.subtract_baseline(row, 0, win)
        sig = oracle.sigma_from_mad(oracle.mad(y))
        assert abs(np.std(y / sig) - 1.0) < 0.02
