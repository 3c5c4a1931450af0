"""Pins of the oracle's sub-band (two-stage) dedispersion variant.

The oracle writes the variant as direct dedispersion with an effective delay
table (hp_oracle.c, hpo_subband_delays).  These tests pin that table and the
search built on it against things fixed independently of it: the two stages
carried out literally (per sub-band partial sums at the nominal trial, then
shifted sums of the partial sums), the reductions S = 1, G = 1 and S >= nchans,
and the closed-form bound on how far an effective delay can move from the
direct one.
"""
import numpy as np
import pytest

import oracle
from paper_2512_00398_gb300 import synth

KDM = 4148.808


def _nominal(d, G, ndm):
    g = d // G
    size = min(G, ndm - g * G)
    return g * G + (size - 1) // 2


def _two_stage(x, delay, S, G):
    """Stage 1 and stage 2 with explicit loops over sub-bands and groups."""
    nsamps, nch = x.shape
    ndm = delay.shape[0]
    nsub = -(-nch // S)
    xi = x.astype(np.int64)
    # the reach of every term, to know which outputs are complete
    reach = 0
    for d in range(ndm):
        n = _nominal(d, G, ndm)
        for s in range(nsub):
            top = s * S
            for c in range(top, min(top + S, nch)):
                reach = max(reach, delay[d, top] + delay[n, c] - delay[n, top])
    nout = nsamps - reach
    out = np.zeros((ndm, nout), np.int64)
    for g in range(-(-ndm // G)):
        n = _nominal(g * G, G, ndm)
        for s in range(nsub):
            top = s * S
            chans = range(top, min(top + S, nch))
            # stage 1: B[u] for every u the group's trials read
            ulen = nout + max(delay[d, top] for d in range(g * G, min(g * G + G, ndm)))
            B = np.zeros(ulen, np.int64)
            for c in chans:
                r = delay[n, c] - delay[n, top]
                B += xi[r:r + ulen, c]
            # stage 2: each trial of the group adds its shifted partial sum
            for d in range(g * G, min(g * G + G, ndm)):
                o = delay[d, top]
                out[d] += B[o:o + nout]
    return out, reach


@pytest.mark.parametrize("nch,ndm,S,G", [(16, 9, 4, 3), (20, 7, 6, 2), (12, 10, 5, 4),
                                         (9, 5, 9, 5), (13, 11, 3, 7)])
def test_two_stage_bruteforce(nch, ndm, S, G):
    rng = np.random.default_rng(nch * 100 + ndm)
    tsamp = 1e-3
    dms = np.sort(rng.uniform(0, 300, ndm)).astype(np.float32)
    delay = oracle.delays(nch, 1400.0, -200.0 / nch, tsamp, dms)
    nsamps = int(delay.max()) + 300
    x = rng.integers(0, 256, size=(nsamps, nch), dtype=np.uint8)
    want, reach = _two_stage(x, delay, S, G)
    e = oracle.subband_delays(delay, S, G)
    assert int(e.max()) == reach
    got = oracle.dedisperse(x, e, nout=nsamps - reach)
    assert np.array_equal(got.astype(np.int64), want)


def test_reductions():
    dms = np.linspace(0, 800, 23).astype(np.float32)
    delay = oracle.delays(64, 1500.0, -500.0 / 64, 64e-6, dms)
    for G in (1, 2, 5, 23, 40):
        assert np.array_equal(oracle.subband_delays(delay, 1, G), delay)
    for S in (1, 3, 8, 64, 100):
        assert np.array_equal(oracle.subband_delays(delay, S, 1), delay)
    # one sub-band: every trial takes its group's nominal row (channel 0 has no delay)
    for G in (2, 4, 7):
        e = oracle.subband_delays(delay, 64, G)
        for d in range(len(dms)):
            assert np.array_equal(e[d], delay[_nominal(d, G, len(dms))])


def test_error_bound_closed_form():
    """e - delay = (a_c - a_top)(DM_n - DM_d) + (four roundings), so
    |e - delay| <= |a_c - a_top| |DM_n - DM_d| + 2 with a_c the delay per unit
    DM of channel c in samples."""
    nch, tsamp, f_top, bw = 256, 49.152e-6, 1500.0, -500.0 / 256
    dms = np.linspace(0, 2000, 301).astype(np.float32)
    delay = oracle.delays(nch, f_top, bw, tsamp, dms)
    f = f_top + np.arange(nch) * bw
    a = KDM * (f ** -2.0 - f_top ** -2.0) / tsamp
    for S, G in ((16, 4), (32, 8), (7, 3)):
        e = oracle.subband_delays(delay, S, G)
        top = (np.arange(nch) // S) * S
        n = np.array([_nominal(d, G, len(dms)) for d in range(len(dms))])
        bound = np.abs(a[None, :] - a[top][None, :]) * np.abs(
            dms[n].astype(np.float64) - dms.astype(np.float64))[:, None] + 2.0 + 1e-9
        assert (np.abs(e.astype(np.int64) - delay) <= bound).all()
        # and the shift is not trivially zero: the bound is approached
        assert np.abs(e - delay).max() >= 0.5 * (bound - 2.0).max() - 1


def test_search_reduces_to_direct_and_keeps_pulses(tiny_workload):
    w, s = tiny_workload
    o = w.obs
    direct = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    same = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         subband=(1, 4))
    assert np.array_equal(direct.clusters, same.clusters)
    # sub-bands of 16 channels, groups of 4 trials: every injected pulse keeps
    # at least 90% of its direct S/N at the best cluster near it
    sub = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                        subband=(16, 4))
    for p in s.pulses:
        t_true = p.t0 / o.tsamp
        def best(cl):
            near = cl[np.abs(cl["sample"] - t_true) < 200]
            return near["snr"].max() if len(near) else 0.0
        assert best(sub.clusters) >= 0.9 * best(direct.clusters), p


def test_argument_errors():
    d = np.zeros((3, 4), np.int32)
    with pytest.raises(ValueError):
        oracle.subband_delays(d, 0, 2)
    with pytest.raises(ValueError):
        oracle.subband_delays(d, 2, 0)


def test_stream_reduces_to_direct_at_one_channel_per_subband():
    """The streamed search takes the variant's table and geometry: with one
    channel per sub-band it is the direct streamed search, gulp by gulp."""
    from paper_2512_00398_gb300 import workloads
    ws = workloads.stream_tiny(nbeams=1, ngulps=5, gulp=4096)
    w = ws[0]
    x = w.generate().data
    o = w.obs
    a = oracle.stream_search(x, 4096, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    b = oracle.stream_search(x, 4096, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                             subband=(1, 3))
    assert [r["B0"] for r in a] == [r["B0"] for r in b]
    for ra, rb in zip(a, b):
        assert np.array_equal(ra["clusters"], rb["clusters"])
    assert sum(len(r["clusters"]) for r in a) > 0
