"""Per-width normalisation (HP_PARAM_WIDTH_SIGMA) on the GPU against the oracle.

The per-width MADs must equal the oracle's exactly (the radix selection is
exact), the sigmas bit for bit (the same FP64 product), the raw candidates'
tuples and sums exactly and the S/N within 1e-4; the whole search must give
the oracle's clusters.  Large magnitudes and a median beyond the first pass (the
restart from the top digit) are checked too.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def hp():
    import paper_2512_00398_gb300 as hp
    return hp


def _plan(hp, w, **params):
    o = w.obs
    return hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                   **params)


@pytest.fixture(scope="module")
def tiny(torch):
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    s = w.generate()
    return w, s, torch.from_numpy(s.data).cuda()


def _key(rows):
    return sorted((int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"]), int(r["S"])) for r in rows)


def test_search_matches_oracle(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         width_sigma=True)
    got = hp.search(_plan(hp, w, width_sigma=1), fb)
    assert len(want.clusters) > 0
    k = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
    assert [k(c) for c in got] == [k(c) for c in want.clusters]
    for a, b in zip(got, want.clusters):
        assert abs(float(a["snr"]) - float(b["snr"])) <= SNR_TOL
        for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
            assert int(a[f]) == int(b[f])


def test_detect_sigmas_and_raw_exact(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    D = oracle.dedisperse(s.data, oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list))
    p = _plan(hp, w, width_sigma=1)
    raw_g, _, _ = hp.detect(p, torch.from_numpy(D).cuda(), D.shape[1])
    sg, md = (t.cpu().numpy() for t in hp.hp_width_sigmas(p))
    raw_o, _, _ = oracle.search_trials(D, 0, o.tsamp, w.widths, w.threshold, width_sigma=True)
    assert _key(raw_g) == _key(raw_o)
    win = oracle.baseline_window(2.0, o.tsamp)
    for d in (0, 1, 37, w.ndm - 1):
        y = oracle.subtract_baseline(D[d], 0, win)
        m_o, s_o = oracle.width_sigma(y, w.widths)
        assert np.array_equal(md[d], m_o), d
        assert np.array_equal(sg[d], s_o), d


def test_large_magnitudes(hp, torch):
    """Series of +-2^20: the medians of |S_k| for the wide widths lie above
    2^24, where the selection counts the high digits first."""
    from paper_2512_00398_gb300 import synth
    rng = np.random.default_rng(5)
    nout, ndm = 40000, 3
    widths = np.array([1, 16, 256, 1024, 4096], np.int32)
    D = rng.integers(-(1 << 20), 1 << 20, size=(ndm, nout)).astype(np.int32)
    D[1] += np.cumsum(rng.integers(-4000, 4001, nout)).astype(np.int32)   # red noise
    p = hp.Plan(64, 1500.0, -1.0, 1e-3, np.zeros(ndm, np.float32), widths, 6.0, width_sigma=1)
    raw_g, _, _ = hp.detect(p, torch.from_numpy(D).cuda(), nout)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    sg, md = (t.cpu().numpy() for t in hp.hp_width_sigmas(p))
    raw_o, _, _ = oracle.search_trials(D, 0, 1e-3, widths, 6.0, width_sigma=True)
    win = oracle.baseline_window(2.0, 1e-3)
    assert (md[:, -1] >= (1 << 24)).all()
    for d in range(ndm):
        y = oracle.subtract_baseline(D[d], 0, win)
        m_o, s_o = oracle.width_sigma(y, widths)
        assert np.array_equal(md[d], m_o), d
        assert np.array_equal(sg[d], s_o), d
    assert _key(raw_g) == _key(raw_o)


def test_median_beyond_the_first_pass(hp, torch):
    """A series whose MAD is 0 (three samples in five are 0) while most wide
    boxcars sum to more than 2^24: the first pass, sized from the MAD, cannot
    resolve the median and the selection restarts from the top digit."""
    nout = 30000
    t = np.arange(nout)
    D = np.where(t % 5 < 2, 1 << 20, 0).astype(np.int32)[None, :].repeat(2, axis=0)
    D[1, ::7] += 3
    widths = np.array([1, 8, 64, 1024], np.int32)
    p = hp.Plan(64, 1500.0, -1.0, 1e-3, np.zeros(2, np.float32), widths, 6.0, width_sigma=1)
    raw_g, _, mad_g = hp.detect(p, torch.from_numpy(D).cuda(), nout)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    sg, md = (t_.cpu().numpy() for t_ in hp.hp_width_sigmas(p))
    win = oracle.baseline_window(2.0, 1e-3)
    raw_o, _, _ = oracle.search_trials(D, 0, 1e-3, widths, 6.0, width_sigma=True)
    for d in range(2):
        y = oracle.subtract_baseline(D[d], 0, win)
        m_o, s_o = oracle.width_sigma(y, widths)
        assert np.array_equal(md[d], m_o), (d, md[d], m_o)
        assert np.array_equal(sg[d], s_o), d
    assert mad_g[0] == 0 and md[0, 2] > (1 << 24)
    assert _key(raw_g) == _key(raw_o)


def test_batch_matches_per_file(hp, torch, tiny):
    """A batched search with per-width sigmas equals the oracle's and the
    plain per-file search (eager, captured, replayed)."""
    w, s, fb = tiny
    o = w.obs
    p1, p2 = _plan(hp, w, width_sigma=1), _plan(hp, w, width_sigma=1)
    want = hp.search(p1, fb)
    ref = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                        width_sigma=True).clusters
    b = hp.Batch([p2])
    for i in range(3):                       # eager, captured, replayed
        got = b.search([fb])
        if i == 0:
            k = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
            assert [k(c) for c in got[0]] == [k(c) for c in ref] and len(ref) > 0
            for a, c in zip(got[0], ref):
                assert abs(float(a["snr"]) - float(c["snr"])) <= SNR_TOL
                for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
                    assert int(a[f]) == int(c[f])
        assert np.array_equal(got[0], want)
    b.close()


def test_mode_switch(hp, torch, tiny):
    w, s, fb = tiny
    p = _plan(hp, w)
    with pytest.raises(hp.HPError):
        hp.hp_width_sigmas(p)                # mode off
    plain = hp.search(p, fb)
    p.set_param("width_sigma", 1)
    with pytest.raises(hp.HPError):
        hp.hp_width_sigmas(p)                # nothing searched in the mode yet
    hp.search(p, fb)
    sg, md = hp.hp_width_sigmas(p)
    assert sg.shape == (w.ndm, len(w.widths))
    p.set_param("width_sigma", 0)
    assert np.array_equal(hp.search(p, fb), plain)


def test_stream_matches_oracle(hp, torch):
    """Two beams pushed gulp by gulp in the per-width mode: every gulp's
    clusters equal the oracle's streamed search with the sigmas of each
    searched buffer."""
    from paper_2512_00398_gb300 import workloads
    G = 4096
    ws = workloads.stream_tiny(nbeams=2, ngulps=6, gulp=G)
    data = [w_.generate().data for w_ in ws]
    w = ws[0]
    o = w.obs
    st = hp.Stream(_plan(hp, w, width_sigma=1), nbeams=2, gulp=G)
    for g in range(6):
        for b in range(2):
            st.push(b, data[b][g * G:(g + 1) * G])
    for b in range(2):
        st.end_beam(b)
    got = {}
    while len(got) < 12:
        r = st.poll(timeout_ms=120000)
        assert r is not None, "stream stalled"
        info, c = r
        assert info["status"] == hp.HP_OK
        got[(info["beam"], info["gulp_index"])] = c
    st.close()
    n = 0
    for b in range(2):
        want = oracle.stream_search(data[b], G, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                                    w.threshold, width_sigma=True)
        for r in want:
            c, wc = got[(b, r["g"])], r["clusters"]
            assert len(c) == len(wc)
            for f in ("dm_idx", "width_idx", "sample", "members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
                assert np.array_equal(c[f], wc[f]), f
            if len(c):
                assert np.abs(c["snr"].astype(np.float64) - wc["snr"]).max() <= SNR_TOL
            n += len(wc)
    assert n > 0


def test_fast_full_size_sampled(hp, torch):
    """The FAST shape: per-width MADs of sampled trials equal the oracle's."""
    from paper_2512_00398_gb300 import workloads
    w = workloads.fast()
    s = w.generate(threads=16)
    fb = torch.from_numpy(s.data).cuda()
    p = _plan(hp, w, width_sigma=1)
    p.bind_workspace(fb.shape[0])
    got = hp.search(p, fb)
    sg, md = (t.cpu().numpy() for t in hp.hp_width_sigmas(p))
    o = w.obs
    tab = p.delays()
    win = oracle.baseline_window(2.0, o.tsamp)
    for d in (0, 777, w.ndm - 1):
        Dd = oracle.dedisperse(s.data, tab, rows=(d, d + 1))[0]
        y = oracle.subtract_baseline(Dd, 0, win)
        m_o, s_o = oracle.width_sigma(y, w.widths)
        assert np.array_equal(md[d], m_o), d
        assert np.array_equal(sg[d], s_o), d
    assert len(got) > 0
