"""Sub-band (two-stage) dedispersion on the GPU against the oracle.

The variant equals direct dedispersion with the effective delay table (the
oracle's hpo_subband_delays), so the GPU's two stages must reproduce the
oracle's sums exactly: on the tiny band for every tile shape that runs the
segmented stage 1, on ragged sub-bands and groups, and sampled at the full
FAST size (several chunks of groups, partial sums held two chunks at a time).
The search on the variant's series must give the oracle's clusters.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4
SEGMENTED = [7, 11, 12, 14]


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
    o = w.obs
    tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list)
    return w, s, torch.from_numpy(s.data).cuda(), tab


@pytest.mark.parametrize("cfg", SEGMENTED)
@pytest.mark.parametrize("S,G", [(16, 4), (48, 7), (128, 3), (1, 5), (32, 1)])
def test_subband_dedisp_bit_exact(hp, torch, tiny, cfg, S, G):
    w, s, fb, tab = tiny
    p = _plan(hp, w, dedisp_config=cfg, subband_chans=S, subband_group=G)
    eff = oracle.subband_delays(tab, S, G)
    assert np.array_equal(p.delays(), eff)
    got = hp.dedisperse(p, fb)
    want = oracle.dedisperse(s.data, eff)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_subband_ragged_and_saturated(hp, torch):
    """Odd channel count, a sub-band size that does not divide it, duplicate
    and widely spaced trials, a group size that does not divide the trial
    count, saturated bytes, a ragged time tail."""
    from paper_2512_00398_gb300 import synth
    rng = np.random.default_rng(12)
    nch, nsamps = 100, 20011
    dms = np.sort(np.concatenate([[0, 0, 3.5, 3.5], rng.uniform(0, 900, 37), [1500.0]]))
    dms = dms.astype(np.float32)
    x = rng.integers(0, 256, size=(nsamps, nch), dtype=np.uint8)
    x[rng.integers(0, nsamps, 50)] = 255
    tab = oracle.delays(nch, 1450.0, -3.0, 1e-4, dms)
    for S, G in ((7, 3), (33, 5), (100, 42)):
        p = hp.Plan(nch, 1450.0, -3.0, 1e-4, dms, synth.widths_pow2(16), 6.0,
                    subband_chans=S, subband_group=G)
        eff = oracle.subband_delays(tab, S, G)
        got = hp.dedisperse(p, torch.from_numpy(x).cuda())
        assert np.array_equal(got, oracle.dedisperse(x, eff)), (S, G)


def test_subband_search_matches_oracle(hp, torch, tiny):
    w, s, fb, tab = tiny
    o = w.obs
    for S, G in ((16, 4), (32, 8)):
        want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                             w.threshold, subband=(S, G))
        got = hp.search(_plan(hp, w, subband_chans=S, subband_group=G), fb)
        assert len(want.clusters) > 0
        key = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
        assert [key(c) for c in got] == [key(c) for c in want.clusters]
        for a, b in zip(got, want.clusters):
            assert abs(float(a["snr"]) - float(b["snr"])) <= SNR_TOL
            for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
                assert int(a[f]) == int(b[f])


def test_subband_autotune_and_direct_switch(hp, torch, tiny):
    w, s, fb, tab = tiny
    p = _plan(hp, w, subband_chans=16, subband_group=4)
    before = hp.dedisperse(p, fb)
    cfg, ms = hp.hp_plan_autotune(p, fb)
    assert cfg in SEGMENTED and ms > 0
    assert np.array_equal(hp.dedisperse(p, fb), before)
    p.set_param("subband_chans", 0)                      # back to the direct sums
    assert np.array_equal(hp.dedisperse(p, fb), oracle.dedisperse(s.data, tab))


def test_subband_in_a_batch_matches_per_file(hp, torch, tiny):
    """A batch mixing a sub-band file and a direct file: the direct file in the
    batched launch, the sub-band file through its own two stages; each equal to
    its plain search (eager, captured, replayed); batch autotuning refuses it."""
    w, s, fb, tab = tiny
    o = w.obs
    p_sb, p_d = _plan(hp, w, subband_chans=16, subband_group=4), _plan(hp, w)
    want = [hp.search(_plan(hp, w, subband_chans=16, subband_group=4), fb), hp.search(_plan(hp, w), fb)]
    b = hp.Batch([p_sb, p_d])
    first = b.search([fb, fb])
    for got, sb in zip(first, [(16, 4), None]):
        ref = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                            w.threshold, subband=sb).clusters
        key = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
        assert [key(c) for c in got] == [key(c) for c in ref] and len(ref) > 0
        for a, c in zip(got, ref):
            assert abs(float(a["snr"]) - float(c["snr"])) <= SNR_TOL
            for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
                assert int(a[f]) == int(c[f])
    for _ in range(3):
        got = b.search([fb, fb])
        for g, w_ in zip(got, want):
            assert np.array_equal(g, w_)
    with pytest.raises(hp.HPError):
        b.autotune([fb, fb])
    b.close()
    # a tile shape without the segmented stage 1
    with pytest.raises(hp.HPError):
        hp.dedisperse(_plan(hp, w, dedisp_config=0, subband_chans=16), fb)


def test_subband_stream_matches_oracle(hp, torch):
    """Two beams streamed with the sub-band variant: every gulp's clusters equal
    the oracle's streamed search on the effective table."""
    from paper_2512_00398_gb300 import workloads
    G = 4096
    ws = workloads.stream_tiny(nbeams=2, ngulps=6, gulp=G)
    data = [w_.generate().data for w_ in ws]
    w = ws[0]
    o = w.obs
    st = hp.Stream(_plan(hp, w, subband_chans=16, subband_group=4), nbeams=2, gulp=G)
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
        got[(info["beam"], info["gulp_index"])] = (info, c)
    st.close()
    n = 0
    for b in range(2):
        want = oracle.stream_search(data[b], G, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                                    w.threshold, subband=(16, 4))
        for r in want:
            info, c = got[(b, r["g"])]
            assert info["window_start"] == r["B0"] and info["window_len"] == r["nwin"]
            wc = r["clusters"]
            assert len(c) == len(wc)
            for f in ("dm_idx", "width_idx", "sample", "members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
                assert np.array_equal(c[f], wc[f]), f
            if len(c):
                assert np.abs(c["snr"].astype(np.float64) - wc["snr"]).max() <= SNR_TOL
            n += len(wc)
    assert n > 0


def test_subband_fast_full_size_sampled(hp, torch):
    """4096 ch x 2^20 samples x ~1500 trials with 64-channel sub-bands and
    groups of 8 trials, in the benchmark's configuration: sampled sums equal
    the oracle's on the effective table (every chunk of groups)."""
    from paper_2512_00398_gb300 import workloads
    w = workloads.fast()
    s = w.generate(threads=16)
    fb = torch.from_numpy(s.data).cuda()
    p = _plan(hp, w, subband_chans=64, subband_group=8)
    eff = p.delays()
    o = w.obs
    assert np.array_equal(eff, oracle.subband_delays(
        oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list), 64, 8))
    nout = p.nout(fb.shape[0])
    D = hp.hp_dedisperse(p, fb)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    rng = np.random.default_rng(31)
    ds = np.concatenate([rng.integers(0, w.ndm, 250), [0, w.ndm - 1, 191, 192, 383, 384]])
    ts = np.concatenate([rng.integers(0, nout, 250), [0, nout - 1, nout - 2, 511, 512, 4095]])
    Dh = D[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
    for d, t, v in zip(ds, ts, Dh):
        assert oracle.dedisperse_point(s.data, eff[d], int(t)) == int(v), (d, t)
    for d in (0, 383, w.ndm - 1):
        Do = oracle.dedisperse(s.data, eff, rows=(d, d + 1))
        assert np.array_equal(Do[0], D[d, :nout].cpu().numpy()), d


def test_subband_search_with_rfi_matches_oracle(hp, torch, tiny):
    """RFI mitigation before the two stages: the oracle cleans the input, then
    searches it with the effective table."""
    w, s, fb, tab = tiny
    o = w.obs
    x = s.data.astype(np.int32)
    x[:, [5, 77]] += 45
    x[::2999, :] += 40
    x = np.clip(x, 0, 255).astype(np.uint8)
    clean = oracle.rfi_clean(x, o.tsamp).cleaned
    want = oracle.search(clean, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         subband=(16, 4))
    p = _plan(hp, w, subband_chans=16, subband_group=4, rfi=1)
    got = hp.search(p, torch.from_numpy(x).cuda())
    key = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
    assert len(want.clusters) > 0
    assert [key(c) for c in got] == [key(c) for c in want.clusters]
    for a, b in zip(got, want.clusters):
        assert abs(float(a["snr"]) - float(b["snr"])) <= SNR_TOL


def test_subband_shortest_input(hp, torch, tiny):
    """The shortest accepted input (nsamps = max effective delay + widest boxcar + 1)
    and one sample less (refused)."""
    w, s, fb, tab = tiny
    o = w.obs
    p = _plan(hp, w, subband_chans=16, subband_group=4)
    eff = p.delays()
    n = int(eff.max()) + int(w.widths.max()) + 1
    x = s.data[:n]
    got = hp.dedisperse(p, torch.from_numpy(np.ascontiguousarray(x)).cuda())
    assert got.shape[1] == n - int(eff.max())
    assert np.array_equal(got, oracle.dedisperse(x, eff))
    with pytest.raises(hp.HPError) as e:
        hp.search(p, torch.from_numpy(np.ascontiguousarray(s.data[:n - 1])).cuda())
    assert e.value.code == hp.HP_ERR_NSAMPS_TOO_SHORT
