"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Dedispersed sums, MADs, sigmas, integer thresholds and candidate tuples must
match exactly; S/N values within 1e-4 (the FP32 S/N of hp_cand against the
oracle's FP64 value; |delta| <= 1e-4 holds for S/N up to ~500 because FP32
rounding is ~6e-8 relative).
"""
import math

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


def _key(rows):
    return sorted((int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"])) for r in rows)


def _compare_clusters(got, want, thr):
    """Exact tuples and member statistics, snr within SNR_TOL.  Clusters whose
    oracle representative lies within SNR_TOL of the threshold may differ."""
    g = {(int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"])): c for c in got}
    w = {(int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"])): c for c in want}
    near = {k for k, c in w.items() if abs(float(c["snr"]) - thr) <= SNR_TOL}
    assert set(g) - near == set(w) - near
    for k in set(w) - near:
        a, b = g[k], w[k]
        assert abs(float(a["snr"]) - float(b["snr"])) <= SNR_TOL, k
        for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
            assert int(a[f]) == int(b[f]), (k, f)


@pytest.fixture(scope="module")
def tiny(torch):
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    s = w.generate()
    return w, s, torch.from_numpy(s.data).cuda()


@pytest.mark.parametrize("cfg", list(range(20)))
def test_dedisp_bit_exact_tiny(hp, torch, tiny, cfg):
    w, s, fb = tiny
    p = _plan(hp, w, dedisp_config=cfg)
    got = hp.dedisperse(p, fb)
    o = w.obs
    want = oracle.dedisperse(s.data, oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list))
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("cfg", list(range(20)))
def test_dedisp_bit_exact_ragged(hp, torch, cfg):
    """Odd channel count (scalar transpose path), duplicate and widely spaced
    trials (adaptive DM tiles), a ragged time tail, saturated bytes."""
    from paper_2512_00398_gb300 import synth
    rng = np.random.default_rng(11)
    nch, nsamps = 100, 20011
    dms = np.sort(np.concatenate([[0, 0, 3.5, 3.5], rng.uniform(0, 900, 37), [1500.0]]))
    dms = dms.astype(np.float32)
    x = rng.integers(0, 256, size=(nsamps, nch), dtype=np.uint8)
    x[rng.integers(0, nsamps, 50)] = 255
    tab = oracle.delays(nch, 1450.0, -3.0, 1e-4, dms)
    p = hp.Plan(nch, 1450.0, -3.0, 1e-4, dms, synth.widths_pow2(16), 6.0, dedisp_config=cfg)
    assert np.array_equal(p.delays(), tab)
    got = hp.dedisperse(p, torch.from_numpy(x).cuda())
    assert np.array_equal(got, oracle.dedisperse(x, tab))


def test_detect_exact_on_oracle_series(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    D = oracle.dedisperse(s.data, oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list))
    raw_o, sig_o, mad_o = oracle.search_trials(D, 0, o.tsamp, w.widths, w.threshold)
    p = _plan(hp, w)
    Dg = torch.from_numpy(D).cuda()
    raw_g, sig_g, mad_g = hp.detect(p, Dg, D.shape[1])
    assert np.array_equal(mad_g, mad_o)
    assert np.array_equal(sig_g, sig_o)                     # same FP64 operations
    assert _key(raw_g) == _key(raw_o)
    go = {(int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"])): int(r["S"]) for r in raw_g}
    for r in raw_o:
        assert go[(int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"]))] == int(r["S"])


@pytest.mark.parametrize("mode", [0, 1])
def test_detect_narrow_and_wide_trials(hp, torch, mode):
    """Trials whose boxcar sums all fit int32 (the 32-bit detection) next to
    trials with spikes of ~2^24 (|y| bound x widest boxcar >= 2^31: the int64
    detection), in one call: MADs, sigmas and raw candidates exact against the
    oracle.  Runs near tile edges, a pulse at the series end."""
    rng = np.random.default_rng(41 + mode)
    ndm, nout = 6, 50000
    widths = np.array([1, 2, 3, 8, 12, 64, 256], np.int32)
    D = rng.normal(0, 30, size=(ndm, nout)).round().astype(np.int64)
    for d in range(ndm):
        for t in rng.integers(0, nout - 300, 6):
            D[d, t:t + int(rng.integers(1, 200))] += int(rng.integers(20, 80))
        D[d, 4096 * 3 - 2:4096 * 3 + 3] += 400          # across a tile edge
        D[d, -5:] += 300                                # up to the last start
    D[4, rng.integers(0, nout, 40)] += 1 << 24           # wide trials
    D[5, rng.integers(0, nout, 40)] -= 1 << 24
    D = D.astype(np.int32)
    raw_o, sig_o, mad_o = oracle.search_trials(D, 0, 1e-3, widths, 5.0, baseline_mode=mode,
                                               baseline_s=0.5)
    p = hp.Plan(16, 1500.0, -1.0, 1e-3, np.zeros(ndm, np.float32), widths, 5.0,
                baseline_mode=mode, baseline_s=0.5)
    raw_g, sig_g, mad_g = hp.detect(p, torch.from_numpy(D).cuda(), nout)
    assert np.array_equal(mad_g, mad_o) and np.array_equal(sig_g, sig_o)
    assert len(raw_o) > 0 and {4, 5} <= set(int(r["dm_idx"]) for r in raw_o)
    go = sorted((int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"]), int(r["S"])) for r in raw_g)
    wo = sorted((int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"]), int(r["S"])) for r in raw_o)
    assert go == wo


def test_search_matches_oracle_tiny(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    p = _plan(hp, w)
    got = hp.search(p, fb)
    assert len(want.clusters) > 0
    _compare_clusters(got, want.clusters, w.threshold)
    assert [tuple(int(c[f]) for f in ("dm_idx", "sample", "width_idx")) for c in got] == \
           [tuple(int(c[f]) for f in ("dm_idx", "sample", "width_idx")) for c in want.clusters]


def test_search_mean_baseline_and_tolerances(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         baseline_mode=1, baseline_s=0.5, dm_tol=2, t_gap=3, w_tol=2)
    p = _plan(hp, w, baseline_mode=1, baseline_s=0.5, dm_tol=2, t_gap=3, w_tol=2)
    got = hp.search(p, fb)
    _compare_clusters(got, want.clusters, w.threshold)


@pytest.mark.parametrize("baseline_s", [1e-5, 0.0005, 30.0])
def test_search_baseline_extremes(hp, torch, tiny, baseline_s):
    """L = 0 (no smoothing: every y is 0, sigma 0, no candidates), a short
    window (many remedian blocks) and a window longer than the series."""
    w, s, fb = tiny
    o = w.obs
    want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         baseline_s=baseline_s)
    got = hp.search(_plan(hp, w, baseline_s=baseline_s), fb)
    _compare_clusters(got, want.clusters, w.threshold)


def test_no_candidates_and_short_input(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    p = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, 1e6)
    assert hp.search(p, fb).size == 0
    short = fb[: p.max_delay + int(w.widths[-1])].contiguous()
    with pytest.raises(hp.HPError) as e:
        hp.search(p, short)
    assert e.value.code == hp.HP_ERR_NSAMPS_TOO_SHORT


def test_raw_overflow_is_reported(hp, torch, tiny):
    w, s, fb = tiny
    p = _plan(hp, w, raw_capacity=1024)
    with pytest.raises(hp.HPError) as e:
        hp.search(p, fb)
    assert e.value.code == hp.HP_ERR_CAND_OVERFLOW
    # the latch is cleared once reported; a roomy plan then succeeds
    p.set_param("raw_capacity", 1 << 20)
    assert hp.search(p, fb).size > 0


def test_output_capacity_truncates(hp, torch, tiny):
    w, s, fb = tiny
    p = _plan(hp, w)
    data, count = hp.hp_search(p, fb, capacity=5)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    n = int(count.item())
    assert n > 5
    full = hp.search(p, fb)
    assert len(full) == n
    part = hp.cands_to_numpy(data, count)
    assert np.array_equal(part, full[:5])


def test_injections_recovered_tiny(hp, torch, tiny):
    from tests.test_oracle_pins import recovered
    w, s, fb = tiny
    got = hp.search(_plan(hp, w), fb)
    for p in s.pulses:
        assert recovered(p, got, w), p


def test_workspace_binding_allocates_once(hp, torch, tiny):
    w, s, fb = tiny
    p = _plan(hp, w)
    ws = p.bind_workspace(fb.shape[0])
    a = hp.search(p, fb)
    b = hp.search(p, fb)
    assert ws.data_ptr() == p._ws.data_ptr()
    assert np.array_equal(a, b)


# ----------------------------------------------------------- full size

@pytest.fixture(scope="module")
def fast_full(torch):
    from paper_2512_00398_gb300 import workloads
    w = workloads.fast()
    s = w.generate(threads=16)
    return w, s, torch.from_numpy(s.data).cuda()


def test_fast_full_size_sampled(hp, torch, fast_full):
    """4096 ch x 2^20 samples x ~1500 trials, in the launch configuration the
    benchmark times: sampled dedispersed sums exact; the per-trial stages exact
    on sampled trials (oracle rows computed from the input); merged clusters
    consistent with the raw candidate count."""
    w, s, fb = fast_full
    o = w.obs
    p = _plan(hp, w)
    p.bind_workspace(fb.shape[0])
    tab = p.delays()
    nout = p.nout(fb.shape[0])
    D = hp.hp_dedisperse(p, fb)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    rng = np.random.default_rng(21)
    ds = rng.integers(0, w.ndm, 200)
    ts = rng.integers(0, nout, 200)
    ts[:8] = [0, 1, nout - 1, nout - 2, nout - 3, nout - 4, 511, 512]
    Dh = D[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
    for d, t, v in zip(ds, ts, Dh):
        assert oracle.dedisperse_point(s.data, tab[d], int(t)) == int(v), (d, t)
    rows = [0, 1, int(w.ndm // 2), w.ndm - 1]
    raw_g, sig_g, mad_g = hp.detect(p, D, nout)
    for d in rows:
        Do = oracle.dedisperse(s.data, tab, rows=(d, d + 1))
        assert np.array_equal(Do[0], D[d, :nout].cpu().numpy())
        raw_o, sig_o, mad_o = oracle.search_trials(Do, d, o.tsamp, w.widths, w.threshold)
        assert mad_g[d] == mad_o[0] and sig_g[d] == sig_o[0]
        assert _key(raw_g[raw_g["dm_idx"] == d]) == _key(raw_o)
    got = hp.search(p, fb)
    assert int(got["members"].sum()) == raw_g.size
    assert (got["dm_lo"] <= got["dm_idx"]).all() and (got["dm_idx"] <= got["dm_hi"]).all()
    assert (got["t_lo"] <= got["sample"]).all() and (got["sample"] < got["t_hi"]).all()
    # the search's clusters are hp_merge's of the raw list hp_detect finds; hp_merge
    # itself is compared with the oracle at this scale in tests/test_gpu_merge.py
    raw_d, cnt_d, sig_d, _ = hp.hp_detect(p, D, nout)
    data, count = hp.hp_merge(p, raw_d, cnt_d, sig_d)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    assert np.array_equal(hp.cands_to_numpy(data, count), got)


def test_stress_full_size_sampled(hp, torch):
    """The stress shape (4096 ch x 2^21 samples, ~4000 trials on DM 0-5000,
    boxcars 1..8192) with zero-DM spikes, narrowband tones and a baseline
    drift: sampled dedispersed sums exact, and on sampled trials (including
    DM 0, where the broadband spikes add up) baseline, sigma and the raw
    candidates equal the oracle's."""
    from paper_2512_00398_gb300 import workloads
    w = workloads.stress()
    s = w.generate(threads=16)
    o = w.obs
    fb = torch.from_numpy(s.data).cuda()
    # the drift leaves long-boxcar residuals above threshold at every DM:
    # ~17 000 raw candidates per trial, ~6e7 in all
    p = _plan(hp, w, raw_capacity=1 << 26)
    tab = p.delays()
    nout = p.nout(fb.shape[0])
    D = hp.hp_dedisperse(p, fb)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    rng = np.random.default_rng(23)
    ds = rng.integers(0, w.ndm, 100)
    ts = rng.integers(0, nout, 100)
    ts[:4] = [0, nout - 1, nout - 2, 895]
    Dh = D[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
    for d, t, v in zip(ds, ts, Dh):
        assert oracle.dedisperse_point(s.data, tab[d], int(t)) == int(v), (d, t)
    raw_g, sig_g, mad_g = hp.detect(p, D, nout, capacity=1 << 26)
    assert raw_g.size > 0
    for d in [0, 1, int(w.ndm // 3), w.ndm - 1]:
        Do = oracle.dedisperse(s.data, tab, rows=(d, d + 1))
        assert np.array_equal(Do[0], D[d, :nout].cpu().numpy())
        raw_o, sig_o, mad_o = oracle.search_trials(Do, d, o.tsamp, w.widths, w.threshold)
        assert mad_g[d] == mad_o[0] and sig_g[d] == sig_o[0]
        assert _key(raw_g[raw_g["dm_idx"] == d]) == _key(raw_o)
    del D
    got = hp.search(p, fb, capacity=1 << 24)
    assert int(got["members"].sum()) == raw_g.size


def test_fast_full_size_recovery(hp, torch, fast_full):
    from tests.test_oracle_pins import recovered
    w, s, fb = fast_full
    got = hp.search(_plan(hp, w), fb)
    bright = [pl for pl in s.pulses if pl.snr >= 10.0]
    missed = [pl for pl in bright if not recovered(pl, got, w, snr_min=w.threshold)]
    assert not missed, missed


@pytest.mark.parametrize("mode", [0, 1])
def test_long_runs_and_tile_edges(hp, torch, mode):
    """Runs far longer than a detect tile plus its halo (finished by the tail
    kernel), runs straddling tile boundaries, and a run reaching the last
    start, compared exactly with the oracle in both baseline modes."""
    rng = np.random.default_rng(31)
    nch, nsamps, ts = 64, 60000, 1e-3
    dms = np.linspace(0, 30, 9).astype(np.float32)
    widths = np.array([1, 2, 8, 32, 256], np.int32)
    x = rng.normal(100, 10, size=(nsamps, nch))
    x[10000:22000] += 12          # a 12 000-sample plateau: runs of ~12 000 starts
    for edge in (4096 * 5 - 3, 4096 * 8 - 1, 4096 * 9 + 2):
        x[edge:edge + 6] += 60    # short pulses across tile boundaries
    x[-400:] += 25                # a run that ends at the series end
    x = np.clip(np.rint(x), 0, 255).astype(np.uint8)
    want = oracle.search(x, 1500.0, -4.0, ts, dms, widths, 4.0, baseline_mode=mode,
                         baseline_s=30.0)
    p = hp.Plan(nch, 1500.0, -4.0, ts, dms, widths, 4.0, baseline_mode=mode, baseline_s=30.0)
    fb = torch.from_numpy(x).cuda()
    D = hp.hp_dedisperse(p, fb)
    raw_g, sig_g, mad_g = hp.detect(p, D, p.nout(nsamps))
    assert np.array_equal(sig_g, want.sigma)
    assert _key(raw_g) == _key(want.raw)
    assert max(int(r["sample"]) for r in want.raw) > 0
    got = hp.search(p, fb)
    _compare_clusters(got, want.clusters, 4.0)


def _small_batch(nfiles=5):
    """Files of 65 536-131 072 samples, DM 0-300: 1024 channels at 49.152 and
    64 us, 2048 at 64 us, 4096 at 49.152 and 64 us (seeds 350..354)."""
    from paper_2512_00398_gb300 import workloads
    return workloads.batch(nfiles=nfiles, seed0=350, len_lo=1 << 16, len_hi=1 << 17,
                           dm_hi=300.0, trial_density=0.4, wmax=256)


def _oracle_search(w, x, **kw):
    o = w.obs
    return oracle.search(x, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold, **kw)


def test_batch_matches_per_file_search(hp, torch):
    """Uneven files (channels, lengths, sampling times) searched as one batch:
    every file's clusters equal the oracle's search of that file (exact tuples
    and member statistics, S/N within 1e-4) and, eager first call, captured
    graph, replays and after autotuning, hp_search of that file alone."""
    files = _small_batch()
    shapes = {(w.obs.nchans, round(w.obs.tsamp * 1e6, 3)) for w in files}
    assert {(1024, 64.0), (4096, 49.152), (2048, 64.0)} <= shapes
    gens = [w.generate() for w in files]
    fbs = [torch.from_numpy(g.data).cuda() for g in gens]
    plans = [_plan(hp, w) for w in files]
    want = [hp.search(p, fb) for p, fb in zip(plans, fbs)]
    assert sum(len(x) for x in want) > 0
    b = hp.Batch(plans)
    first = b.search(fbs)
    for w, g, got in zip(files, gens, first):
        _compare_clusters(got, _oracle_search(w, g.data).clusters, w.threshold)
    for _ in range(3):
        got = b.search(fbs)
        for g, w_ in zip(got, want):
            assert np.array_equal(g, w_)
    assert b.kernels_per_call() > 0
    cfg, ms = b.autotune(fbs)
    assert 0 <= cfg < hp.HP_NUM_DEDISP_CONFIGS and ms > 0
    for _ in range(2):
        got = b.search(fbs)
        for g, w_ in zip(got, want):
            assert np.array_equal(g, w_)
    # a different output set re-captures
    outs = [hp.new_cand_buf(1 << 12) for _ in fbs]
    b.search_async(fbs, outs=outs)
    assert b.sync_status() == hp.HP_OK
    for (d, c), w_ in zip(outs, want):
        assert np.array_equal(hp.cands_to_numpy(d, c), w_)
    b.close()


def test_plan_autotune_keeps_results(hp, torch, tiny):
    w, s, fb = tiny
    p = _plan(hp, w)
    before = hp.search(p, fb)
    cfg, ms = hp.hp_plan_autotune(p, fb)
    assert p.get_param("dedisp_config") == cfg and ms > 0
    assert np.array_equal(hp.search(p, fb), before)


def test_torch_caching_allocator(hp, torch, tiny):
    """Plan memory from torch's caching allocator: the same results, the
    memory shows up in torch's accounting and is returned when the plan goes."""
    w, s, fb = tiny
    want = hp.search(_plan(hp, w), fb)
    p = _plan(hp, w)
    p.use_torch_allocator()
    before = torch.cuda.memory_allocated()
    got = hp.search(p, fb)
    held = torch.cuda.memory_allocated() - before
    assert np.array_equal(got, want)
    assert held >= p.workspace_bytes(fb.shape[0])
    p.close()
    assert torch.cuda.memory_allocated() - before < held


def test_batch_with_rfi_matches_per_file(hp, torch):
    """A batch with RFI mitigation on, planted tones and spikes: each file
    equals the oracle's search of the oracle-cleaned input and its plain
    per-file search."""
    files = _small_batch(nfiles=3)
    xs, fbs = [], []
    for w in files:
        x = w.generate().data.astype(np.int32)
        x[:, [1, 2]] += 50
        x[::5000, :] += 60
        xs.append(np.clip(x, 0, 255).astype(np.uint8))
        fbs.append(torch.from_numpy(xs[-1]).cuda())
    plans = [_plan(hp, w, rfi=1) for w in files]
    want = [hp.search(p, fb) for p, fb in zip(plans, fbs)]
    b = hp.Batch(plans)
    first = b.search(fbs)
    for w, x, got in zip(files, xs, first):
        cleaned = oracle.rfi_clean(x, w.obs.tsamp).cleaned
        _compare_clusters(got, _oracle_search(w, cleaned).clusters, w.threshold)
    for _ in range(2):
        for g, w_ in zip(b.search(fbs), want):
            assert np.array_equal(g, w_)
    b.close()


@pytest.mark.parametrize("case", ["one_channel", "one_trial_one_width", "widest_boxcar"])
def test_degenerate_and_maximum_shapes(hp, torch, case):
    """One channel (every delay 0), a single trial and width, and the widest
    boxcar the library accepts (16384 samples, a detect halo four tiles long),
    each compared exactly with the oracle."""
    rng = np.random.default_rng({"one_channel": 1, "one_trial_one_width": 2,
                                 "widest_boxcar": 3}[case])
    if case == "one_channel":
        nch, nsamps, dms, widths = 1, 30000, np.array([0.0, 50.0], np.float32), [1, 2, 4, 8]
    elif case == "one_trial_one_width":
        nch, nsamps, dms, widths = 48, 20000, np.array([12.0], np.float32), [3]
    else:
        nch, nsamps, dms = 32, 120000, np.array([0.0, 20.0, 40.0], np.float32)
        widths = [1, 64, 4096, 16384]
    x = rng.normal(100, 10, size=(nsamps, nch))
    x[nsamps // 3: nsamps // 3 + 9] += 40
    x[nsamps // 2: nsamps // 2 + 20000] += 1.5      # a long weak plateau for the wide boxcars
    x = np.clip(np.rint(x), 0, 255).astype(np.uint8)
    widths = np.array(widths, np.int32)
    want = oracle.search(x, 1500.0, -2.0, 1e-3, dms, widths, 5.0)
    p = hp.Plan(nch, 1500.0, -2.0, 1e-3, dms, widths, 5.0)
    fb = torch.from_numpy(x).cuda()
    D = hp.hp_dedisperse(p, fb)
    tab = p.delays()
    assert np.array_equal(D[:, :p.nout(nsamps)].cpu().numpy(), oracle.dedisperse(x, tab))
    raw_g, sig_g, _ = hp.detect(p, D, p.nout(nsamps))
    assert np.array_equal(sig_g, want.sigma)
    assert _key(raw_g) == _key(want.raw) and len(want.raw) > 0
    _compare_clusters(hp.search(p, fb), want.clusters, 5.0)
