"""With HP_PARAM_FUSE_LEVELS = 1 the dedispersion kernel forms the second
remedian level (medians of the five medians of five consecutive sums) of every
25-sample group inside one of its time tiles while the sums are still on chip;
the search forms the groups that straddle a tile edge or the end of the series
from D and starts its remedian from those values (Section II-B: baseline
removal after dedispersion).

With a baseline window of 25-124 samples the second level is the knot series
itself (L = 2), so any wrong group value moves the baseline of the samples
around it; with 125-624 samples (L = 3) one remedian pass runs over it.  Every
tile shape (tile lengths 384-2432 samples, one or two trials per warp, one or
two warps along time) is compared with the oracle's search at a low threshold
(many candidates); so are batches of uneven files and streamed gulps, which
take the fused levels too.
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


def _compare(got, want, thr):
    g = {(int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"])): c for c in got}
    w = {(int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"])): c for c in want}
    near = {k for k, c in w.items() if abs(float(c["snr"]) - thr) <= SNR_TOL}
    assert set(g) - near == set(w) - near
    for k in set(w) - near:
        assert abs(float(g[k]["snr"]) - float(w[k]["snr"])) <= SNR_TOL, k
        for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
            assert int(g[k][f]) == int(w[k][f]), (k, f)


@pytest.fixture(scope="module")
def tiny(torch):
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    s = w.generate()
    return w, s, torch.from_numpy(s.data).cuda()


THR = 3.5


@pytest.fixture(scope="module")
def tiny_oracle(tiny):
    w, s, _ = tiny
    o = w.obs
    out = {}
    for bs in (0.002, 0.01):
        out[bs] = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, THR,
                                baseline_s=bs).clusters
    return out


@pytest.mark.parametrize("baseline_s", [0.002, 0.01])
@pytest.mark.parametrize("cfg", list(range(20)))
def test_fused_levels_every_tile_shape(hp, torch, tiny, tiny_oracle, cfg, baseline_s):
    w, s, fb = tiny
    o = w.obs
    assert oracle.remedian_levels(oracle.baseline_window(baseline_s, o.tsamp)) == \
        (2 if baseline_s == 0.002 else 3)
    want = tiny_oracle[baseline_s]
    assert len(want) > 50
    p = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, THR,
                baseline_s=baseline_s, dedisp_config=cfg, fuse_levels=1)
    got = hp.search(p, fb)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    _compare(got, want, THR)


@pytest.mark.parametrize("cfg", [0, 3, 12, 17, 19])
@pytest.mark.parametrize("tail", ["inside", "edge"])
def test_fused_levels_ragged(hp, torch, cfg, tail):
    """Odd channel count, duplicate and widely spaced trials; a series that
    ends inside a 25-sample group and one that ends on a group edge (L = 2)."""
    from paper_2512_00398_gb300 import synth
    rng = np.random.default_rng(13)
    nch = 100
    dms = np.sort(np.concatenate([[0, 0, 3.5, 3.5], rng.uniform(0, 900, 37), [1500.0]]))
    dms = dms.astype(np.float32)
    widths = synth.widths_pow2(16)
    p = hp.Plan(nch, 1450.0, -3.0, 1e-4, dms, widths, THR, baseline_s=0.004, dedisp_config=cfg,
                fuse_levels=1)
    maxd = p.max_delay
    nsamps = 26011 if tail == "inside" else maxd + 25 * ((26011 - maxd) // 25)
    nout = p.nout(nsamps)
    assert (nout % 25 == 0) == (tail == "edge")
    assert oracle.remedian_levels(oracle.baseline_window(0.004, 1e-4)) == 2
    x = rng.normal(128, 14, size=(nsamps, nch)).round().clip(0, 255).astype(np.uint8)
    x[rng.integers(0, nsamps, 30)] = 255
    want = oracle.search(x, 1450.0, -3.0, 1e-4, dms, widths, THR, baseline_s=0.004).clusters
    assert len(want) > 50
    got = hp.search(p, torch.from_numpy(x).cuda())
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    _compare(got, want, THR)


@pytest.mark.parametrize("baseline_s", [0.002, 2.0])
def test_fused_levels_param_same_results(hp, torch, tiny, baseline_s):
    """HP_PARAM_FUSE_LEVELS = 0 (the default: the remedian reads D) and 1 give
    the same clusters; the parameter takes only 0 and 1."""
    w, s, fb = tiny
    o = w.obs
    p = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, THR,
                baseline_s=baseline_s)
    assert p.get_param("fuse_levels") == 0
    plain = hp.search(p, fb)
    p.set_param("fuse_levels", 1)
    fused = hp.search(p, fb)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    assert len(fused) > 0 and np.array_equal(fused, plain)
    for bad in (-1, 0.5, 2):
        with pytest.raises(hp.HPError):
            p.set_param("fuse_levels", bad)


def test_fused_levels_batch(hp, torch):
    """Uneven files (1024-4096 channels, 49.152 and 64 us) as one batch with the
    fused levels, every file equal to the oracle's search of it."""
    from paper_2512_00398_gb300 import workloads
    files = workloads.batch(nfiles=4, seed0=350, len_lo=1 << 16, len_hi=1 << 17, dm_hi=300.0,
                            trial_density=0.4, wmax=256)
    gens = [w.generate() for w in files]
    plans = [hp.Plan(w.obs.nchans, w.obs.f_top, w.obs.chan_bw, w.obs.tsamp, w.dm_list, w.widths,
                     4.0, baseline_s=0.005, fuse_levels=1) for w in files]
    b = hp.Batch(plans)
    got = b.search([torch.from_numpy(g.data).cuda() for g in gens])
    assert b.sync_status() == hp.HP_OK
    n = 0
    for w, g, c in zip(files, gens, got):
        o = w.obs
        want = oracle.search(g.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                             4.0, baseline_s=0.005).clusters
        _compare(c, want, 4.0)
        n += len(want)
    assert n > 100
    b.close()


def test_fused_levels_stream(hp, torch):
    """Gulps of three beams with the fused levels (L = 3), every gulp's
    clusters equal to the oracle's streamed search."""
    from paper_2512_00398_gb300 import workloads
    G = 4096
    ws = workloads.stream_tiny(nbeams=3, ngulps=6, gulp=G)
    data = [w.generate().data for w in ws]
    o = ws[0].obs
    p = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, ws[0].dm_list, ws[0].widths,
                ws[0].threshold, baseline_s=0.01, fuse_levels=1)
    st = hp.Stream(p, nbeams=3, gulp=G)
    for g in range(6):
        for b in range(3):
            st.push(b, data[b][g * G:(g + 1) * G])
    for b in range(3):
        st.end_beam(b)
    got = {}
    while len(got) < 18:
        r = st.poll(timeout_ms=120000)
        assert r is not None, "stream stalled"
        info, c = r
        assert info["status"] == hp.HP_OK
        got[(info["beam"], info["gulp_index"])] = c
    st.close()
    n = 0
    for b, w in enumerate(ws):
        want = oracle.stream_search(data[b], G, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                                    w.threshold, baseline_s=0.01)
        for r in want:
            c = got[(b, r["g"])]
            assert len(c) == len(r["clusters"])
            for f in ("dm_idx", "width_idx", "sample", "members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
                assert np.array_equal(c[f], r["clusters"][f]), f
            if len(c):
                assert np.abs(c["snr"].astype(np.float64) - r["clusters"]["snr"]).max() <= SNR_TOL
            n += len(c)
    assert n > 0
