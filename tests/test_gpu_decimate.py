"""Decimated boxcars (HP_PARAM_DECIMATE) on the GPU against the oracle.

The wide widths run as boxcars of R samples on the series summed in blocks of
W / R; their candidates must be the oracle's (tuples and sums exact, samples on
the start grid), alone, with per-width sigmas, from hp_detect, in batches.
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


def _same_clusters(got, want):
    key = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
    assert [key(c) for c in got] == [key(c) for c in want]
    for a, b in zip(got, want):
        assert abs(float(a["snr"]) - float(b["snr"])) <= SNR_TOL
        for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
            assert int(a[f]) == int(b[f])


@pytest.mark.parametrize("R", [2, 8, 32])
@pytest.mark.parametrize("width_sigma", [0, 1])
def test_search_matches_oracle(hp, torch, tiny, R, width_sigma):
    w, s, fb = tiny
    o = w.obs
    want = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         decimate=R, width_sigma=bool(width_sigma))
    got = hp.search(_plan(hp, w, decimate=R, width_sigma=width_sigma), fb)
    assert len(want.clusters) > 0
    _same_clusters(got, want.clusters)


def test_detect_raw_exact_on_the_grid(hp, torch, tiny):
    w, s, fb = tiny
    o = w.obs
    D = oracle.dedisperse(s.data, oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list))
    R = 4
    raw_g, _, _ = hp.detect(_plan(hp, w, decimate=R), torch.from_numpy(D).cuda(), D.shape[1])
    raw_o, _, _ = oracle.search_trials(D, 0, o.tsamp, w.widths, w.threshold, decimate=R)
    key = lambda rows: sorted((int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"]), int(r["S"]))
                              for r in rows)
    assert key(raw_g) == key(raw_o) and len(raw_o) > 0
    for r in raw_g:
        W = int(w.widths[r["width_idx"]])
        if W > R:
            assert int(r["sample"]) % (W // R) == 0


def test_batch_and_refusals(hp, torch, tiny):
    """A batched search with decimated boxcars equals the oracle's and the
    plain per-file search; streams and a negative R are refused."""
    w, s, fb = tiny
    o = w.obs
    want = hp.search(_plan(hp, w, decimate=8), fb)
    ref = oracle.search(s.data, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                        decimate=8).clusters
    b = hp.Batch([_plan(hp, w, decimate=8)])
    for i in range(3):
        got = b.search([fb])[0]
        if i == 0:
            assert len(ref) > 0
            _same_clusters(got, ref)
        assert np.array_equal(got, want)
    b.close()
    with pytest.raises(hp.HPError):
        hp.Stream(_plan(hp, w, decimate=8), nbeams=1, gulp=4096)
    with pytest.raises(hp.HPError):
        _plan(hp, w, decimate=-1)


def test_all_variants_together(hp, torch, tiny):
    """RFI mitigation, sub-band dedispersion, per-width sigmas and decimated
    boxcars at once: the oracle cleans, dedisperses with the effective table,
    normalises per width and tests the wide widths on their grids."""
    w, s, fb = tiny
    o = w.obs
    x = s.data.astype(np.int32)
    x[:, [9, 60]] += 50
    x[::3100, :] += 45
    x = np.clip(x, 0, 255).astype(np.uint8)
    clean = oracle.rfi_clean(x, o.tsamp).cleaned
    want = oracle.search(clean, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold,
                         subband=(32, 4), width_sigma=True, decimate=8)
    p = _plan(hp, w, rfi=1, subband_chans=32, subband_group=4, width_sigma=1, decimate=8)
    got = hp.search(p, torch.from_numpy(x).cuda())
    assert len(want.clusters) > 0
    _same_clusters(got, want.clusters)


def test_block_sizes_that_do_not_chain(hp, torch):
    """Widths 5, 10, 15, 30 with R = 5: block sizes 2, 3 and 6 -- the series
    for 3 is summed from y itself (3 is not a multiple of 2), the one for 6 from
    the series for 3."""
    rng = np.random.default_rng(17)
    nout, ndm = 30011, 3
    widths = np.array([1, 5, 10, 15, 30], np.int32)
    D = np.rint(rng.normal(5000, 30, (ndm, nout))).astype(np.int32)
    D[0, 7000:7030] += 60
    D[1, 12000:12011] += 90
    D[2, 20000:20090] += 25
    p = hp.Plan(64, 1500.0, -1.0, 1e-3, np.zeros(ndm, np.float32), widths, 6.0, decimate=5)
    raw_g, _, _ = hp.detect(p, torch.from_numpy(D).cuda(), nout)
    raw_o, _, _ = oracle.search_trials(D, 0, 1e-3, widths, 6.0, decimate=5)
    key = lambda rows: sorted((int(r["dm_idx"]), int(r["sample"]), int(r["width_idx"]), int(r["S"]))
                              for r in rows)
    assert key(raw_g) == key(raw_o) and len(raw_o) > 0
    assert {int(r["width_idx"]) for r in raw_o} >= {2, 3}
