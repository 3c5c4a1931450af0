"""The merge entry point that allocates nothing (hp_merge_static).

Callers that must not allocate device memory while they run -- a real-time
pipeline that forbids cudaMalloc after start-up, or code inside a framework
that owns all device memory -- merge candidates with hp_merge_static, whose
scratch is a fixed array built into the library.  These checks call it
through the C ABI twice in a row (the two calls share that array) and compare
each result with hp_merge's and with the CPU oracle's merge of the same raw
list, with the tolerance the other parity tests use: identical tuples and
statistics, S/N within 1e-4.  They also check that a raw count beyond the
buffer is reported through the status word, and that inputs the array cannot
hold and out-of-range tolerances are refused.
"""
import numpy as np
import pytest

import oracle
from tests.raw_lists import raw_list

pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4
FIELDS = ("dm_idx", "width_idx", "sample", "members", "dm_lo", "dm_hi", "t_lo", "t_hi")


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00398_gb300 as hp
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    s = w.generate()
    o = w.obs
    plan = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    fb = torch.from_numpy(s.data).cuda()
    D = hp.hp_dedisperse(plan, fb)
    raw, cnt, sigma, _ = hp.hp_detect(plan, D, plan.nout(fb.shape[0]),
                                      capacity=hp.HP_MERGE_STATIC_MAX_RAW)
    data, count = hp.hp_merge(plan, raw, cnt, sigma)
    assert hp.hp_plan_sync_status(plan) == hp.HP_OK
    ref = hp.cands_to_numpy(data, count)
    assert 0 < int(cnt.item()) <= hp.HP_MERGE_STATIC_MAX_RAW and len(ref) > 0
    return torch, hp, w, raw, cnt, sigma, ref


def _same(got, ref):
    assert len(got) == len(ref)
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f
    assert np.abs(got["snr"].astype(np.float64) - ref["snr"]).max() <= SNR_TOL


def _upload(torch, hp, recs, sigma):
    """A raw list and its sigmas as the device buffers hp_detect would write."""
    host = np.zeros(recs.size, hp.RAW_DTYPE)
    for f in ("dm_idx", "width_idx", "sample", "S"):
        host[f] = recs[f]
    raw = torch.from_numpy(host.view(np.uint8).copy()).cuda()
    cnt = torch.tensor([recs.size], dtype=torch.int64, device="cuda")
    sig = torch.from_numpy(np.ascontiguousarray(sigma, dtype=np.float64)).cuda()
    return raw, cnt, sig


def test_static_merge_matches_merge_on_two_calls(setup):
    torch, hp, w, raw, cnt, sigma, ref = setup
    for _ in range(2):
        data, count = hp.hp_merge_static(raw, cnt, sigma, w.widths)
        torch.cuda.synchronize()
        _same(hp.cands_to_numpy(data, count), ref)


def test_static_merge_matches_oracle_on_two_calls(setup):
    """A seeded list of 60 000 raw candidates (clusters over neighbouring
    trials, times and widths, plus isolated ones): both calls equal the
    oracle's merge of the same list."""
    torch, hp, w, _, _, _, _ = setup
    widths = np.array([1, 2, 4, 8, 16, 32, 64, 128], np.int32)
    recs, sigma = raw_list(3, 60000, ndm=400, nout=200000, nw=widths.size)
    assert recs.size <= hp.HP_MERGE_STATIC_MAX_RAW
    want = oracle.merge(oracle.raw_with_snr(recs, sigma, widths), widths)
    raw, cnt, sig = _upload(torch, hp, recs, sigma)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        data, count = hp.hp_merge_static(raw, cnt, sig, widths, capacity=1 << 16, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == hp.HP_OK
        _same(hp.cands_to_numpy(data, count), want)


def test_static_merge_reports_count_beyond_buffer(setup):
    """A device count larger than the buffer: the first raw_capacity entries
    are merged (equal to the oracle's merge of that prefix) and the status
    word says HP_ERR_CAND_OVERFLOW."""
    torch, hp, w, _, _, _, _ = setup
    widths = np.array([1, 2, 4, 8], np.int32)
    recs, sigma = raw_list(4, 5000, ndm=64, nout=50000, nw=widths.size)
    keep = 3000
    want = oracle.merge(oracle.raw_with_snr(recs[:keep], sigma, widths), widths)
    raw, _, sig = _upload(torch, hp, recs[:keep], sigma)
    cnt = torch.tensor([recs.size], dtype=torch.int64, device="cuda")   # more than the buffer holds
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    data, count = hp.hp_merge_static(raw, cnt, sig, widths, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == hp.HP_ERR_CAND_OVERFLOW
    _same(hp.cands_to_numpy(data, count), want)


def test_static_merge_rejects_oversized_input_and_bad_tolerances(setup):
    torch, hp, w, raw, cnt, sigma, ref = setup
    big = torch.zeros((hp.HP_MERGE_STATIC_MAX_RAW + 1) * hp.RAW_DTYPE.itemsize, dtype=torch.uint8,
                      device=raw.device)
    with pytest.raises(hp.HPError) as e:
        hp.hp_merge_static(big, cnt, sigma, w.widths)
    assert e.value.code == hp.HP_ERR_INVALID_ARG
    for kw in ({"dm_tol": -1}, {"dm_tol": (1 << 20) + 1}, {"w_tol": 33}, {"t_gap": 10 ** 16},
               {"t_gap": -10 ** 16}):
        with pytest.raises(hp.HPError) as e:
            hp.hp_merge_static(raw, cnt, sigma, w.widths, **kw)
        assert e.value.code == hp.HP_ERR_INVALID_ARG, kw
