"""The merge entry point that allocates nothing (hp_merge_static).

Callers that must not allocate device memory while they run -- a real-time
pipeline that forbids cudaMalloc after start-up, or code inside a framework
that owns all device memory -- merge candidates with hp_merge_static, whose
scratch is a fixed array built into the library.  These checks call it
through the C ABI twice in a row (the two calls share that array) and compare
each result with hp_merge's, with the tolerance the other parity tests use:
identical tuples and statistics, S/N within 1e-4.  They also check that it
refuses more raw candidates than its array holds.
"""
import numpy as np
import pytest

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


def test_static_merge_matches_merge_on_two_calls(setup):
    torch, hp, w, raw, cnt, sigma, ref = setup
    for _ in range(2):
        data, count = hp.hp_merge_static(raw, cnt, sigma, w.widths)
        torch.cuda.synchronize()
        _same(hp.cands_to_numpy(data, count), ref)


def test_static_merge_rejects_oversized_input(setup):
    torch, hp, w, raw, cnt, sigma, ref = setup
    big = torch.zeros((hp.HP_MERGE_STATIC_MAX_RAW + 1) * hp.RAW_DTYPE.itemsize, dtype=torch.uint8,
                      device=raw.device)
    with pytest.raises(hp.HPError) as e:
        hp.hp_merge_static(big, cnt, sigma, w.widths)
    assert e.value.code == hp.HP_ERR_INVALID_ARG
