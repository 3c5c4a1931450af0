"""Candidate merging on the GPU (hp_merge) against the oracle's merge at the
scale of the full searches.

The raw lists are seeded (tests/raw_lists.py), with the size of the FAST-file
search's raw output and of the stress search's, so that the merge runs
through many sort chunks and merge passes; each list is merged by hp_merge
through the C ABI and by the oracle, and the clusters must match exactly
(tuples, members, trial and time ranges), S/N within 1e-4.
"""
import numpy as np
import pytest

import oracle
from tests.raw_lists import raw_list

pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00398_gb300 as hp
    return torch, hp


def _same(got, want):
    key = lambda c: (int(c["dm_idx"]), int(c["sample"]), int(c["width_idx"]))
    assert [key(c) for c in got] == [key(c) for c in want]
    for f in ("members", "dm_lo", "dm_hi", "t_lo", "t_hi"):
        assert np.array_equal(got[f].astype(np.int64), want[f].astype(np.int64)), f
    assert np.abs(got["snr"].astype(np.float64) - want["snr"]).max() <= SNR_TOL


@pytest.mark.parametrize("case", ["fast", "stress"])
def test_merge_matches_oracle_at_search_scale(env, case):
    """fast: 300 000 raw candidates over 1500 trials and 955 060 starts, 13
    widths; stress: 3 000 000 over 4000 trials and 1 854 597 starts, 14 widths,
    with dm_tol 2 and t_gap 4 (larger clusters)."""
    torch, hp = env
    from paper_2512_00398_gb300 import synth
    if case == "fast":
        n, ndm, nout, wmax, tol = 300_000, 1500, 955_060, 4096, (1, 0)
        seed = 11
    else:
        n, ndm, nout, wmax, tol = 3_000_000, 4000, 1_854_597, 8192, (2, 4)
        seed = 12
    widths = synth.widths_pow2(wmax)
    recs, sigma = raw_list(seed, n, ndm=ndm, nout=nout, nw=widths.size)
    want = oracle.merge(oracle.raw_with_snr(recs, sigma, widths), widths, dm_tol=tol[0],
                        t_gap=tol[1])
    dms = np.linspace(0.0, 2000.0, ndm).astype(np.float32)
    p = hp.Plan(4096, 1500.0, -500.0 / 4096, 49.152e-6, dms, widths, 6.0,
                raw_capacity=recs.size, dm_tol=tol[0], t_gap=tol[1])
    host = np.zeros(recs.size, hp.RAW_DTYPE)
    for f in ("dm_idx", "width_idx", "sample", "S"):
        host[f] = recs[f]
    raw = torch.from_numpy(host.view(np.uint8).copy()).cuda()
    cnt = torch.tensor([recs.size], dtype=torch.int64, device="cuda")
    sig = torch.from_numpy(sigma.astype(np.float64)).cuda()
    data, count = hp.hp_merge(p, raw, cnt, sig, capacity=want.size + 16)
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
    got = hp.cands_to_numpy(data, count)
    assert int(count.item()) == want.size and want.size > 1000
    assert int(got["members"].sum()) == recs.size
    _same(got, want)
