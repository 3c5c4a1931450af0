"""Failure detection without a GPU fault: the bounded device waits.

Every staged kernel waits on shared-memory barriers for its bulk copies with a
time limit; a wait that runs out latches HP_ERR_TIMEOUT, raises the block's
abort flag and returns, so the launch ends with a status the host reads and
the context stays usable.  The self-test makes a wait run out on a barrier
that nothing completes and checks the status, the abort path and a barrier
that does complete; a search afterwards still matches the oracle.
"""
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_wait_runs_out_with_a_status(torch):
    import paper_2512_00398_gb300 as hp
    for limit_ns in (2_000_000, 50_000_000):
        t0 = time.perf_counter()
        r = hp.hp_selftest_bounded_wait(limit_ns)
        dt = time.perf_counter() - t0
        assert r["status"] == hp.HP_ERR_TIMEOUT
        assert r["warp0_ran_out"] and r["warp1_gave_up"]
        assert r["completed_wait_ok"]
        assert dt >= limit_ns * 1e-9 and dt < limit_ns * 1e-9 + 30.0


def test_context_usable_after_a_timeout(torch):
    import paper_2512_00398_gb300 as hp
    from paper_2512_00398_gb300 import workloads
    assert hp.hp_selftest_bounded_wait(1_000_000)["status"] == hp.HP_ERR_TIMEOUT
    w = workloads.tiny()
    s = w.generate()
    o = w.obs
    p = hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)
    got = hp.dedisperse(p, torch.from_numpy(s.data).cuda())
    tab = oracle.delays(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list)
    assert np.array_equal(got, oracle.dedisperse(s.data, tab))
    assert hp.hp_plan_sync_status(p) == hp.HP_OK
