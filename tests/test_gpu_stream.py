"""Streamed search on the GPU (hp_stream_*), checked against the oracle's
gulp-by-gulp search (Sections III-B, V-C; the window / carry rule is written
out in oracle/hp_oracle.c and include/hp.h).

Each beam of the tiny band is pushed gulp by gulp; every gulp's merged
candidates must equal the oracle's: identical tuples and statistics, S/N
within 1e-4.  A beam's results must be the same alone and mixed with other
beams, and the same when a small device budget makes beams wait for a slot.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SNR_TOL = 1e-4
G = 4096
FIELDS = ("dm_idx", "width_idx", "sample", "members", "dm_lo", "dm_hi", "t_lo", "t_hi")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00398_gb300 as hp
    return torch, hp


@pytest.fixture(scope="module")
def beams(env):
    from paper_2512_00398_gb300 import workloads
    ws = workloads.stream_tiny(nbeams=3, ngulps=8, gulp=G)
    data = [w.generate().data for w in ws]
    want = []
    for w, d in zip(ws, data):
        o = w.obs
        want.append(oracle.stream_search(d, G, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                                         w.threshold))
    assert sum(len(r["clusters"]) for b in want for r in b) > 0
    return ws, data, want


def _plan(hp, w):
    o = w.obs
    return hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold)


def _run(hp, plan, data, order, **kw):
    """Push gulps in `order` ((beam, g) pairs), end every beam, poll all."""
    st = hp.Stream(plan, nbeams=len(data), gulp=G, **kw)
    for b, g in order:
        st.push(b, data[b][g * G:(g + 1) * G])
    for b in range(len(data)):
        st.end_beam(b)
    got, seq = {}, []
    while len(got) < len(order):
        r = st.poll(timeout_ms=120000)
        assert r is not None, "stream stalled"
        info, c = r
        assert info["status"] == hp.HP_OK
        got[(info["beam"], info["gulp_index"])] = (info, c)
        seq.append(info["beam"])
    stats = st.stats()
    st.close()
    return got, seq, stats


def _same(got, want):
    assert len(got) == len(want)
    for f in FIELDS:
        assert np.array_equal(got[f], want[f]), f
    if len(got):
        assert np.abs(got["snr"].astype(np.float64) - want["snr"]).max() <= SNR_TOL


def _round_robin(nbeams, ngulps):
    return [(b, g) for g in range(ngulps) for b in range(nbeams)]


def test_stream_matches_oracle(env, beams):
    torch, hp = env
    ws, data, want = beams
    plan = _plan(hp, ws[0])
    got, _, stats = _run(hp, plan, data, _round_robin(3, 8))
    for b in range(3):
        for r in want[b]:
            info, c = got[(b, r["g"])]
            assert info["window_start"] == r["B0"] and info["window_len"] == r["nwin"]
            _same(c, r["clusters"])
    assert stats["gulps"] == 24 and stats["max_batch_seen"] >= 2


def test_alone_equals_mix(env, beams):
    torch, hp = env
    ws, data, want = beams
    plan = _plan(hp, ws[0])
    mix, _, _ = _run(hp, plan, data, _round_robin(3, 8))
    for b in range(3):
        alone, _, _ = _run(hp, plan, [data[b]], [(0, g) for g in range(8)])
        for g in range(8):
            a, m = alone[(0, g)], mix[(b, g)]
            assert a[0]["window_start"] == m[0]["window_start"]
            assert np.array_equal(a[1], m[1])


def test_small_budget_makes_beams_wait(env, beams):
    torch, hp = env
    ws, data, want = beams
    plan = _plan(hp, ws[0])
    # device bytes of one step slot + one / two beam slots
    s1 = hp.Stream(plan, nbeams=1, gulp=G, max_batch=1)
    b1 = s1.stats()["device_bytes"]
    s1.close()
    s2 = hp.Stream(plan, nbeams=2, gulp=G, max_batch=1)
    b2 = s2.stats()["device_bytes"]
    s2.close()
    budget = b1 + (b2 - b1) // 2          # room for one beam slot only
    got, seq, stats = _run(hp, plan, data, _round_robin(3, 8), hbm_budget=budget)
    assert stats["beam_slots"] == 1 and stats["max_batch"] == 1
    # one beam at a time, in order of first push
    assert seq == sorted(seq)
    for b in range(3):
        for r in want[b]:
            _same(got[(b, r["g"])][1], r["clusters"])


def test_stream_argument_errors(env, beams):
    torch, hp = env
    ws, data, want = beams
    plan = _plan(hp, ws[0])
    st = hp.Stream(plan, nbeams=2, gulp=G)
    with pytest.raises(hp.HPError):
        st.push(0, data[0][:G - 64])                    # wrong size
    with pytest.raises(hp.HPError):
        st.push(5, data[0][:G])                         # no such beam
    assert st.poll(timeout_ms=50) is None               # nothing pushed
    st.push(1, data[1][:G])
    st.end_beam(1)
    with pytest.raises(hp.HPError):
        st.push(1, data[1][G:2 * G])                    # ended
    info, c = st.poll(timeout_ms=60000)
    assert info["beam"] == 1 and info["window_len"] == 0 and len(c) == 0
    st.close()
    with pytest.raises(hp.HPError):
        hp.Stream(plan, nbeams=2, gulp=G, hbm_budget=1 << 20)   # cannot hold one slot


def test_stream_with_rfi_matches_oracle(env, beams):
    """Each searched buffer cleaned on its own before the search (HP_PARAM_RFI)."""
    torch, hp = env
    ws, data, want = beams
    w = ws[0]
    o = w.obs
    x = data[0].astype(np.int32)
    x[:, [7, 90]] += 50
    x[::3001, :] += 60
    x = np.clip(x, 0, 255).astype(np.uint8)
    plan = _plan(hp, w)
    plan.set_param("rfi", 1)
    got, _, _ = _run(hp, plan, [x], [(0, g) for g in range(8)])
    ref = oracle.stream_search(x, G, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths,
                               w.threshold, rfi=(5, 5.0))
    for r in ref:
        _same(got[(0, r["g"])][1], r["clusters"])
