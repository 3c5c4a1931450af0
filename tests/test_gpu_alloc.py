"""No device allocation in steady state.

The paper counts cudaMalloc calls (Section V-B, Table II: 198 392 for
Heimdall, 4 810 with its shared allocator) because allocating inside the
per-trial loop was a bottleneck.  Here every plan sizes its device memory up
front: the first search allocates the plan's tables and workspace, and after
that repeated searches, batch calls (eager, captured, replayed) and stream
steps make no allocation request at all.  Counted twice: at the allocator
hook (hp_plan_set_allocator) and by the library's own counters
(hp_stats.device_allocs, hp_stream_stats.device_allocs).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_00398_gb300 as hp
    return torch, hp


def _plan(hp, w, **kw):
    o = w.obs
    return hp.Plan(o.nchans, o.f_top, o.chan_bw, o.tsamp, w.dm_list, w.widths, w.threshold, **kw)


class Counting:
    """An allocator hook that takes memory from torch's caching allocator and
    counts the library's requests."""

    def __init__(self, torch):
        self.torch = torch
        self.allocs = 0
        self.frees = 0

    def alloc(self, n):
        self.allocs += 1
        return self.torch.cuda.caching_allocator_alloc(n)

    def free(self, ptr, n):
        self.frees += 1
        self.torch.cuda.caching_allocator_delete(ptr)


def test_repeated_searches_allocate_nothing(env):
    torch, hp = env
    from paper_2512_00398_gb300 import workloads
    w = workloads.tiny()
    fb = torch.from_numpy(w.generate().data).cuda()
    hook = Counting(torch)
    p = _plan(hp, w)
    p.use_allocator(hook.alloc, hook.free)
    first = hp.search(p, fb)
    n0 = hook.allocs
    assert n0 > 0 and hp.hp_plan_stats(p)["device_allocs"] == n0
    for _ in range(5):
        assert np.array_equal(hp.search(p, fb), first)
    assert hook.allocs == n0 and hook.frees == 0
    assert hp.hp_plan_stats(p)["device_allocs"] == n0
    # the same with the library's own cudaMalloc
    q = _plan(hp, w)
    hp.search(q, fb)
    m0 = hp.hp_plan_stats(q)["device_allocs"]
    assert m0 > 0
    for _ in range(5):
        hp.search(q, fb)
    assert hp.hp_plan_stats(q)["device_allocs"] == m0
    p.close()
    assert hook.frees == hook.allocs


def test_batch_calls_allocate_nothing_after_the_first(env):
    """Eager first call, then capture and replays of the CUDA graph."""
    torch, hp = env
    from paper_2512_00398_gb300 import workloads
    files = workloads.batch(nfiles=3, seed0=350, len_lo=1 << 16, len_hi=1 << 17, dm_hi=300.0,
                            trial_density=0.4, wmax=256)
    fbs = [torch.from_numpy(f.generate().data).cuda() for f in files]
    hooks = [Counting(torch) for _ in files]
    plans = [_plan(hp, f) for f in files]
    for p, h in zip(plans, hooks):
        p.use_allocator(h.alloc, h.free)
    b = hp.Batch(plans)
    first = b.search(fbs)
    n0 = [h.allocs for h in hooks]
    s0 = [hp.hp_plan_stats(p)["device_allocs"] for p in plans]
    assert all(n > 0 for n in n0) and s0 == n0
    for _ in range(4):
        for g, f in zip(b.search(fbs), first):
            assert np.array_equal(g, f)
    assert [h.allocs for h in hooks] == n0
    assert [hp.hp_plan_stats(p)["device_allocs"] for p in plans] == s0
    b.close()


def test_stream_steps_allocate_nothing(env):
    """All of a stream's device memory is taken at open; pushing and searching
    every gulp of three beams adds none."""
    torch, hp = env
    from paper_2512_00398_gb300 import workloads
    G = 4096
    ws = workloads.stream_tiny(nbeams=3, ngulps=6, gulp=G)
    data = [w.generate().data for w in ws]
    st = hp.Stream(_plan(hp, ws[0]), nbeams=3, gulp=G)
    a0 = st.stats()["device_allocs"]
    assert a0 >= 1
    n = 0
    for g in range(6):
        for b in range(3):
            st.push(b, data[b][g * G:(g + 1) * G])
            n += 1
    for b in range(3):
        st.end_beam(b)
    done = 0
    while done < n:
        r = st.poll(timeout_ms=120000)
        assert r is not None, "stream stalled"
        assert r[0]["status"] == hp.HP_OK
        done += 1
    stats = st.stats()
    assert stats["gulps"] == n and stats["device_allocs"] == a0
    st.close()
