"""The N > 1 path of the benchmark on CPU: two ranks over gloo.

The search shards by file (every rank its own file, no exchange), so the only
multi-rank logic is the per-rank workload, the max-over-ranks timing and the
whole-job aggregate; the reference arm runs on rank 0 only.  These run as two
processes on 127.0.0.1 with the gloo backend.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 0.5 * rank], dist, "cpu")
        w = bench.rank_workload(rank, world, 1 << 17)
        out.put((rank, got, w.seed, w.obs.nchans, w.obs.nsamps, w.ndm))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_and_weak_scaling_workloads():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q), daemon=True) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, s0, c0, n0, d0), (r1, m1, s1, c1, n1, d1) = res
    assert m0 == m1 == [2.0, 5.0, 0.5]          # the slowest rank sets each time
    assert s0 != s1                             # a different file per rank
    assert (c0, n0, d0) == (c1, n1, d1)         # of the same shape (weak scaling)


def test_aggregate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2, 1000, 0.5) == 4000.0
    assert bench.aggregate(1, 1000, 0.5) == 2000.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def _worker_one_fails(rank, world, port, out):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=10))
    bench.max_over_ranks([1.0 + rank], dist, "cpu")      # step 1: both ranks
    if rank == 1:
        os._exit(3)                  # this rank dies between steps
    try:
        bench.max_over_ranks([1.0], dist, "cpu")          # step 2: the survivor alone
        out.put((rank, "no error"))
    except Exception as e:           # the survivor learns of it on the host
        out.put((rank, type(e).__name__))


def test_a_failed_rank_ends_the_survivors_exchange_with_an_error():
    torch = pytest.importorskip("torch")
    import queue
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker_one_fails, args=(r, 2, port, q), daemon=True)
             for r in range(2)]
    for p in procs:
        p.start()
    try:
        rank, what = q.get(timeout=120)
    except queue.Empty:
        rank, what = None, "survivor never returned"
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():         # our own child: end it by its handle
                p.kill()
                p.join(timeout=30)
    assert rank == 0 and what not in ("no error", "survivor never returned"), what
    assert procs[1].exitcode == 3
