"""The multi-rank path of bench.py on the CPU: two gloo ranks on 127.0.0.1 reduce the timed
region to the slowest rank's time, the job rate counts every rank's units over that time,
and each rank reconstructs its own scan (seed + rank)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 5.0 * rank                  # the ranks' own timed regions
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.job_rate(1000, world, slowest, 4)
        s = bench.make_workload("small", rank)
        q.put((rank, slowest, rate, float(s.frames.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[1] for r in res] == [15.0, 15.0]                  # max over ranks, on every rank
    assert res[0][2] == pytest.approx(1000 * 2 * 4 / 0.015)     # all ranks' units / slowest time
    assert res[0][3] != res[1][3]                               # one scan per rank


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_rate(10, 1, 1000.0, 3) == pytest.approx(30.0)
