"""The multi-rank benchmark logic on CPU: two gloo ranks, replicas with no collective
on the data path; the job time is the slowest rank's and the rate counts every
rank's units."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [120.0, 300.0][rank]
    m = bench.max_over_ranks(local_ms, dist)
    rate = bench.whole_job_rate(1000, world, 10, m)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, rate))


def test_two_gloo_ranks_take_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in out] == [300.0, 300.0]
    assert all(abs(rate - 2 * 1000 * 10 / 0.3) < 1e-6 for _, _, rate in out)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(5.0) == 5.0
    assert bench.whole_job_rate(10, 1, 2, 1000.0) == 20.0
