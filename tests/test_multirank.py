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


def _slab_rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import slabs

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    v, t = mg.clipped_kuhn_lattice(10, 0.25, 21, mg.torus_sdf(0.3, 0.12))
    res3, h = (40, 36, 44), 1.0 / 44
    w = slabs.slice_weights(v, t, (0, 0, 0), h, res3[2])
    z0, z1 = slabs.rank_slab(res3[2], rank, world, w)
    mine = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3, z0=z0, z1=z1)
    got = [None] * world
    dist.all_gather_object(got, (z0, z1, mine))
    dist.destroy_process_group()
    full = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3)
    cat = np.concatenate([g for _, _, g in sorted(got, key=lambda x: x[0])], axis=0)
    q.put((rank, (z0, z1), bool((cat == full).all()), [c[:2] for c in got]))


def test_two_gloo_ranks_slabs_concatenate_to_grid():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, _, ok, _ in out)
    (a0, a1), (b0, b1) = out[0][1], out[1][1]
    assert a0 == 0 and a1 == b0 and b1 == 44 and 0 < a1 < 44


def test_slab_cuts_cover_and_balance():
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2106_01326_gb300 import slabs

    assert slabs.slab_cuts(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slabs.slab_cuts(2, 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]
    assert slabs.slab_cuts(0, 2) == [(0, 0), (0, 0)]
    w = np.zeros(100)
    w[60:80] = 1.0  # all the work in slices 60..79
    cuts = slabs.slab_cuts(100, 4, w)
    assert cuts[0][0] == 0 and cuts[-1][1] == 100
    assert all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
    shares = [w[a:b].sum() for a, b in cuts]
    assert max(shares) == 5.0 and min(shares) == 5.0
    with pytest.raises(ValueError):
        slabs.slab_cuts(5, 0)


def _slab_rank_gpu_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import slabs
    from paper_2106_01326_gb300 import voxtet as vt

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    v, t = mg.clipped_kuhn_lattice(16, 0.25, 21, mg.torus_sdf(0.3, 0.12))
    res3, h = (200, 180, 220), 1.0 / 220
    w = slabs.slice_weights(v, t, (0, 0, 0), h, res3[2])
    z0, z1 = slabs.rank_slab(res3[2], rank, world, w)
    sv, st = slabs.slab_mesh(v, t, (0, 0, 0), h, z0, z1)  # this rank's tets and only their vertices
    out = []
    for kernel in (vt.KERNEL_SPANS, vt.KERNEL_SLICES):
        g = vt.voxelize_grid(torch.from_numpy(sv).cuda(), torch.from_numpy(st).cuda(), (0, 0, 0), h, res3,
                             z_range=(z0, z1), kernel=kernel)
        out.append(g.cpu().numpy().view(np.uint32))
    got = [None] * world
    dist.all_gather_object(got, (z0, z1, out[0], out[1]))
    dist.destroy_process_group()
    full = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3)
    parts = sorted(got, key=lambda x: x[0])
    ok = [bool((np.concatenate([p[2 + k] for p in parts], axis=0) == full).all()) for k in range(2)]
    q.put((rank, (z0, z1), ok))


@pytest.mark.gpu
def test_two_gloo_ranks_cuda_slabs_concatenate_to_oracle_grid():
    """Each of two gloo ranks voxelizes its weighted z-slab through the CUDA path (both work
    distributions) from its own compacted mesh; the gathered slabs equal the oracle's whole grid."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2106_01326_gb300 import build as vbuild

    vbuild.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_rank_gpu_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(all(ok) for _, _, ok in out), out
    (a0, a1), (b0, b1) = out[0][1], out[1][1]
    assert a0 == 0 and a1 == b0 and b1 == 220 and 0 < a1 < 220
