"""Serving: continuous batching gives every request the grid it gets alone.

A small arena forces admission stalls, several plan slots keep batches in flight
at once, and every finished request's grid is compared bit for bit with the same
request voxelized alone, and, in a stream of more than 200 requests that includes
the pool's largest and smallest meshes, with the CPU oracle's grid.  The
autotuner is exercised on the same meshes.
"""
import numpy as np
import pytest

import oracle
from paper_2106_01326_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2106_01326_gb300 import batch, server
    from paper_2106_01326_gb300 import build as vbuild
    from paper_2106_01326_gb300 import voxtet

    vbuild.build()
    voxtet.load()
    pool = [batch.Mesh.from_numpy(v, t) for v, t in mg.mesh_pool(6, seed=91, tets_lo=500, tets_hi=60000)]
    return voxtet, batch, server, pool


def _alone(vt, pool, cache, mesh_id, res):
    key = (mesh_id, res)
    if key not in cache:
        m = pool[mesh_id]
        cache[key] = vt.voxelize(m.verts, m.tets, (0, 0, 0), 1.0 / res, res)
    return cache[key]


@pytest.mark.parametrize("realtime", [True, False])
def test_served_results_equal_alone(env, realtime):
    import torch

    vt, batch, server, pool = env
    reqs = mg.poisson_stream(90, rate_per_s=3000.0, n_pool=len(pool), seed=5, resolutions=(16, 32, 64, 128, 256))
    cache = {}
    seen = []

    def check(tk, grid):
        ref = _alone(vt, pool, cache, tk.mesh_id, tk.res)
        seen.append((tk.rid, bool(torch.equal(grid, ref))))

    # arena for about five 256^3 grids: admissions have to wait for memory
    srv = server.Server(pool, arena_bytes=5 * server.grid_bytes(256), n_slots=3,
                        slot_workspace_bytes=64 << 20, max_jobs=8, on_result=check)
    try:
        rep = srv.serve(reqs, realtime=realtime)
    finally:
        srv.close()
    assert len(seen) == len(reqs)
    assert all(ok for _, ok in seen), [rid for rid, ok in seen if not ok]
    assert all(t.status == vt.OK for t in rep.tickets)
    s = rep.summary()
    assert s["batches"] > 3
    assert rep.peak_arena_bytes <= 5 * server.grid_bytes(256) + 4096
    if not realtime:
        assert rep.admission_stalls > 0
        # batches on different slots overlapped in time
        spans = [(t.launched_s, t.done_s, t.slot) for t in rep.tickets]
        overlap = any(a0 < b1 and b0 < a1 and sa != sb for a0, a1, sa in spans for b0, b1, sb in spans)
        assert overlap


def test_served_results_equal_oracle(env):
    """242 served requests (a Poisson stream plus the largest mesh at the finest grid and the
    smallest at the coarsest), each grid compared bit for bit with the oracle's grid of the
    same mesh and resolution; batches overlap and admissions stall on the arena."""
    import torch

    vt, batch, server, pool_dev = env
    host = mg.mesh_pool(6, seed=91, tets_lo=500, tets_hi=60000)
    sizes = [len(t) for _, t in host]
    big, small = int(np.argmax(sizes)), int(np.argmin(sizes))
    ress = (16, 32, 64, 128)
    reqs = mg.poisson_stream(240, rate_per_s=1e6, n_pool=len(pool_dev), seed=17, resolutions=ress)
    reqs.append(mg.Request(240, reqs[-1].arrival_s, big, max(ress)))
    reqs.append(mg.Request(241, reqs[-1].arrival_s, small, min(ress)))
    oracle.build()
    ref = {}
    for r in reqs:
        key = (r.mesh_id, r.res)
        if key not in ref:
            v, t = host[key[0]]
            ref[key] = torch.from_numpy(oracle.voxelize(v, t, (0, 0, 0), 1.0 / key[1], key[1]).view(np.int32)).cuda()
    seen = {}

    def check(tk, grid):
        seen[tk.rid] = bool(torch.equal(grid, ref[(tk.mesh_id, tk.res)]))

    srv = server.Server(pool_dev, arena_bytes=6 * server.grid_bytes(128), n_slots=3,
                        slot_workspace_bytes=64 << 20, max_jobs=16, on_result=check)
    try:
        rep = srv.serve(reqs, realtime=False)
    finally:
        srv.close()
    assert len(seen) == len(reqs) >= 200
    assert all(seen.values()), sorted(rid for rid, ok in seen.items() if not ok)
    assert all(t.status == vt.OK for t in rep.tickets)
    assert rep.admission_stalls > 0 and rep.batches > 10


def test_served_strict_mode_equals_alone(env):
    import torch

    vt, batch, server, pool = env
    reqs = mg.poisson_stream(20, rate_per_s=1e6, n_pool=len(pool), seed=6, resolutions=(32, 64))
    bad = []

    def check(tk, grid):
        m = pool[tk.mesh_id]
        ref = vt.voxelize(m.verts, m.tets, (0, 0, 0), 1.0 / tk.res, tk.res, mode=1)
        if not torch.equal(grid, ref):
            bad.append(tk.rid)

    srv = server.Server(pool, arena_bytes=64 << 20, n_slots=2, slot_workspace_bytes=64 << 20, max_jobs=16,
                        mode=1, on_result=check)
    try:
        srv.serve(reqs, realtime=False)
    finally:
        srv.close()
    assert not bad


def test_autotune_keeps_grid_and_caches(env, tmp_path, monkeypatch):
    import torch

    vt, batch, server, pool = env
    from paper_2106_01326_gb300 import autotune

    monkeypatch.setenv("VOXTET_TUNE_CACHE", str(tmp_path / "tune.json"))
    m = pool[int(np.argmax([p.n_tets for p in pool]))]
    res = 128
    r = autotune.tune(m.verts, m.tets, (0, 0, 0), 1.0 / res, res, spans=(64, 256), culls=(1, 2), reps=2)
    assert r["kernel"] in (1, 2) and r["span_rows"] in (0, 64, 256) and r["row_cull"] in (1, 2)
    assert len(r["table"]) == 6  # 2 span sizes x 2 culls, and slice units x 2 culls
    assert autotune.lookup(res)["span_rows"] == r["span_rows"]
    assert autotune.settings_for(res) == (r["span_rows"], r["row_cull"], r["kernel"])
    g = vt.voxelize(m.verts, m.tets, (0, 0, 0), 1.0 / res, res, span_rows=r["span_rows"], row_cull=r["row_cull"],
                    kernel=r["kernel"])
    assert torch.equal(g, vt.voxelize(m.verts, m.tets, (0, 0, 0), 1.0 / res, res))
