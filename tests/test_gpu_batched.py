"""Batched voxelization (one persistent launch over many meshes, CUDA-graph plans).

Every job's grid must equal the same job voxelized alone (and the oracle on a
sample of jobs), bit for bit, whatever the mix of sizes and resolutions, across
graph replays with different batches, and with invalid jobs in the mix.
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
    from paper_2106_01326_gb300 import batch
    from paper_2106_01326_gb300 import build as vbuild
    from paper_2106_01326_gb300 import voxtet

    vbuild.build()
    oracle.build()
    voxtet.load()
    return voxtet, batch


@pytest.fixture(scope="module")
def workload():
    return mg.batch_workload(n_meshes=40, seed=77, tets_lo=200, tets_hi=20000, resolutions=(1, 8, 32, 64, 128, 256))


def _specs(batch, vt, jobs, fill=0):
    import torch

    specs = []
    for j in jobs:
        m = batch.Mesh.from_numpy(j.verts, j.tets)
        out = vt.alloc_grid(j.res)
        out.fill_(fill)
        specs.append(batch.JobSpec(m, j.res, out, j.origin, j.voxel_size))
    return specs


def test_batched_matches_single_calls_and_oracle(env, workload):
    vt, batch = env
    specs = _specs(batch, vt, workload, fill=-1)
    st = batch.voxelize_batched(specs)
    assert st == [vt.OK] * len(specs)
    for i, (sp, j) in enumerate(zip(specs, workload)):
        ref = vt.voxelize(sp.mesh.verts, sp.mesh.tets, j.origin, j.voxel_size, j.res)
        assert bool((sp.out == ref).all()), f"job {i} res={j.res} tets={len(j.tets)}"
        if i % 7 == 0:
            o = oracle.voxelize(j.verts, j.tets, j.origin, j.voxel_size, j.res)
            assert np.array_equal(sp.out.cpu().numpy().view(np.uint32), o), f"job {i} vs oracle"


@pytest.mark.parametrize("mode", [0, 1])
def test_plan_replays_with_different_batches(env, workload, mode):
    vt, batch = env
    a = _specs(batch, vt, workload[:15])
    b = _specs(batch, vt, workload[10:40])
    need = max(batch.batch_workspace_size(a, 32), batch.batch_workspace_size(b, 32))
    plan = batch.Plan(need, 32, mode=mode)
    try:
        for specs in (a, b, a):
            for sp in specs:
                sp.out.fill_(-1)
            assert plan.run(specs) == vt.OK
            assert plan.wait() == [vt.OK] * len(specs)
            for sp in specs:
                ref = vt.voxelize(sp.mesh.verts, sp.mesh.tets, sp.origin, sp.voxel_size, sp.res, mode=mode)
                assert bool((sp.out == ref).all())
    finally:
        plan.close()


@pytest.mark.parametrize("row_cull", [1, 2])
def test_batches_with_culling_on_and_off(env, workload, row_cull):
    """A batch's jobs share one culling choice, and each choice runs a kernel with only its tile
    path compiled in: with rows outside the cross-sections skipped (1) and visited (2), every
    grid of a plan (replayed with another batch in between) and of a one-off batched call
    equals the job's single call with the same choice."""
    vt, batch = env
    jobs_a, jobs_b = workload[:12], workload[12:30]
    kinds = [_specs(batch, vt, jobs_a), _specs(batch, vt, jobs_b)]
    need = max(batch.batch_workspace_size(s, 32) for s in kinds)
    plan = batch.Plan(need, 32, row_cull=row_cull)
    try:
        for specs in (kinds[0], kinds[1], kinds[0]):
            for sp in specs:
                sp.out.fill_(-1)
            assert plan.run(specs) == vt.OK
            assert plan.wait() == [vt.OK] * len(specs)
            for sp in specs:
                ref = vt.voxelize(sp.mesh.verts, sp.mesh.tets, sp.origin, sp.voxel_size, sp.res, row_cull=row_cull)
                assert bool((sp.out == ref).all()), sp.res
    finally:
        plan.close()
    specs = _specs(batch, vt, jobs_b, fill=-1)
    assert batch.voxelize_batched(specs, row_cull=row_cull) == [vt.OK] * len(specs)
    for sp in specs:
        ref = vt.voxelize(sp.mesh.verts, sp.mesh.tets, sp.origin, sp.voxel_size, sp.res, row_cull=row_cull)
        assert bool((sp.out == ref).all()), sp.res


def test_plan_reports_workspace_overflow(env, workload):
    vt, batch = env
    specs = _specs(batch, vt, workload[:8])
    need = batch.batch_workspace_size(specs, 8)
    plan = batch.Plan(need - 4096, 8)
    try:
        assert plan.run(specs) == vt.ERR_NOMEM
    finally:
        plan.close()


def test_batched_per_job_errors(env, workload):
    import torch

    vt, batch = env
    specs = _specs(batch, vt, workload[:6])
    bad_res = batch.JobSpec(specs[0].mesh, 12, vt.alloc_grid(8))
    bad_res.out.fill_(7)
    v = workload[1].verts.copy()
    v[3, 1] = np.nan
    nan_mesh = batch.Mesh.from_numpy(v, workload[1].tets)
    bad_nan = batch.JobSpec(nan_mesh, 32, vt.alloc_grid(32))
    mixed = specs[:3] + [bad_res] + specs[3:] + [bad_nan]
    st = batch.voxelize_batched(mixed)
    assert st[3] == vt.ERR_RES
    assert st[-1] == vt.ERR_NAN
    assert [s for i, s in enumerate(st) if i not in (3, len(st) - 1)] == [vt.OK] * 6
    assert bool((bad_res.out == 7).all())  # a rejected job touches nothing
    for sp in specs:
        ref = vt.voxelize(sp.mesh.verts, sp.mesh.tets, sp.origin, sp.voxel_size, sp.res)
        assert bool((sp.out == ref).all())


def test_batched_empty_and_single(env, workload):
    vt, batch = env
    assert batch.voxelize_batched([]) == []
    specs = _specs(batch, vt, workload[:1])
    assert batch.voxelize_batched(specs) == [vt.OK]
