"""The pipelined host API: a stream of host meshes gives, job by job, the grid each mesh
gets from a single call, and a device-detected error in one job is reported for it."""
import numpy as np
import pytest

from paper_2106_01326_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vt():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2106_01326_gb300 import build as vbuild
    from paper_2106_01326_gb300 import voxtet

    vbuild.build()
    voxtet.load()
    return voxtet


def test_pipeline_equals_single_calls(vt):
    import torch

    from paper_2106_01326_gb300 import pipeline

    res = 128
    meshes = [mg.clipped_mesh(n, seed=40 + i) for i, n in enumerate([3000, 20000, 500, 12000, 7000, 20000, 900])]
    max_v = max(len(v) for v, _ in meshes)
    max_t = max(len(t) for _, t in meshes)
    pipe = pipeline.HostPipeline(max_v, max_t, res, depth=2)
    hosts = []
    for v, t in meshes:
        hv, ht = torch.from_numpy(v).pin_memory(), torch.from_numpy(t).pin_memory()
        hg = torch.empty((res, res, res // 32), dtype=torch.int32).pin_memory()
        hosts.append((hv, ht, hg))
        pipe.submit(hv, ht, hg, (0, 0, 0), 1.0 / res)
    assert pipe.wait() == [vt.OK] * len(meshes)
    for (v, t), (_, _, hg) in zip(meshes, hosts):
        ref = vt.voxelize(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), (0, 0, 0), 1.0 / res, res)
        assert torch.equal(hg, ref.cpu())
        assert hg.any()


def test_pipeline_reports_the_failing_job(vt):
    import torch

    from paper_2106_01326_gb300 import pipeline

    res = 64
    v, t = mg.clipped_mesh(2000, seed=9)
    bad = t.copy()
    bad[5, 2] = len(v) + 3  # a vertex index out of range
    pipe = pipeline.HostPipeline(len(v), len(t), res, depth=3)
    hv = torch.from_numpy(v).pin_memory()
    grids = [torch.empty((res, res, 2), dtype=torch.int32).pin_memory() for _ in range(4)]
    for k, tt in enumerate([t, t, bad, t]):
        pipe.submit(hv, torch.from_numpy(tt).pin_memory(), grids[k], (0, 0, 0), 1.0 / res)
    with pytest.raises(vt.VoxtetError) as e:
        pipe.wait()
    assert e.value.status == vt.ERR_INDEX and "job 2" in str(e.value)
    assert torch.equal(grids[0], grids[1]) and torch.equal(grids[0], grids[3])
    with pytest.raises(ValueError):
        pipe.submit(hv, torch.from_numpy(np.concatenate([t, t])).pin_memory(), grids[0], (0, 0, 0), 1.0 / res)
