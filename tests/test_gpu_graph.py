"""Single-mesh calls captured into a CUDA graph and replayed.

A call's kernels are chained on the caller's stream: each after the first is launched as a
programmatic dependent of the one before it and waits for it on the device.  A stream capture
keeps those dependencies as graph edges, so a captured call (sync = 0, workspace and grid
preallocated) must replay to the same grid as the eager call, every time, with either work
distribution of the scanline step, and leave an OK status in its workspace.
"""
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


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("name", ["torus_48", "plain_8"])
def test_captured_call_replays_to_the_eager_grid(vt, name, kernel):
    import torch

    c = mg.single_mesh_config(name)
    verts = torch.from_numpy(c["verts"]).cuda()
    tets = torch.from_numpy(c["tets"]).cuda()
    res = c["res"]
    ref = vt.voxelize(verts, tets, c["origin"], c["voxel_size"], res, kernel=kernel)
    ws = vt.alloc_workspace(len(c["tets"]), len(c["verts"]), res)
    out = vt.alloc_grid(res)
    s = torch.cuda.Stream()
    args = (verts, tets, c["origin"], c["voxel_size"], res)
    kw = dict(out=out, workspace=ws, sync=False, stream=s, kernel=kernel)
    with torch.cuda.stream(s):  # first call outside the capture (device set-up, occupancy queries)
        vt.voxelize(*args, **kw)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vt.voxelize(*args, **kw)
    for _ in range(3):
        out.fill_(-1)  # every word rewritten by the replay (the prologue clears the grid)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"{name} kernel={kernel}"
        assert vt.last_status(ws) == vt.OK


def test_captured_call_reports_a_bad_index(vt):
    """Device-detected errors of a replay land in the workspace header like an eager call's."""
    import torch

    c = mg.single_mesh_config("plain_8")
    verts = torch.from_numpy(c["verts"]).cuda()
    tets = torch.from_numpy(c["tets"]).cuda()
    res = c["res"]
    bad = tets.clone()
    ws = vt.alloc_workspace(len(c["tets"]), len(c["verts"]), res)
    out = vt.alloc_grid(res)
    s = torch.cuda.Stream()
    kw = dict(out=out, workspace=ws, sync=False, stream=s)
    with torch.cuda.stream(s):
        vt.voxelize(verts, bad, c["origin"], c["voxel_size"], res, **kw)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vt.voxelize(verts, bad, c["origin"], c["voxel_size"], res, **kw)
    g.replay()
    torch.cuda.synchronize()
    assert vt.last_status(ws) == vt.OK
    bad[5, 1] = verts.shape[0]  # one past the last vertex, in the captured buffer
    g.replay()
    torch.cuda.synchronize()
    assert vt.last_status(ws) == vt.ERR_INDEX
    bad.copy_(tets)
    g.replay()
    torch.cuda.synchronize()
    assert vt.last_status(ws) == vt.OK
    assert np.array_equal(out.cpu().numpy(), vt.voxelize(verts, tets, c["origin"], c["voxel_size"], res).cpu().numpy())
