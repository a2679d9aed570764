"""The entry point that allocates nothing, checked against the workspace entry point.

voxelize_tets_noalloc serves callers that cannot allocate device memory when they
call (for example during a stream capture, or inside a host application that owns
the device-memory budget).  Its workspace is a fixed array inside the library, so
this test calls it twice in a row through the C ABI, on different meshes, and
requires each grid to equal the one voxelize_tets produces with its own
workspace (bit for bit, the tolerance of every parity test here).
"""
import ctypes

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


def test_noalloc_matches_workspace_entry_point_on_two_calls(vt):
    import torch

    for name in ("torus_48", "plain_8"):  # the larger mesh first, so stale scratch would show
        c = mg.single_mesh_config(name)
        verts = torch.from_numpy(c["verts"]).cuda()
        tets = torch.from_numpy(c["tets"]).cuda()
        ref = vt.voxelize(verts, tets, c["origin"], c["voxel_size"], c["res"])
        out = torch.full_like(ref, -1)
        st = vt.voxelize_noalloc(verts, tets, c["origin"], c["voxel_size"], c["res"], out)
        assert st == vt.OK, vt.strerror(st)
        assert torch.equal(out, ref), name


def test_noalloc_rejects_meshes_beyond_the_scratch(vt):
    import torch

    lib = vt.load()
    verts = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    tets = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    out = vt.alloc_grid(8)
    org = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    o = vt.make_opts()
    big = 1 << 26  # needs far more workspace than the fixed scratch holds; nothing is read
    assert vt.workspace_size(big, 4, 8) > vt.NOALLOC_SCRATCH_BYTES
    st = lib.voxelize_tets_noalloc(verts.data_ptr(), 4, tets.data_ptr(), big, ctypes.byref(org), 0.125, 8,
                                   out.data_ptr(), ctypes.byref(o), None)
    assert st == vt.ERR_NOMEM
