"""The entry point that allocates nothing, checked against the workspace entry point.

voxelize_tets_noalloc serves callers that cannot allocate device memory when they
call: a plugin inside a host application that owns the whole device-memory budget,
or a latency-critical loop that must not enter the allocator.  Its workspace is a
fixed array inside the library, so this test calls it twice in a row through the C
ABI, on different meshes, and requires each grid to equal the one voxelize_tets
produces with its own workspace (bit for bit, the tolerance of every parity test
here).  It also checks the size limit on real buffers and the status read that
works without a workspace pointer.
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
    """2^22 tetrahedra need more workspace than the 16 MiB array; the buffers are real and as
    large as the counts claim, so nothing out of bounds could be read even if the check failed."""
    import torch

    lib = vt.load()
    n_t = 1 << 22
    verts = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    tets = torch.zeros((n_t, 4), dtype=torch.int32, device="cuda")  # 64 MiB, every index 0
    out = vt.alloc_grid(8)
    org = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    o = vt.make_opts()
    assert vt.workspace_size(n_t, 1, 8) > vt.NOALLOC_SCRATCH_BYTES
    st = lib.voxelize_tets_noalloc(verts.data_ptr(), 1, tets.data_ptr(), n_t, ctypes.byref(org), 0.125, 8,
                                   out.data_ptr(), ctypes.byref(o), None)
    assert st == vt.ERR_NOMEM


def test_noalloc_status_without_sync(vt):
    """With sync = 0 the device-detected status comes from voxtet_noalloc_status_async: a bad
    vertex index is reported, and the next good call reports OK and the right grid."""
    import torch

    c = mg.single_mesh_config("plain_8")
    verts = torch.from_numpy(c["verts"]).cuda()
    tets = torch.from_numpy(c["tets"]).cuda()
    ref = vt.voxelize(verts, tets, c["origin"], c["voxel_size"], c["res"])
    word = torch.zeros(1, dtype=torch.int32).pin_memory()
    bad = tets.clone()
    bad[7, 2] = verts.shape[0]  # one past the last vertex: the kernel's index check reports it
    out = torch.empty_like(ref)
    for t, want in ((bad, vt.ERR_INDEX), (tets, vt.OK)):
        st = vt.voxelize_noalloc(verts, t, c["origin"], c["voxel_size"], c["res"], out, sync=False)
        assert st == vt.OK
        assert vt.noalloc_status_async(word) == vt.OK
        torch.cuda.current_stream().synchronize()
        assert vt.status_of_word(int(word[0])) == want
    assert torch.equal(out, ref)
