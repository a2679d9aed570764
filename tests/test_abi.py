"""The C-ABI library loads and exports every symbol include/voxtet.h declares.

Host-only calls (no GPU): option defaults, workspace sizing, status strings and
the argument checks that run before anything is launched.
"""
import ctypes
import os
import re

import pytest

from paper_2106_01326_gb300 import build as vbuild
from paper_2106_01326_gb300 import voxtet as vt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    vbuild.build()
    return vt.load()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", src, flags=re.M):
            if m.group(1) not in ("if", "defined"):
                names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    assert declared == set(vt.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_host_side_calls(lib):
    o = vt.Opts()
    lib.voxtet_default_opts(ctypes.byref(o))
    assert (o.mode, o.accumulate, o.use_filter, o.sync, o.span_rows, o.block, o.profile, o.row_cull,
            o.kernel) == (0, 0, 1, 1, 0, 0, 0, 0, 0)
    assert vt.workspace_size(10, 100, 64) >= 256 + 16 * 100
    assert vt.workspace_size(-1, 1, 64) == 0
    assert vt.strerror(vt.ERR_INDEX) == "tetrahedron vertex index out of range"
    assert vt.launch_count() >= 0


def test_argument_checks_before_launch(lib):
    """Invalid arguments are rejected on the host; fake non-null pointers are never touched."""
    P = 1 << 20  # a 256-aligned fake address, never dereferenced
    o = vt.make_opts()
    org = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    ws = vt.workspace_size(1, 4, 8)

    def call(res=8, h=0.125, n_t=1, n_v=4, wsb=ws, tets=P, opts=o, out=P, work=P):
        return lib.voxelize_tets(P, n_v, tets, n_t, ctypes.byref(org), h, res, out, work, wsb, ctypes.byref(opts), None)

    assert call(res=12) == vt.ERR_RES
    assert call(res=0) == vt.ERR_RES
    assert call(res=vt.MAX_RES * 2) == vt.ERR_RES
    assert call(h=0.0) == vt.ERR_ARG
    assert call(h=float("nan")) == vt.ERR_ARG
    assert call(n_t=-1) == vt.ERR_ARG
    assert call(tets=P + 4) == vt.ERR_ARG  # tets must be 16-byte aligned
    assert call(wsb=ws - 1) == vt.ERR_WORKSPACE
    assert call(work=P + 16) == vt.ERR_WORKSPACE
    assert call(out=0) == vt.ERR_ARG
    bad = vt.make_opts(mode=2)
    assert call(opts=bad) == vt.ERR_ARG
    bad = vt.make_opts(block=96)
    assert call(opts=bad) == vt.ERR_ARG
    assert lib.voxelize_tets_fixed(P, 4, P, 1, 7, P, P, ws, ctypes.byref(o), None) == vt.ERR_RES


def test_grid_argument_checks_before_launch(lib):
    """voxelize_tets_grid rejects bad sides, slabs and buffers on the host."""
    P = 1 << 20
    o = vt.make_opts()
    org = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    ws = vt.workspace_size(1, 4, 8)

    def call(res=(5, 7, 9), z0=0, z1=9, h=0.1, out=P, work=P, wsb=ws, res_ptr=True):
        r3 = (ctypes.c_int32 * 3)(*res)
        rp = ctypes.byref(r3) if res_ptr else None
        return lib.voxelize_tets_grid(P, 4, P, 1, ctypes.byref(org), h, rp, z0, z1, out, work, wsb,
                                      ctypes.byref(o), None)

    assert call(res=(0, 7, 9)) == vt.ERR_RES
    assert call(res=(5, vt.MAX_RES + 1, 9)) == vt.ERR_RES
    assert call(res=(5, 7, -3), z1=0) == vt.ERR_RES
    assert call(z0=-1) == vt.ERR_ARG
    assert call(z0=5, z1=4) == vt.ERR_ARG
    assert call(z1=10) == vt.ERR_ARG
    assert call(res_ptr=False) == vt.ERR_ARG
    assert call(out=0) == vt.ERR_ARG
    assert call(z0=3, z1=3, out=0, h=-1.0) == vt.ERR_ARG  # NULL output allowed for an empty slab only
    assert call(h=-1.0) == vt.ERR_ARG
    assert call(wsb=ws - 1) == vt.ERR_WORKSPACE


def test_sparse_host_sizing(lib):
    """Slab depth defaults and scratch sizes of the brick-sparse path (no launch)."""
    dsd = vt.default_slab_depth
    assert dsd((256, 256, 256)) == 256  # 8 MiB grid: one slab
    assert dsd((300, 100, 150)) == 152  # fits: one slab, rounded up to whole bricks
    assert dsd((4096, 4096, 4096)) == 64  # 2 MiB per slice: 128 MiB slabs
    assert dsd((8192, 8192, 8192)) == 16
    assert dsd((65536, 65536, 64)) == 8  # 512 MiB per slice: the minimum depth
    for r3 in [(1, 1, 1), (33, 17, 9), (4096, 100, 5000), (65536, 32, 40)]:
        d = dsd(r3)
        assert d % 8 == 0 and d >= 8
        per_slice = r3[1] * ((r3[0] + 31) // 32) * 4
        assert d * per_slice <= 128 << 20 or d == 8 or d >= r3[2]
    # scratch = 256 B header + the dense slab + block counts + slab marks, each 256-byte aligned
    r3 = (256, 256, 256)
    slab = 64 * 256 * 8 * 4
    assert vt.sparse_scratch_size(r3, 64) >= 256 + slab
    assert vt.sparse_scratch_size(r3, 64) % 256 == 0
    assert vt.sparse_scratch_size(r3, 128) > vt.sparse_scratch_size(r3, 64)
    assert vt.sparse_scratch_size(r3, 12) == 0  # not a multiple of 8
    assert vt.sparse_scratch_size(r3, 0) == 0
    assert vt.sparse_scratch_size((vt.SPARSE_MAX_SIDE + 1, 8, 8), 8) == 0
    assert vt.sparse_scratch_size((0, 8, 8), 8) == 0


def test_batch_workspace_sizing(lib):
    """voxtet_batch_workspace_size on jobs with fake device pointers (sizing never touches them)."""
    P = 1 << 20

    def jobs(sizes):
        arr = (vt.Job * max(len(sizes), 1))()
        for i, (nv, nt, res) in enumerate(sizes):
            j = arr[i]
            j.d_verts, j.n_verts, j.d_tets, j.n_tets = P, nv, P, nt
            j.voxel_size, j.res, j.d_out_bits = 1.0 / res, res, P
        return arr

    sizes = [(100, 400, 32), (5000, 20000, 64), (10, 10, 128)]
    a = jobs(sizes)
    n = len(sizes)
    total = lib.voxtet_batch_workspace_size(a, n, n)
    assert total > 0 and total % 256 == 0
    assert total >= sum(vt.workspace_size(nt, nv, res) for nv, nt, res in sizes)
    assert lib.voxtet_batch_workspace_size(a, n, 4 * n) > total  # the table grows with max_jobs
    assert lib.voxtet_batch_workspace_size(a, n, n - 1) == 0      # max_jobs < n_jobs
    assert lib.voxtet_batch_workspace_size(a, -1, n) == 0
    assert lib.voxtet_batch_workspace_size(None, n, n) == 0
    bigger = jobs([(100, 400, 32), (5000, 80000, 64), (10, 10, 128)])
    assert lib.voxtet_batch_workspace_size(bigger, n, n) > total
    assert lib.voxtet_batch_workspace_size(jobs([]), 0, 1) > 0  # an empty batch still has its table
