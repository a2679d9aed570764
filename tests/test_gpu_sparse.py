"""GPU parity of the brick-sparse output against the oracle's dense grid cut into bricks.

The oracle computes the dense grid (general grids share the cubic grid's lattice
rule), ``oracle.dense_to_bricks`` cuts it into 32 x 8 x 8 bricks in numpy, and the
GPU's keys and words must match bit for bit -- for cubic and general grids, several
slab depths (including ones that do not divide the grid), sides beyond the dense
limit of 8192, and a 16384^3 grid whose content lies in a corner block the oracle
can hold.
"""
import ctypes

import numpy as np
import pytest
from conftest import KERNEL_IDS, KERNELS, KernelBound

import oracle
from paper_2106_01326_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=KERNELS, ids=KERNEL_IDS)
def vt(request):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2106_01326_gb300 import build as vbuild
    from paper_2106_01326_gb300 import voxtet

    vbuild.build()
    voxtet.load()
    return KernelBound(voxtet, request.param)


def _mesh(res3, fill=(1.0, 1.0, 1.0), N=6, seed=0):
    """Torus-and-sphere-clipped lattice scaled to `fill` of the grid's box on each axis."""
    sdf = mg.union_sdf([mg.torus_sdf(0.3, 0.12), mg.sphere_sdf((0.7, 0.3, 0.6), 0.25)])
    v, t = mg.clipped_kuhn_lattice(N, 0.3, seed, sdf)
    h = 1.0 / max(res3)
    ext = np.array(res3, dtype=np.float64) * h * np.array(fill)
    return (v.astype(np.float64) * ext).astype(np.float32), t, h


def _dev(v, t):
    import torch

    return torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()


def _check(vt, v, t, h, res3, ref_res3=None, **kw):
    dv, dt = _dev(v, t)
    keys, words = vt.voxelize_sparse(dv, dt, (0, 0, 0), h, res3, **kw)
    ref = oracle.voxelize_grid(v, t, (0, 0, 0), h, ref_res3 or res3, mode=kw.get("mode", 0))
    rk, rw = oracle.dense_to_bricks(ref, (ref_res3 or res3)[0])
    k = keys.cpu().numpy().view(np.uint64)
    w = words.cpu().numpy().view(np.uint32)
    assert len(rk) > 0
    assert k.shape == rk.shape and (k == rk).all()
    assert (w == rw).all()
    return len(k)


@pytest.mark.parametrize("depth", [8, 64, 72, 256])
def test_sparse_cubic_matches_oracle(vt, depth):
    _check(vt, *_mesh((256, 256, 256)), (256, 256, 256), slab_depth=depth)


@pytest.mark.parametrize("mode", [0, 1])
def test_sparse_general_grid(vt, mode):
    _check(vt, *_mesh((300, 100, 150), seed=3), (300, 100, 150), slab_depth=48, mode=mode)


def test_sparse_side_beyond_dense_limit(vt):
    """16384 voxels along x (twice the dense limit), 32 x 40 in y, z."""
    res3 = (16384, 32, 40)
    _check(vt, *_mesh(res3, seed=5), res3, slab_depth=16)


def test_sparse_16384_cubed_corner_content(vt):
    """A 16384^3 grid (a dense one would be 512 GiB) whose mesh lies in the corner block
    16384 x 32 x 40: its bricks are those of that block (same lattice: K = 14)."""
    block = (16384, 32, 40)
    v, t, h = _mesh(block, fill=(1.0, 0.97, 0.97), seed=6)
    _check(vt, v, t, h, (16384, 16384, 16384), ref_res3=block)


def test_sparse_capacity_and_errors(vt):
    import torch

    res3 = (128, 128, 128)
    v, t, h = _mesh(res3, seed=7)
    dv, dt = _dev(v, t)
    keys, _ = vt.voxelize_sparse(dv, dt, (0, 0, 0), h, res3)
    n_true = len(keys)
    lib = vt.load()
    depth = 32
    scratch = torch.empty(vt.sparse_scratch_size(res3, depth), dtype=torch.uint8, device="cuda")
    ws = vt.alloc_workspace(len(t), len(v), 1)
    small = max(n_true // 3, 1)
    k = torch.zeros(small, dtype=torch.int64, device="cuda")
    w = torch.zeros((small, vt.BRICK_WORDS), dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    o = vt.make_opts()
    org = (ctypes.c_float * 3)(0.0, 0.0, 0.0)

    def call(r3=res3, d=depth, cap=small):
        r = (ctypes.c_int32 * 3)(*r3)
        return lib.voxelize_tets_sparse(dv.data_ptr(), len(v), dt.data_ptr(), len(t), ctypes.byref(org), h,
                                        ctypes.byref(r), d, k.data_ptr(), w.data_ptr(), cap, ctypes.byref(n),
                                        scratch.data_ptr(), scratch.numel(), ws.data_ptr(), ws.numel(),
                                        ctypes.byref(o), None)

    assert call() == vt.ERR_NOMEM and n.value == n_true
    assert (k.cpu().numpy() == keys[:small].cpu().numpy()).all()  # the first bricks are written
    assert call(d=12) == vt.ERR_ARG
    assert call(r3=(128, vt.SPARSE_MAX_SIDE + 1, 8)) == vt.ERR_RES
    assert call(d=depth * 8) == vt.ERR_WORKSPACE  # the scratch was sized for `depth`
    # no tets: no bricks
    e_keys, e_words = vt.voxelize_sparse(dv, dt[:0], (0, 0, 0), h, res3)
    assert len(e_keys) == 0 and e_words.shape == (0, vt.BRICK_WORDS)


def test_sparse_coplanar_ties_wide_grid(vt):
    """Tie-heavy soup (faces on planes through samples) in a 4096 x 256 x 64 grid through the
    sparse path (clamped filter, strided slab tiles), against the oracle's bricks."""
    import torch

    res3 = (4096, 256, 64)
    xyz, tets = mg.coplanar_face_soup(400, 4096, seed=31, spread=20, region=((0, 4096), (24, 232), (24, 40)))
    h = 1.0 / 4096
    v = (xyz.astype(np.float64) * (h / 256)).astype(np.float32)  # lattice step 2^(20-12) = 256 per voxel
    assert (v.astype(np.float64) * (256 / h) == xyz).all()  # exact round trip: the snap gives xyz back
    _check(vt, v, tets, h, res3, slab_depth=16)
    _check(vt, v, tets, h, res3, slab_depth=24, mode=1)


def test_sparse_mesh_in_a_middle_band(vt):
    """Mesh confined to z in [0.40, 0.62] of a 256^3 grid, 8-slice slabs: the slabs no tet reaches
    (including slab 0, which is voxelized anyway) hold no bricks; the rest match the oracle."""
    v, t, h = _mesh((256, 256, 256), seed=11)
    v = v.astype(np.float64)
    v[:, 2] = 0.40 + 0.22 * v[:, 2]
    v = v.astype(np.float32)
    n = _check(vt, v, t, h, (256, 256, 256), slab_depth=8)
    dv, dt = _dev(v, t)
    keys, _ = vt.voxelize_sparse(dv, dt, (0, 0, 0), h, (256, 256, 256), slab_depth=8)
    bz = keys.cpu().numpy().view(np.uint64) >> np.uint64(32)
    assert len(keys) == n and bz.min() >= 12 and bz.max() <= 20  # z in [0.40, 0.62] x 32 bricks


def test_sparse_bad_index_reported_when_low_slabs_are_empty(vt):
    """All tets high in z, one with a vertex index out of range: the error is still reported
    (slab 0 is always voxelized and reports it)."""
    v, t, h = _mesh((128, 128, 128), seed=12)
    v = v.astype(np.float64)
    v[:, 2] = 0.7 + 0.25 * v[:, 2]
    v = v.astype(np.float32)
    t = t.copy()
    t[len(t) // 2, 1] = len(v) + 5
    dv, dt = _dev(v, t)
    with pytest.raises(vt.VoxtetError) as e:
        vt.voxelize_sparse(dv, dt, (0, 0, 0), h, (128, 128, 128), slab_depth=16)
    assert e.value.status == vt.ERR_INDEX


def test_sparse_dirty_scratch_and_reuse(vt):
    """A scratch full of set bits gives the same bricks (the first slab is cleared; later slabs
    rely on the previous slab's compaction having cleared every brick it held), and so does a
    second call on the same scratch; ragged grid (ry, rz not multiples of 8 or of the depth)."""
    import torch

    res3 = (200, 100, 150)
    v, t, h = _mesh(res3, seed=13)
    dv, dt = _dev(v, t)
    depth = 24
    scratch = torch.full((vt.sparse_scratch_size(res3, depth),), 255, dtype=torch.uint8, device="cuda")
    ref = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3)
    rk, rw = oracle.dense_to_bricks(ref, res3[0])
    for _ in range(2):
        keys, words = vt.voxelize_sparse(dv, dt, (0, 0, 0), h, res3, slab_depth=depth, scratch=scratch)
        assert (keys.cpu().numpy().view(np.uint64) == rk).all()
        assert (words.cpu().numpy().view(np.uint32) == rw).all()
