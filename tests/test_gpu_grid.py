"""GPU parity of general grids (any sides, not only cubic powers of two) and z-slabs.

Every grid is compared bit for bit with the oracle's general-grid function on the
same seeded inputs; slabs are compared with the oracle's slabs and with the whole
grid they partition.
"""
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


def _mesh_for(res3, N=6, jitter=0.3, seed=0, overhang=1.08):
    """A jittered Kuhn lattice clipped to a torus and a sphere, stretched over the grid's box
    (the lattice overhangs the box on every side; about half the samples are inside)."""
    sdf = mg.union_sdf([mg.torus_sdf(0.3, 0.12), mg.sphere_sdf((0.7, 0.3, 0.6), 0.25)])
    v, t = mg.clipped_kuhn_lattice(N, jitter, seed, sdf)
    h = 1.0 / max(res3)
    ext = np.array(res3, dtype=np.float64) * h
    v = ((v.astype(np.float64) * overhang - (overhang - 1) / 2) * ext).astype(np.float32)
    return v, t, h


def _dev(v, t):
    import torch

    return torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()


@pytest.mark.parametrize("res3", [(50, 37, 61), (100, 60, 80), (33, 1, 7), (1, 1, 1), (129, 64, 3),
                                  (300, 17, 200), (64, 64, 64), (31, 95, 2)])
@pytest.mark.parametrize("mode", [0, 1])
def test_grid_matches_oracle(vt, res3, mode):
    v, t, h = _mesh_for(res3, seed=sum(res3) + mode)
    dv, dt = _dev(v, t)
    got = vt.voxelize_grid(dv, dt, (0, 0, 0), h, res3, mode=mode).cpu().numpy().view(np.uint32)
    ref = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3, mode=mode)
    assert got.shape == ref.shape
    assert (got == ref).all()


@pytest.mark.parametrize("cull", [1, 2])
def test_grid_torus_slivers(vt, cull):
    """A clipped torus with near-flat slivers on a 200 x 150 x 100 grid (filter fallbacks included)."""
    v, t = mg.clipped_kuhn_lattice(24, 0.25, 11, mg.torus_sdf(0.3, 0.12))
    v, t, _ = mg.add_slivers(v, t, 0.05, 12, d_lattice_units=(1, 2, 3))
    res3 = (200, 150, 100)
    h = 1.0 / 200
    dv, dt = _dev(v, t)
    got = vt.voxelize_grid(dv, dt, (0, 0, 0.25), h, res3, row_cull=cull).cpu().numpy().view(np.uint32)
    ref = oracle.voxelize_grid(v, t, (0, 0, 0.25), h, res3)
    assert (got == ref).all()
    assert ref.any()


def test_cubic_grid_equals_voxelize(vt):
    import torch

    v, t, h = _mesh_for((64, 64, 64), seed=3)
    dv, dt = _dev(v, t)
    a = vt.voxelize(dv, dt, (0, 0, 0), h, 64)
    b = vt.voxelize_grid(dv, dt, (0, 0, 0), h, (64, 64, 64))
    assert torch.equal(a, b)


@pytest.mark.parametrize("res3", [(96, 40, 77), (256, 256, 256)])
def test_slabs_partition_the_grid(vt, res3):
    import torch

    v, t, h = _mesh_for(res3, N=8, seed=5)
    dv, dt = _dev(v, t)
    full = vt.voxelize_grid(dv, dt, (0, 0, 0), h, res3)
    rz = res3[2]
    cuts = [0, 3, rz // 2, rz // 2, rz - 1, rz]
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        g = vt.voxelize_grid(dv, dt, (0, 0, 0), h, res3, z_range=(a, b))
        assert g.shape[0] == b - a
        parts.append(g)
        if 0 < b - a <= 8:
            ref = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3, z0=a, z1=b)
            assert (g.cpu().numpy().view(np.uint32) == ref).all()
    assert torch.equal(torch.cat(parts, dim=0), full)


def test_longest_side_at_the_limit(vt):
    """rx = VOXTET_MAX_RES with a thin y, z: the lattice step is 2^7, words per row 256."""
    res3 = (vt.MAX_RES, 3, 2)
    v, t, h = _mesh_for(res3, N=2, seed=9)
    dv, dt = _dev(v, t)
    got = vt.voxelize_grid(dv, dt, (0, 0, 0), h, res3).cpu().numpy().view(np.uint32)
    ref = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3)
    assert (got == ref).all()


def test_grid_errors(vt):
    v, t, h = _mesh_for((8, 8, 8))
    dv, dt = _dev(v, t)
    for bad in [(0, 8, 8), (8, vt.MAX_RES + 1, 8)]:
        st, _ = vt.voxelize_grid(dv, dt, (0, 0, 0), h, bad, out=vt.alloc_grid(8), raise_on_error=False)
        assert st == vt.ERR_RES
    st, _ = vt.voxelize_grid(dv, dt, (0, 0, 0), h, (8, 8, 8), z_range=(2, 9), out=vt.alloc_grid(8),
                             raise_on_error=False)
    assert st == vt.ERR_ARG
    # an empty slab is a valid call that writes nothing
    g = vt.voxelize_grid(dv, dt, (0, 0, 0), h, (8, 8, 8), z_range=(4, 4))
    assert g.shape == (0, 8, 1)


def test_slabs_from_their_tet_subsets(vt):
    """A rank voxelizes its slab from slabs.tets_for_slab alone: the slabs still concatenate to the
    grid of the whole mesh (the subset is a superset of the tets that reach the slab)."""
    import torch

    from paper_2106_01326_gb300 import slabs

    res3 = (128, 96, 120)
    v, t, h = _mesh_for(res3, N=10, seed=13)
    dv, dt = _dev(v, t)
    full = vt.voxelize_grid(dv, dt, (0, 0, 0), h, res3)
    w = slabs.slice_weights(v, t, (0, 0, 0), h, res3[2])
    parts = []
    for z0, z1 in slabs.slab_cuts(res3[2], 5, w):
        sub = slabs.tets_for_slab(v, t, (0, 0, 0), h, z0, z1)
        assert len(sub) < len(t)
        parts.append(vt.voxelize_grid(dv, torch.from_numpy(sub).cuda(), (0, 0, 0), h, res3, z_range=(z0, z1)))
    assert torch.equal(torch.cat(parts, dim=0), full)
