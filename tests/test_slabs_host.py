"""Host logic of the z-slab partition against the oracle (CPU): a rank that voxelizes its slab
from ``slabs.tets_for_slab`` alone gets exactly the slab of the whole mesh, and the slice weights
count the tets whose sample range covers each slice."""
import numpy as np
import pytest

import oracle
from paper_2106_01326_gb300 import meshgen as mg
from paper_2106_01326_gb300 import slabs


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _meshes():
    sdf = mg.union_sdf([mg.torus_sdf(0.3, 0.12), mg.sphere_sdf((0.7, 0.3, 0.6), 0.25)])
    v, t = mg.clipped_kuhn_lattice(7, 0.3, 21, sdf)
    yield "lattice", v, t, (0.0, 0.0, 0.0), 1.0 / 48, (48, 40, 48)
    # vertices exactly on slice sample planes and voxel boundaries, a shifted origin, h not a power of two
    rng = np.random.default_rng(22)
    h = 1.0 / 37
    origin = (0.1, -0.2, 0.05)
    n = 300
    base = rng.integers(0, 30, (n, 3)).astype(np.float64)
    pts = base[:, None, :] + rng.integers(0, 6, (n, 4, 3)) * 0.5  # multiples of half a voxel
    v = (np.asarray(origin) + pts.reshape(-1, 3) * h).astype(np.float32)
    t = np.arange(4 * n, dtype=np.int32).reshape(n, 4)
    yield "half-voxel soup", v, t, origin, h, (37, 33, 37)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_slab_from_its_tets_equals_slab_of_whole_mesh(world):
    for name, v, t, origin, h, res3 in _meshes():
        w = slabs.slice_weights(v, t, origin, h, res3[2])
        for z0, z1 in slabs.slab_cuts(res3[2], world, w):
            sub = slabs.tets_for_slab(v, t, origin, h, z0, z1)
            whole = oracle.voxelize_grid(v, t, origin, h, res3, z0, z1)
            part = oracle.voxelize_grid(v, sub, origin, h, res3, z0, z1)
            assert np.array_equal(whole, part), (name, z0, z1)
            assert len(sub) <= len(t)


def test_tets_for_slab_is_a_tight_superset():
    """The kept tets are those whose snapped z-range reaches the slab's samples, plus only tets
    within about one slice of it (the margin for the snap)."""
    sdf = mg.torus_sdf(0.3, 0.12)
    v, t = mg.clipped_kuhn_lattice(24, 0.25, 5, sdf)
    res, z0, z1 = 256, 120, 128
    sub = slabs.tets_for_slab(v, t, (0, 0, 0), 1 / res, z0, z1)
    st, xyz = oracle.snap(v, (0, 0, 0), 1 / res, res)
    assert st == 0
    z = xyz[:, 2][t].astype(np.int64)  # lattice units, 2^20 / 256 = 4096 per voxel
    unit = (1 << 20) // res

    def reaching(lo_slice, hi_slice):  # tets whose z-extent meets [lo_slice, hi_slice] in voxel units
        return set(map(tuple, t[(z.max(axis=1) >= lo_slice * unit) & (z.min(axis=1) <= (hi_slice + 1) * unit)]))

    kept = set(map(tuple, sub))
    assert reaching(z0, z1 - 1) <= kept
    assert kept <= reaching(z0 - 2, z1 + 1)


def test_slice_weights_count_covering_tets():
    v = np.array([[0.1, 0.1, 0.10], [0.9, 0.1, 0.10], [0.1, 0.9, 0.10], [0.1, 0.1, 0.55],
                  [0.1, 0.1, 0.40], [0.9, 0.1, 0.40], [0.1, 0.9, 0.40], [0.1, 0.1, 0.97]], dtype=np.float32)
    t = np.array([[0, 1, 2, 3], [4, 5, 6, 7]], dtype=np.int32)
    w = slabs.slice_weights(v, t, (0, 0, 0), 0.1, 10)  # samples at z = 0.05, 0.15, ..., 0.95
    # tet 0 covers samples 0.15 .. 0.55 (slices 1-5), tet 1 samples 0.45 .. 0.95 (slices 4-9);
    # the boundary 0.95 of a float32 0.95 would fall just below the sample, so tet 1 ends at 0.97
    expect = np.array([0, 1, 1, 1, 2, 2, 1, 1, 1, 1], dtype=np.float64)
    assert np.array_equal(w, expect)


@pytest.mark.parametrize("world", [2, 4])
def test_slab_mesh_with_compacted_vertices_equals_slab_of_whole_mesh(world):
    """slab_mesh renumbers a slab's tets onto only the vertices they name; the slab's bits do not
    change (the snap is per vertex), and no unused vertex is kept."""
    for name, v, t, origin, h, res3 in _meshes():
        w = slabs.slice_weights(v, t, origin, h, res3[2])
        for z0, z1 in slabs.slab_cuts(res3[2], world, w):
            sv, st = slabs.slab_mesh(v, t, origin, h, z0, z1)
            assert len(np.unique(st)) == len(sv) <= len(v)
            whole = oracle.voxelize_grid(v, t, origin, h, res3, z0, z1)
            part = oracle.voxelize_grid(sv, st, origin, h, res3, z0, z1)
            assert np.array_equal(whole, part), (name, z0, z1)


def test_slab_helpers_reject_what_the_whole_mesh_call_rejects():
    """A negative or too-large index, or a non-finite coordinate, raises instead of being dropped
    from (or wrapped into) a slab: the whole-mesh call reports such a mesh, so a slab must too."""
    v = np.array([[0.1, 0.1, 0.1], [0.9, 0.1, 0.1], [0.1, 0.9, 0.1], [0.1, 0.1, 0.9]], dtype=np.float32)
    good = np.array([[0, 1, 2, 3]], dtype=np.int32)
    assert len(slabs.tets_for_slab(v, good, (0, 0, 0), 0.1, 0, 10)) == 1
    for bad_t in (np.array([[0, 1, 2, -1]], dtype=np.int32), np.array([[0, 1, 2, 4]], dtype=np.int32)):
        for fn in (slabs.tets_for_slab, slabs.slab_mesh):
            with pytest.raises(ValueError):
                fn(v, bad_t, (0, 0, 0), 0.1, 0, 10)
        with pytest.raises(ValueError):
            slabs.slice_weights(v, bad_t, (0, 0, 0), 0.1, 10)
    for bad in (np.nan, np.inf):
        vb = v.copy()
        vb[3, 2] = bad
        with pytest.raises(ValueError):
            slabs.tets_for_slab(vb, good, (0, 0, 0), 0.1, 0, 10)
        with pytest.raises(ValueError):
            slabs.slab_mesh(vb, good, (0, 0, 0), 0.1, 0, 10)
