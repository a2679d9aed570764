"""Pins of the oracle's general grids (non-cubic, any side length) and z-slabs.

A general grid res = (rx, ry, rz) keeps the cubic grid's sample rule: voxel
centres sit on lattice points (2i+1)s, with the lattice step 2s = 2^(20-K) per
voxel and K = ceil(log2(max side)).  The pins tie it to things fixed
independently of the general code path:

* the crop identity: for max side in (2^(K-1), 2^K], the general grid is exactly
  the [0:rz, 0:ry, 0:rx] block of the cubic 2^K grid with the same origin and
  voxel size (same lattice, same samples, smaller clamp), and the cubic grid is
  pinned by test_oracle_pins.py;
* closed-form counts of axis-aligned boxes on voxel boundaries, clipped to the grid;
* the pure-Python checker (a different formulation in unbounded integers);
* the unpruned all-pairs loop;
* slabs that concatenate to the whole grid.
"""
import numpy as np
import pytest

import oracle
from oracle import bigint_check as bc
from paper_2106_01326_gb300 import meshgen as mg


def _s(res3):
    return 1 << (19 - oracle.grid_exponent(res3))


def _grid_soup(rng, n_tets, res3, spread=1.0):
    """Random tets over (and a little beyond) the grid's extent, some coordinates on sample planes."""
    s = _s(res3)
    ext = np.array(res3, dtype=np.float64) * 2 * s  # x, y, z extents in lattice units
    c = rng.uniform(-0.15, 1.15, size=(n_tets, 1, 3)) * ext
    size = rng.uniform(0.05, 0.6, size=(n_tets, 1, 1)) * ext.max() * spread
    pts = c + rng.uniform(-1, 1, size=(n_tets, 4, 3)) * size
    xyz = np.clip(np.rint(pts), -(1 << 21), 1 << 21).astype(np.int64).reshape(-1, 3)
    mask = rng.random(size=xyz.shape) < 0.3
    on_plane = (np.rint(xyz / (2 * s)) * 2 + 1) * s
    xyz = np.where(mask, np.clip(on_plane, -(1 << 21), 1 << 21), xyz).astype(np.int32)
    return xyz, np.arange(4 * n_tets, dtype=np.int32).reshape(n_tets, 4)


@pytest.mark.parametrize("res3,K", [((1, 1, 1), 0), ((2, 1, 1), 1), ((3, 2, 1), 2), ((100, 60, 80), 7),
                                    ((64, 64, 64), 6), ((65, 1, 1), 7), ((8192, 5, 3), 13), ((1, 1, 1 << 19), 19)])
def test_grid_exponent(res3, K):
    assert oracle.grid_exponent(res3) == K
    assert bc.grid_exponent_py(res3) == K


@pytest.mark.parametrize("res3", [(50, 37, 61), (64, 17, 33), (5, 3, 7), (33, 64, 1), (1, 1, 1), (100, 60, 80)])
def test_grid_equals_crop_of_cubic_grid(oracle_lib, res3):
    K = oracle.grid_exponent(res3)
    R = 1 << K
    rx, ry, rz = res3
    h = 1.0 / max(res3)
    for seed in range(2):
        v, t = mg.kuhn_lattice(4, 0.3, 40 + seed)
        v = (v * np.array([rx, ry, rz], dtype=np.float32) * np.float32(h)).astype(np.float32)
        v = v * np.float32(1.1) - np.float32(0.03)  # overhang the grid on every side
        for mode in (0, 1):
            full = oracle.unpack(oracle.voxelize(v, t, (0, 0, 0), h, R, mode=mode), R)
            g = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3, mode=mode)
            assert g.shape == (rz, ry, (rx + 31) // 32)
            assert (oracle.unpack_grid(g, rx) == full[:rz, :ry, :rx]).all()
            # padding bits beyond rx stay zero
            assert (oracle.pack_grid(oracle.unpack_grid(g, rx)) == g).all()


def _box_tets(lo, hi):
    """Axis-aligned box [lo, hi] (per-axis lattice units) split into its 6 Kuhn tets."""
    ijk, tets = mg.kuhn_lattice_int(1)
    lo, hi = np.asarray(lo), np.asarray(hi)
    return (lo + ijk * (hi - lo)).astype(np.int32), tets


@pytest.mark.parametrize("res3,p,q", [((7, 5, 3), (0, 0, 0), (7, 5, 3)), ((40, 9, 17), (3, 1, 4), (31, 8, 15)),
                                      ((12, 30, 6), (-4, 10, 2), (5, 45, 9)), ((1, 1, 1), (0, 0, 0), (1, 1, 1)),
                                      ((100, 3, 70), (99, 0, 0), (100, 3, 70))])
def test_grid_box_count_closed_form(oracle_lib, res3, p, q):
    """A box on voxel boundaries [2s p_a, 2s q_a] holds the samples p_a <= i < q_a of each axis,
    clipped to the grid: the count is a product, every sample inside is set, nothing outside."""
    s = _s(res3)
    xyz, tets = _box_tets([2 * s * a for a in p], [2 * s * b for b in q])
    for mode in (0, 1):
        occ = oracle.unpack_grid(oracle.voxelize_grid_fixed(xyz, tets, res3, mode=mode), res3[0])
        lo = [max(p[a], 0) for a in range(3)]
        hi = [min(q[a], res3[a]) for a in range(3)]
        if mode == 0:
            assert occ.sum() == np.prod([max(hi[a] - lo[a], 0) for a in range(3)])
            assert occ[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].all()
        else:  # strict: no sample lies on a box face, but samples on the split's inner faces drop out
            assert occ.sum() <= np.prod([max(hi[a] - lo[a], 0) for a in range(3)])


@pytest.mark.parametrize("seed", range(6))
def test_grid_matches_python_checker(oracle_lib, seed):
    rng = np.random.default_rng(300 + seed)
    res3 = [(5, 3, 7), (9, 16, 2), (1, 1, 1), (17, 4, 3), (6, 6, 11), (3, 12, 5)][seed]
    xyz, tets = _grid_soup(rng, 10, res3)
    for mode in (0, 1):
        got = oracle.unpack_grid(oracle.voxelize_grid_fixed(xyz, tets, res3, mode=mode), res3[0])
        ref = bc.voxelize_grid_py(xyz, tets, res3, mode=mode)
        assert (got == ref).all()


@pytest.mark.parametrize("seed", range(4))
def test_grid_pruned_loop_matches_all_pairs(oracle_lib, seed):
    rng = np.random.default_rng(400 + seed)
    res3 = [(13, 7, 5), (33, 2, 9), (4, 4, 20), (31, 1, 1)][seed]
    xyz, tets = _grid_soup(rng, 20, res3)
    for mode in (0, 1):
        a = oracle.voxelize_grid_fixed(xyz, tets, res3, mode=mode)
        b = oracle.all_pairs_grid(xyz, tets, res3, mode=mode)
        assert (a == b).all()


@pytest.mark.parametrize("res3", [(48, 20, 37), (64, 64, 64)])
def test_grid_slabs_concatenate(oracle_lib, res3):
    v, t = mg.kuhn_lattice(5, 0.25, 7)
    h = 1.0 / max(res3)
    full = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3)
    rz = res3[2]
    cuts = [0, 1, rz // 3, rz // 3, rz - 2, rz]
    parts = [oracle.voxelize_grid(v, t, (0, 0, 0), h, res3, z0=a, z1=b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert parts[2].shape[0] == 0  # an empty slab is allowed
    assert (np.concatenate(parts, axis=0) == full).all()


def test_grid_snap_matches_restatement(oracle_lib):
    rng = np.random.default_rng(5)
    v = rng.uniform(-0.5, 1.5, size=(400, 3)).astype(np.float32)
    for origin, h, res3 in [((0.1, -0.2, 0.3), 0.013, (100, 60, 80)), ((0, 0, 0), 0.01, (100, 100, 100)),
                            ((-1.0, 0.5, 0.0), 0.0071, (300, 7, 129))]:
        st, xyz = oracle.snap_grid(v, origin, h, res3)
        if st != 0:
            assert st == oracle.ERR_RANGE
            continue
        assert (xyz == bc.snap_grid_py(v, origin, h, res3)).all()


def test_grid_error_codes(oracle_lib):
    xyz = np.array([[0, 0, 0], [1 << 20, 0, 0], [0, 1 << 20, 0], [0, 0, 1 << 20]], dtype=np.int32)
    t = np.array([[0, 1, 2, 3]], dtype=np.int32)
    for bad in [(0, 4, 4), (4, -1, 4), (4, 4, (1 << 19) + 1)]:
        with pytest.raises(oracle.OracleError) as e:
            oracle.voxelize_grid_fixed(xyz, t, bad)
        assert e.value.status == oracle.ERR_RES
    for z0, z1 in [(-1, 4), (3, 2), (0, 5)]:
        with pytest.raises(oracle.OracleError) as e:
            oracle.voxelize_grid_fixed(xyz, t, (4, 4, 4), z0=z0, z1=z1)
        assert e.value.status == oracle.ERR_ARG


@pytest.mark.parametrize("res3", [(50, 37, 61), (64, 64, 64), (33, 1, 7), (200, 9, 16)])
def test_brick_conversion_round_trip(oracle_lib, res3):
    """dense_to_bricks keeps every set bit, in the brick the layout names, and nothing else."""
    v, t = mg.kuhn_lattice(4, 0.3, 11)
    h = 1.0 / max(res3)
    ext = np.array(res3, dtype=np.float64) * h
    v = ((v.astype(np.float64) * 0.7 + 0.1) * ext).astype(np.float32)  # inside the grid, not filling it
    g = oracle.voxelize_grid(v, t, (0, 0, 0), h, res3)
    keys, words = oracle.dense_to_bricks(g, res3[0])
    assert (np.diff(keys.astype(np.int64)) > 0).all()
    assert words.any(axis=1).all()
    assert (oracle.bricks_to_dense(keys, words, res3) == g).all()
    occ = oracle.unpack_grid(g, res3[0])
    assert int(np.unpackbits(words.view(np.uint8)).sum()) == int(occ.sum()) > 0
    # one brick by hand: voxel (i, j, l) is bit i % 32 of word (l % 8) * 8 + j % 8 of brick (i//32, j//8, l//8)
    l, j, i = [int(x[0]) for x in np.nonzero(occ)]
    key = (i // 32) | ((j // 8) << 16) | ((l // 8) << 32)
    row = words[np.searchsorted(keys, np.uint64(key))]
    assert (int(row[(l % 8) * 8 + j % 8]) >> (i % 32)) & 1
