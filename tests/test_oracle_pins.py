"""Pins for the CPU oracle: things the paper and the mathematics fix.

None of these re-types the oracle's formula: they check it against closed
forms (Theorem 1's determinants for the corner simplex, lattice-aligned cube and
Kuhn-tet sample counts), an independent Python formulation, all-pairs brute
force, hand-derived fixtures, grid invariants and the volume bound.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import bigint_check as bc
from paper_2106_01326_gb300 import meshgen as mg

L = 1 << 20
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def s_of(res):
    return 1 << (19 - (res.bit_length() - 1))


# ------------------------------------------------------------- Theorem 1 determinants

@pytest.mark.parametrize("Lc,p,q,r", [(8, 1, 2, 3), (10, 0, 0, 0), (7, 7, 0, 0), (9, 3, 3, 3), (5, -2, 1, 9),
                                      (1 << 21, 12345, -777, 1 << 19)])
def test_theorem1_dets_corner_closed_form(oracle_lib, Lc, p, q, r):
    """For A=0, B=L e_x, C=L e_y, D=L e_z and P=(p,q,r): D_a = L^2 (L-p-q-r), D_b = -L^2 p,
    D_c = L^2 q, D_d = -L^2 r (each is L^3 times a signed barycentric coordinate)."""
    A, B, C, D = (0, 0, 0), (Lc, 0, 0), (0, Lc, 0), (0, 0, Lc)
    Da, Db, Dc, Dd = oracle.theorem1_dets(A, B, C, D, (p, q, r))
    assert Da == Lc * Lc * (Lc - p - q - r)
    assert Db == -Lc * Lc * p
    assert Dc == Lc * Lc * q
    assert Dd == -Lc * Lc * r


def test_theorem1_dets_identities(oracle_lib):
    """Random points: D_a - D_b + D_c - D_d equals det(AB, AC, AD) (the four sub-volumes
    partition the tet), the determinants vanish at a vertex as expected, and they are
    translation invariant (Section 4, Lemma 1.1 / 2.1 sign structure)."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        pts = rng.integers(-(1 << 21), (1 << 21) + 1, size=(5, 3))
        A, B, C, D, P = [tuple(int(v) for v in x) for x in pts]
        Da, Db, Dc, Dd = oracle.theorem1_dets(A, B, C, D, P)
        v6 = bc.orient(A, B, C, D)
        assert Da - Db + Dc - Dd == v6
        # at P = A the vectors a = 0, so D_b = D_c = D_d = 0 and D_a = det(AB, AC, AD)
        assert oracle.theorem1_dets(A, B, C, D, A) == (v6, 0, 0, 0)
        t = rng.integers(-1000, 1000, size=3)
        sh = [tuple(int(v) for v in (np.array(x) + t)) for x in (A, B, C, D, P)]
        assert oracle.theorem1_dets(*sh) == (Da, Db, Dc, Dd)
        # Lemma 1.1: swapping two vertices flips the signed volume's sign
        assert bc.orient(A, C, B, D) == -v6


# ------------------------------------------------------------- hand-derived fixtures

def _read_fixture():
    cases = {}
    cur = None
    with open(os.path.join(GOLDEN, "corner_tets_res4.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].isalpha():
                cur = (parts[0], int(parts[1]))
                cases[cur] = (int(parts[2]), [])
            else:
                cases[cur][1].append(tuple(int(x) for x in parts))
    return cases


def test_golden_corner_tets(oracle_lib):
    shapes = {"corner": [(0, 0, 0), (L, 0, 0), (0, L, 0), (0, 0, L)],
              "kuhn": [(0, 0, 0), (L, 0, 0), (L, L, 0), (L, L, L)]}
    cases = _read_fixture()
    assert len(cases) == 4
    for (name, mode), (count, triples) in cases.items():
        assert len(triples) == count
        xyz = np.array(shapes[name], dtype=np.int32)
        g = oracle.voxelize_fixed(xyz, np.array([[0, 1, 2, 3]], dtype=np.int32), 4, mode=mode)
        occ = oracle.unpack(g, 4)
        got = sorted((i, j, l) for l, j, i in zip(*np.nonzero(occ)))
        assert got == sorted(triples), (name, mode)


# ------------------------------------------------------------- closed-form counts

def _cube_tets(lo, hi):
    """Aligned cube [lo, hi]^3 (lattice units) split into its 6 Kuhn tets."""
    ijk, tets = mg.kuhn_lattice_int(1)
    xyz = (lo + ijk * (hi - lo)).astype(np.int32)
    return xyz, tets


@pytest.mark.parametrize("res,p,q", [(8, 0, 8), (16, 3, 11), (32, 5, 6), (64, 17, 49), (2, 0, 2), (1, 0, 1)])
def test_cube_count_closed_form(oracle_lib, res, p, q):
    """Cube on voxel boundaries [2sp, 2sq]^3: exactly (q-p)^3 samples, all of them once."""
    s = s_of(res)
    xyz, tets = _cube_tets(2 * s * p, 2 * s * q)
    g = oracle.voxelize_fixed(xyz, tets, res)
    occ = oracle.unpack(g, res)
    assert occ.sum() == (q - p) ** 3
    assert occ[p:q, p:q, p:q].all()


@pytest.mark.parametrize("res,p,q", [(8, 0, 8), (16, 2, 13), (32, 9, 10), (64, 0, 64)])
def test_kuhn_tet_counts_closed_form(oracle_lib, res, p, q):
    """Each single Kuhn tet of an aligned cube with n samples per axis holds C(n+2, 3)
    samples (the closed reading counts the shared diagonal faces), so the six counts
    sum to n(n+1)(n+2), and the union is the n^3 cube."""
    n = q - p
    s = s_of(res)
    xyz, tets = _cube_tets(2 * s * p, 2 * s * q)
    total = 0
    for t in range(6):
        g, st = oracle.voxelize_fixed(xyz, tets[t:t + 1], res, with_stats=True)
        occ = oracle.unpack(g, res)
        assert occ.sum() == math.comb(n + 2, 3)
        # x-rows (j, l) holding a sample: the (y, z) order the tet fixes (j >= l or l >= j), with a
        # sample i always available between them, so n(n+1)/2 whichever slot x takes in the order
        assert st["rows_with_samples"] == n * (n + 1) // 2
        total += int(occ.sum())
    assert total == n * (n + 1) * (n + 2)
    _, st = oracle.voxelize_fixed(xyz, tets, res, with_stats=True)
    assert st["rows_with_samples"] == 3 * n * (n + 1)


def test_plain_lattice_fills_grid(oracle_lib):
    """The unjittered 8^3 Kuhn lattice over the whole grid sets every one of the 64^3 bits."""
    ijk, tets = mg.kuhn_lattice_int(8)
    xyz = (ijk * (L // 8)).astype(np.int32)
    g, st = oracle.voxelize_fixed(xyz, tets, 64, with_stats=True)
    assert st["set"] == 64 ** 3
    assert (g == 0xFFFFFFFF).all()


def test_strict_mode_leaves_diagonal_holes(oracle_lib):
    """The paper's strict test loses samples on faces shared by two tets; the closed
    reading does not.  On the unjittered lattice every sample with i == j inside a cell
    lies on a shared Kuhn face."""
    ijk, tets = mg.kuhn_lattice_int(4)
    xyz = (ijk * (L // 4)).astype(np.int32)
    closed = oracle.unpack(oracle.voxelize_fixed(xyz, tets, 16, mode=0), 16)
    strict = oracle.unpack(oracle.voxelize_fixed(xyz, tets, 16, mode=1), 16)
    assert closed.all()
    assert not strict.all()
    assert (strict <= closed).all()


def test_degenerate_tet_marks_nothing(oracle_lib):
    flat = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0], [L // 2, L // 2, 0]], dtype=np.int32)
    g = oracle.voxelize_fixed(flat, np.array([[0, 1, 2, 3]], dtype=np.int32), 8)
    assert not g.any()
    # collinear and coincident vertices too
    line = np.array([[0, 0, 0], [L, L, L], [L // 2, L // 2, L // 2], [L // 4, L // 4, L // 4]], dtype=np.int32)
    assert not oracle.voxelize_fixed(line, np.array([[0, 1, 2, 3]], dtype=np.int32), 8).any()


# ------------------------------------------------------------- independent formulations

def _random_soup(rng, n_tets, res, spread=1.3):
    s = s_of(res)
    n_v = 4 * n_tets
    c = rng.uniform(-0.15, 1.15, size=(n_tets, 1, 3)) * L
    size = rng.uniform(0.05, 0.6, size=(n_tets, 1, 1)) * L * spread
    pts = c + rng.uniform(-1, 1, size=(n_tets, 4, 3)) * size
    xyz = np.clip(np.rint(pts), -(1 << 21), 1 << 21).astype(np.int32).reshape(n_v, 3)
    # snap a few coordinates onto sample planes to provoke ties
    mask = rng.random(size=xyz.shape) < 0.3
    on_plane = ((np.rint(xyz / (2 * s)) * 2 + 1) * s).astype(np.int64)
    xyz = np.where(mask, np.clip(on_plane, -(1 << 21), 1 << 21), xyz).astype(np.int32)
    tets = np.arange(n_v, dtype=np.int32).reshape(n_tets, 4)
    return xyz, tets


@pytest.mark.parametrize("seed", range(6))
def test_c_oracle_matches_python_checker(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    res = [4, 8, 16][seed % 3]
    xyz, tets = _random_soup(rng, 12, res)
    for mode in (0, 1):
        got = oracle.unpack(oracle.voxelize_fixed(xyz, tets, res, mode=mode), res)
        ref = bc.voxelize_py(xyz, tets, res, mode=mode)
        assert (got == ref).all()


@pytest.mark.parametrize("seed", range(4))
def test_c_oracle_matches_python_checker_jittered_lattice(oracle_lib, seed):
    v, t = mg.kuhn_lattice(3, 0.3, seed)
    res = 16
    st, xyz = oracle.snap(v, (0, 0, 0), 1.0 / res, res)
    assert st == 0
    got = oracle.unpack(oracle.voxelize_fixed(xyz, t, res), res)
    ref = bc.voxelize_py(xyz, t, res)
    assert (got == ref).all()
    assert got.all()  # a conforming lattice over the cube covers every sample


@pytest.mark.parametrize("seed", range(5))
def test_pruned_loop_matches_all_pairs(oracle_lib, seed):
    rng = np.random.default_rng(200 + seed)
    res = [2, 8, 16, 32, 1][seed]
    xyz, tets = _random_soup(rng, 25, res)
    for mode in (0, 1):
        a = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
        b = oracle.all_pairs(xyz, tets, res, mode=mode)
        assert (a == b).all()


def test_slab_matches_full_grid(oracle_lib):
    v, t = mg.kuhn_lattice(5, 0.25, 3)
    st, xyz = oracle.snap(v, (0, 0, 0), 1 / 32, 32)
    full = oracle.voxelize_fixed(xyz, t, 32)
    for z0, z1 in [(0, 32), (3, 9), (31, 32), (7, 7)]:
        assert (oracle.voxelize_fixed_slab(xyz, t, 32, z0, z1) == full[z0:z1]).all()


def test_thread_count_does_not_change_grid(oracle_lib):
    v, t = mg.kuhn_lattice(6, 0.25, 9)
    st, xyz = oracle.snap(v, (0, 0, 0), 1 / 64, 64)
    g1 = oracle.voxelize_fixed(xyz, t, 64, n_threads=1)
    g4 = oracle.voxelize_fixed(xyz, t, 64, n_threads=4)
    assert (g1 == g4).all()


def test_thread_count_of_one_call_does_not_leak(oracle_lib):
    """A call with n_threads = 1 must not lower the team of later default calls (the
    oracle and the paper's CPU method time themselves on all cores by default)."""
    v, t = mg.kuhn_lattice(6, 0.25, 9)
    st, xyz = oracle.snap(v, (0, 0, 0), 1 / 64, 64)
    default = oracle.num_threads()
    oracle.voxelize_fixed(xyz, t, 64, n_threads=1)
    assert oracle.last_threads() == 1
    assert oracle.num_threads() == default
    oracle.voxelize_fixed(xyz, t, 64)
    assert oracle.last_threads() == default
    oracle.paper_cpu(xyz, t, 64, "float", n_threads=1)
    assert oracle.last_threads() == 1
    oracle.paper_cpu(xyz, t, 64, "double")
    assert oracle.last_threads() == default
    oracle.voxelize_fixed_slab(xyz, t, 64, 10, 20, n_threads=2)
    assert oracle.last_threads() == 2
    assert oracle.num_threads() == default


# ------------------------------------------------------------- invariants

def _jittered(N=4, res=32, seed=0, jitter=0.3):
    v, t = mg.kuhn_lattice(N, jitter, seed)
    st, xyz = oracle.snap(v * 0.75 + 0.1, (0, 0, 0), 1.0 / res, res)
    assert st == 0
    return xyz, t


def test_invariant_translation_by_whole_voxels(oracle_lib):
    res = 32
    xyz, t = _jittered(res=res)
    base = oracle.unpack(oracle.voxelize_fixed(xyz, t, res), res)
    unit = 2 * s_of(res)
    for d in [(1, 0, 0), (0, 2, 0), (0, 0, -3), (2, -1, 1)]:
        moved = oracle.unpack(oracle.voxelize_fixed(xyz + np.array(d) * unit, t, res), res)
        dx, dy, dz = d
        exp = np.roll(base, shift=(dz, dy, dx), axis=(0, 1, 2))
        # nothing wraps: the mesh stays well inside the grid
        assert (moved == exp).all()


def test_invariant_axis_permutation_and_mirror(oracle_lib):
    res = 16
    xyz, t = _jittered(res=res, seed=4)
    base = oracle.unpack(oracle.voxelize_fixed(xyz, t, res), res)  # [z, y, x]
    for perm in itertools.permutations(range(3)):
        p = oracle.unpack(oracle.voxelize_fixed(xyz[:, list(perm)], t, res), res)
        # new axis a takes old axis perm[a]; arrays are indexed (z, y, x) = (2, 1, 0)
        exp = np.transpose(base, axes=[2 - perm[2], 2 - perm[1], 2 - perm[0]])
        assert (p == exp).all(), perm
    mir = xyz.copy()
    mir[:, 0] = L - mir[:, 0]
    m = oracle.unpack(oracle.voxelize_fixed(mir, t, res), res)
    assert (m == base[:, :, ::-1]).all()


def test_invariant_vertex_order_shuffle_duplicates(oracle_lib):
    res = 16
    xyz, t = _jittered(N=3, res=res, seed=7)
    base = oracle.voxelize_fixed(xyz, t, res)
    for perm in itertools.permutations(range(4)):
        assert (oracle.voxelize_fixed(xyz, t[:, list(perm)], res) == base).all()
    rng = np.random.default_rng(1)
    shuf = t[rng.permutation(len(t))]
    assert (oracle.voxelize_fixed(xyz, shuf, res) == base).all()
    dup = np.concatenate([t, t[: len(t) // 2]])
    assert (oracle.voxelize_fixed(xyz, dup, res) == base).all()


def test_volume_bound_conforming_mesh(oracle_lib):
    """For a conforming mesh the set-bit count differs from the enclosed volume (in voxels)
    by at most the number of voxels the boundary surface can touch."""
    res = 64
    v, t = mg.kuhn_lattice(10, 0.25, 11)
    v, t = mg.clip_by_centroid(v, t, mg.sphere_sdf((0.5, 0.5, 0.5), 0.35))
    st, xyz = oracle.snap(v, (0, 0, 0), 1 / res, res)
    g, stats = oracle.voxelize_fixed(xyz, t, res, with_stats=True)
    X = xyz.astype(np.int64)
    vol6 = 0
    for a, b, c, d in t:
        vol6 += abs(bc.orient(X[a], X[b], X[c], X[d]))
    unit = 2 * s_of(res)
    volume = Fraction(vol6, 6 * unit ** 3)
    # boundary area in voxel units: faces used by exactly one tet
    faces = {}
    for tet in t:
        for f in itertools.combinations(sorted(int(x) for x in tet), 3):
            faces[f] = faces.get(f, 0) + 1
    area = 0.0
    for f, cnt in faces.items():
        if cnt == 1:
            p0, p1, p2 = (X[i].astype(np.float64) / unit for i in f)
            area += 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0))
    bound = 2 * (math.sqrt(3) / 2) * area + 8
    assert abs(stats["set"] - float(volume)) <= bound
    assert stats["set"] > 0.5 * float(volume)


# ------------------------------------------------------------- snapping and errors

def test_snap_unit_grid_is_exact_rounding(oracle_lib):
    """origin 0 and voxel size 1/res make the snap X = round_half_even(v * 2^20) exactly."""
    rng = np.random.default_rng(3)
    v = rng.uniform(-0.9, 1.9, size=(2000, 3)).astype(np.float32)
    v[:10] = np.float32(0.5) + np.float32(2.0 ** -21)  # exact ties at the lattice half-step
    for res in (1, 64, 512, 1 << 19):
        st, xyz = oracle.snap(v, (0, 0, 0), 1.0 / res, res)
        assert st == 0
        exp = [[round(Fraction(float(x)) * L) for x in row] for row in v]  # Fraction rounds half to even
        assert (xyz == np.array(exp)).all()


def test_snap_matches_double_restatement(oracle_lib):
    rng = np.random.default_rng(4)
    v = rng.uniform(-1.0, 2.0, size=(500, 3)).astype(np.float32)
    for origin, h, res in [((0.1, -0.2, 0.3), 0.013, 64), ((-1.0, 0.5, 0.0), 0.0071, 256), ((0, 0, 0), 0.3, 8)]:
        st, xyz = oracle.snap(v, origin, h, res)
        if st != 0:
            assert st == oracle.ERR_RANGE
            continue
        assert (xyz == bc.snap_py(v, origin, h, res)).all()


def test_error_codes(oracle_lib):
    xyz = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0], [0, 0, L]], dtype=np.int32)
    t = np.array([[0, 1, 2, 3]], dtype=np.int32)
    assert oracle.voxelize_fixed(xyz, t, 12, raise_on_error=False)[0] == oracle.ERR_RES
    assert oracle.voxelize_fixed(xyz, t, 0, raise_on_error=False)[0] == oracle.ERR_RES
    assert oracle.voxelize_fixed(xyz, np.array([[0, 1, 2, 4]], np.int32), 8, raise_on_error=False)[0] == oracle.ERR_INDEX
    assert oracle.voxelize_fixed(xyz, np.array([[0, -1, 2, 3]], np.int32), 8, raise_on_error=False)[0] == oracle.ERR_INDEX
    big = xyz.copy()
    big[1, 0] = (1 << 21) + 1
    assert oracle.voxelize_fixed(big, t, 8, raise_on_error=False)[0] == oracle.ERR_RANGE
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float32)
    bad = v.copy()
    bad[2, 1] = np.nan
    assert oracle.voxelize(bad, t, (0, 0, 0), 0.25, 4, raise_on_error=False)[0] == oracle.ERR_NAN
    far = v.copy()
    far[3, 2] = 3.0
    assert oracle.voxelize(far, t, (0, 0, 0), 0.25, 4, raise_on_error=False)[0] == oracle.ERR_RANGE
    assert oracle.voxelize(v, t, (0, 0, 0), 0.0, 4, raise_on_error=False)[0] == oracle.ERR_ARG
    # empty mesh: a zero grid
    g = oracle.voxelize_fixed(xyz, np.zeros((0, 4), np.int32), 8)
    assert not g.any()
