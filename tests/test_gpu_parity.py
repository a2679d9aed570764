"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Small and medium cases are compared element by element over the whole grid, and
so is the benchmark's workload (the 1.3M-tet sliver mesh at 512^3) in every
launch shape the autotuner can pick; the 1024^3 and larger grids are compared
on sampled z-slabs the oracle computes directly.
"""
import numpy as np
import pytest
from conftest import KERNEL_IDS, KERNELS, KernelBound

import oracle
from paper_2106_01326_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

L = 1 << 20


@pytest.fixture(scope="module", params=KERNELS, ids=KERNEL_IDS)
def vt(request):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2106_01326_gb300 import build as vbuild
    from paper_2106_01326_gb300 import voxtet

    vbuild.build()
    oracle.build()
    voxtet.load()
    return KernelBound(voxtet, request.param)


def _dev(a, dtype):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def gpu_fixed(vt, xyz, tets, res, **kw):
    import torch

    g = vt.voxelize_fixed(_dev(xyz, torch.int32), _dev(tets.reshape(-1, 4), torch.int32), res, **kw)
    return g.cpu().numpy().view(np.uint32)


def gpu_world(vt, verts, tets, origin, h, res, **kw):
    import torch

    g = vt.voxelize(_dev(verts, torch.float32), _dev(tets.reshape(-1, 4), torch.int32), origin, h, res, **kw)
    return g.cpu().numpy().view(np.uint32)


def assert_same(got, ref, res, what=""):
    got = np.asarray(got).view(np.uint32).reshape(ref.shape)
    if np.array_equal(got, ref):
        return
    a, b = oracle.unpack(got, res), oracle.unpack(ref, ref.shape[1])
    bad = np.argwhere(a != b)
    l, j, i = bad[0]
    raise AssertionError(f"{what}: {len(bad)} samples differ; first (i={i}, j={j}, l={l}): gpu={a[l, j, i]} "
                         f"oracle={b[l, j, i]}")


def s_of(res):
    return 1 << (19 - (res.bit_length() - 1))


def random_soup(rng, n_tets, res, spread=1.0, tie_frac=0.3, lo=-0.15, hi=1.15):
    s = s_of(res)
    c = rng.uniform(lo, hi, size=(n_tets, 1, 3)) * L
    size = rng.uniform(0.02, 0.5, size=(n_tets, 1, 1)) * L * spread
    pts = c + rng.uniform(-1, 1, size=(n_tets, 4, 3)) * size
    xyz = np.clip(np.rint(pts), -(1 << 21), 1 << 21).astype(np.int64).reshape(-1, 3)
    mask = rng.random(size=xyz.shape) < tie_frac
    on_plane = (np.rint(xyz / (2 * s)) * 2 + 1) * s
    xyz = np.where(mask, np.clip(on_plane, -(1 << 21), 1 << 21), xyz).astype(np.int32)
    tets = np.arange(len(xyz), dtype=np.int32).reshape(n_tets, 4)
    return xyz, tets


# ------------------------------------------------------------------ small, whole grid

@pytest.mark.parametrize("use_filter", [True, False])
@pytest.mark.parametrize("span_rows", [1, 16, 4096])
def test_plain_lattice_world_coords(vt, use_filter, span_rows):
    c = mg.single_mesh_config("plain_8")
    ref = oracle.voxelize(c["verts"], c["tets"], c["origin"], c["voxel_size"], c["res"])
    got = gpu_world(vt, c["verts"], c["tets"], c["origin"], c["voxel_size"], c["res"], use_filter=use_filter,
                    span_rows=span_rows)
    assert_same(got, ref, c["res"], "plain_8")


@pytest.mark.parametrize("seed", range(12))
def test_random_soup_all_modes(vt, seed):
    rng = np.random.default_rng(1000 + seed)
    res = [1, 2, 4, 8, 16, 32, 64, 128, 256, 32, 64, 16][seed]
    xyz, tets = random_soup(rng, 60 + 20 * seed, res)
    for mode in (0, 1):
        ref = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
        for use_filter in (True, False):
            got = gpu_fixed(vt, xyz, tets, res, mode=mode, use_filter=use_filter, span_rows=1 + seed % 5)
            assert_same(got, ref, res, f"soup seed={seed} res={res} mode={mode} filter={use_filter}")


@pytest.mark.parametrize("res", [16, 64, 128])
def test_unjittered_lattice_ties(vt, res):
    """Every shared Kuhn face passes through samples; many faces are parallel to x."""
    for N, off in [(4, 0), (8, 3 * s_of(res)), (5, 2 * s_of(res))]:
        ijk, tets = mg.kuhn_lattice_int(N)
        xyz = (ijk * (L // N) + off).astype(np.int32)
        for mode in (0, 1):
            ref = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
            got = gpu_fixed(vt, xyz, tets, res, mode=mode)
            assert_same(got, ref, res, f"lattice N={N} off={off} mode={mode}")


@pytest.mark.parametrize("res,spread,n", [(64, 60, 400), (256, 30, 2000), (256, 200, 150), (1024, 400, 40)])
def test_coplanar_face_ties(vt, res, spread, n):
    """Faces on planes through many samples, vertices at unaligned lattice points: exact zeros
    that only appear after cancellation (float and double both get some of these wrong)."""
    xyz, tets = mg.coplanar_face_soup(n, res, seed=res + spread, spread=spread)
    for mode in (0, 1):
        ref = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
        for use_filter in (True, False):
            got = gpu_fixed(vt, xyz, tets, res, mode=mode, use_filter=use_filter)
            assert (got == ref).all(), (mode, use_filter)


@pytest.mark.parametrize("mode", [0, 1])
def test_filter_defers_ties_and_never_certifies_a_wrong_row(vt, mode):
    """The single-precision filter on inputs built to defeat it (faces through many samples,
    vertices at unaligned lattice points).  It must hand rows it cannot decide to the exact
    kernels (fallback rows counted) and every row it certifies must agree with exact
    arithmetic: the grid equals the exact-only grid and the oracle's."""
    import torch

    res = 256
    xyz, tets = mg.coplanar_face_soup(2000, res, seed=4242 + mode, spread=30)
    ref = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
    ws = vt.alloc_workspace(len(tets), len(xyz), res)
    d_xyz, d_tets = _dev(xyz, torch.int32), _dev(tets.reshape(-1, 4), torch.int32)
    got = vt.voxelize_fixed(d_xyz, d_tets, res, workspace=ws, mode=mode).cpu().numpy().view(np.uint32)
    st = vt.read_stats(ws)
    exact_only = vt.voxelize_fixed(d_xyz, d_tets, res, mode=mode, use_filter=False).cpu().numpy().view(np.uint32)
    assert st["rows"] > 0 and 0 < st["fallback_rows"] < st["rows"], st
    assert_same(got, ref, res, f"filter mode={mode}")
    assert np.array_equal(got, exact_only)


@pytest.mark.parametrize("mode", [0, 1])
def test_coplanar_face_ties_clamped_filter(vt, mode):
    """2048^3: the filter clamps each face's bracket to where the face can change a row; ties
    placed on planes through samples must still come out exact at the clamp boundaries."""
    res = 2048
    xyz, tets = mg.coplanar_face_soup(300, res, seed=77 + mode, spread=24)
    ref = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
    got = gpu_fixed(vt, xyz, tets, res, mode=mode)
    assert (got == ref).all()
    assert ref.any()


def test_wide_tets_128bit_path(vt):
    """Tets wider than 2^20 lattice units take the 128-bit exact path."""
    rng = np.random.default_rng(7)
    for res in (8, 32, 128):
        xyz, tets = random_soup(rng, 40, res, spread=4.0, lo=-0.5, hi=1.5)
        for mode in (0, 1):
            ref = oracle.voxelize_fixed(xyz, tets, res, mode=mode)
            got = gpu_fixed(vt, xyz, tets, res, mode=mode)
            assert_same(got, ref, res, f"wide res={res} mode={mode}")
    # the extreme corners of the coordinate range
    C = 1 << 21
    xyz = np.array([[-C, -C, -C], [C, -C, -C], [-C, C, -C], [-C, -C, C], [C, C, C]], dtype=np.int32)
    tets = np.array([[0, 1, 2, 3], [4, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    ref = oracle.voxelize_fixed(xyz, tets, 32)
    assert_same(gpu_fixed(vt, xyz, tets, 32), ref, 32, "corners")


def test_slivers_and_degenerates(vt):
    v, t = mg.kuhn_lattice(12, 0.25, 5)
    v, t, _ = mg.add_slivers(v, t, 0.05, 6, d_lattice_units=range(0, 9))
    res = 128
    for mode in (0, 1):
        ref = oracle.voxelize(v, t, (0, 0, 0), 1 / res, res, mode=mode)
        got = gpu_world(vt, v, t, (0, 0, 0), 1 / res, res, mode=mode)
        assert_same(got, ref, res, f"slivers mode={mode}")
    flat = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0], [L // 2, L // 2, 0]], dtype=np.int32)
    got = gpu_fixed(vt, flat, np.array([[0, 1, 2, 3]], np.int32), 16)
    assert not got.any()


def test_world_coords_general_origin_and_voxel_size(vt):
    """Non-power-of-two voxel size (double division in the snap) and an offset origin."""
    v, t = mg.kuhn_lattice(6, 0.3, 8)
    v = (v * 1.7 - 0.35).astype(np.float32)
    for origin, h, res in [((-0.4, -0.3, -0.35), 1.6 / 64, 64), ((0.1, 0.2, -0.1), 0.0123, 128),
                           ((-0.5, -0.5, -0.5), 0.125, 16)]:
        st, _ = oracle.snap(v, origin, h, res)
        if st != 0:
            continue
        ref = oracle.voxelize(v, t, origin, h, res)
        got = gpu_world(vt, v, t, origin, h, res)
        assert_same(got, ref, res, f"origin={origin} h={h}")


def test_accumulate_ors_into_existing_grid(vt):
    import torch

    rng = np.random.default_rng(3)
    res = 64
    xa, ta = random_soup(rng, 30, res)
    xb, tb = random_soup(rng, 30, res)
    ref = oracle.voxelize_fixed(xa, ta, res) | oracle.voxelize_fixed(xb, tb, res)
    g = vt.voxelize_fixed(_dev(xa, torch.int32), _dev(ta, torch.int32), res)
    vt.voxelize_fixed(_dev(xb, torch.int32), _dev(tb, torch.int32), res, out=g, accumulate=True)
    assert_same(g.cpu().numpy(), ref, res, "accumulate")


def test_shuffle_and_duplicates_idempotent(vt):
    """Lost or racing OR writes would show up as order dependence."""
    c = mg.single_mesh_config("torus_48")
    rng = np.random.default_rng(0)
    t = c["tets"]
    base = gpu_world(vt, c["verts"], t, (0, 0, 0), 1 / 256, 256)
    shuf = np.concatenate([t, t[rng.permutation(len(t))[: len(t) // 3]]])[rng.permutation(len(t) + len(t) // 3)]
    got = gpu_world(vt, c["verts"], shuf, (0, 0, 0), 1 / 256, 256)
    assert np.array_equal(base, got)


def test_empty_and_tiny_inputs(vt):
    import torch

    g = vt.voxelize_fixed(torch.zeros((0, 3), dtype=torch.int32, device="cuda"),
                          torch.zeros((0, 4), dtype=torch.int32, device="cuda"), 64)
    assert int(torch.count_nonzero(g)) == 0
    # res = 1: one sample at the grid centre
    xyz = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0], [0, 0, L]], dtype=np.int32)
    assert gpu_fixed(vt, xyz, np.array([[0, 1, 2, 3]], np.int32), 1).ravel()[0] == 0  # centre outside corner tet
    xyz2 = np.array([[0, 0, 0], [L, 0, 0], [L, L, 0], [L, L, L]], dtype=np.int32)
    assert gpu_fixed(vt, xyz2, np.array([[0, 1, 2, 3]], np.int32), 1).ravel()[0] == 1  # on the diagonal: closed


def test_error_statuses(vt):
    import torch

    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float32)
    t = np.array([[0, 1, 2, 3]], dtype=np.int32)
    dv = lambda a: _dev(a, torch.float32)
    dt = lambda a: _dev(a, torch.int32)
    bad = v.copy()
    bad[1, 2] = np.inf
    st, _ = vt.voxelize(dv(bad), dt(t), (0, 0, 0), 0.25, 4, raise_on_error=False)
    assert st == vt.ERR_NAN
    far = v.copy()
    far[2, 0] = 5.0
    st, _ = vt.voxelize(dv(far), dt(t), (0, 0, 0), 0.25, 4, raise_on_error=False)
    assert st == vt.ERR_RANGE
    st, _ = vt.voxelize(dv(v), dt(np.array([[0, 1, 2, 9]], np.int32)), (0, 0, 0), 0.25, 4, raise_on_error=False)
    assert st == vt.ERR_INDEX
    st, _ = vt.voxelize(dv(v), dt(np.array([[0, -3, 2, 1]], np.int32)), (0, 0, 0), 0.25, 4, raise_on_error=False)
    assert st == vt.ERR_INDEX
    xyz = np.array([[0, 0, 0], [(1 << 21) + 1, 0, 0], [0, L, 0], [0, 0, L]], dtype=np.int32)
    st, _ = vt.voxelize_fixed(dt(xyz), dt(t), 8, raise_on_error=False)
    assert st == vt.ERR_RANGE
    # a bad vertex no tet names is reported too: with tets (the snap's error bits are folded in
    # by the last kernel of the call) and without any (the snap reports them itself)
    extra = np.concatenate([v, np.array([[np.nan, 0.5, 0.5]], np.float32)])
    st, _ = vt.voxelize(dv(extra), dt(t), (0, 0, 0), 0.25, 4, raise_on_error=False)
    assert st == vt.ERR_NAN
    st, _ = vt.voxelize(dv(extra), dt(np.zeros((0, 4), np.int32)), (0, 0, 0), 0.25, 4, raise_on_error=False)
    assert st == vt.ERR_NAN
    st, _ = vt.voxelize_grid(dv(extra), dt(t), (0, 0, 0), 0.25, (4, 3, 2), raise_on_error=False)
    assert st == vt.ERR_NAN
    xyz_extra = np.concatenate([xyz[:1], np.array([[0, L, 0], [L, 0, 0], [0, 0, L], [-(1 << 21) - 5, 0, 0]],
                                                  np.int32)])
    st, _ = vt.voxelize_fixed(dt(xyz_extra), dt(t), 8, raise_on_error=False)
    assert st == vt.ERR_RANGE
    # asynchronous form: the status is read afterwards from the workspace
    ws = vt.alloc_workspace(1, 4, 4)
    st, _ = vt.voxelize(dv(bad), dt(t), (0, 0, 0), 0.25, 4, workspace=ws, sync=False, raise_on_error=False)
    assert st == vt.OK
    assert vt.last_status(ws) == vt.ERR_NAN
    # a clean call afterwards on the same workspace reports OK again
    st, _ = vt.voxelize(dv(v), dt(t), (0, 0, 0), 0.25, 4, workspace=ws, raise_on_error=False)
    assert st == vt.OK


# ------------------------------------------------------------------ medium, whole grid

def test_torus_48_full_grid(vt):
    c = mg.single_mesh_config("torus_48")
    ref = oracle.voxelize(c["verts"], c["tets"], c["origin"], c["voxel_size"], c["res"])
    got = gpu_world(vt, c["verts"], c["tets"], c["origin"], c["voxel_size"], c["res"])
    assert_same(got, ref, c["res"], "torus_48")


# ------------------------------------------------------------------ full size, sampled slabs

def _slab_check(vt, name, n_slabs, depth, seed):
    import torch

    c = mg.single_mesh_config(name)
    res = c["res"]
    verts, tets = c["verts"], c["tets"]
    ws = vt.alloc_workspace(len(tets), len(verts), res)
    g = vt.voxelize(_dev(verts, torch.float32), _dev(tets, torch.int32), c["origin"], c["voxel_size"], res,
                    workspace=ws)
    stats = vt.read_stats(ws)
    st, xyz = oracle.snap(verts, c["origin"], c["voxel_size"], res)
    assert st == 0
    rng = np.random.default_rng(seed)
    starts = sorted(set([0, res - depth] + list(rng.integers(0, res - depth, size=n_slabs - 2))))
    for z0 in starts:
        ref = oracle.voxelize_fixed_slab(xyz, tets, res, int(z0), int(z0) + depth)
        got = g[z0:z0 + depth].cpu().numpy().view(np.uint32)
        if not np.array_equal(got, ref):
            a, b = oracle.unpack(got.reshape(depth * res, res, -1), res), oracle.unpack(
                ref.reshape(depth * res, res, -1), res)
            raise AssertionError(f"{name}: slab z0={z0} differs in {(a != b).sum()} samples")
    return stats


def test_full_size_sliver_60_at_512(vt):
    stats = _slab_check(vt, "sliver_60", n_slabs=6, depth=3, seed=1)
    assert stats["degenerate_tets"] > 0  # snapped slivers that became exactly flat
    assert stats["rows"] > 0
    assert stats["fallback_rows"] < 0.01 * stats["rows"]


@pytest.fixture(scope="module")
def sliver_512_oracle():
    """The whole 512^3 grid of the benchmark mesh from the oracle (all host cores)."""
    c = mg.single_mesh_config("sliver_60")
    st, xyz = oracle.snap(c["verts"], c["origin"], c["voxel_size"], c["res"])
    assert st == 0
    return c, oracle.voxelize_fixed(xyz, c["tets"], c["res"])


@pytest.mark.parametrize("span_rows,row_cull", [(0, 0), (1024, 1), (256, 1), (512, 2), (64, 1)])
def test_full_grid_sliver_60_at_512(vt, sliver_512_oracle, span_rows, row_cull):
    """The benchmark's workload compared with the oracle over every sample of the grid, in each
    launch shape the autotuner can choose (span sizes, culling on and off)."""
    import torch

    c, ref = sliver_512_oracle
    res = c["res"]
    ws = vt.alloc_workspace(len(c["tets"]), len(c["verts"]), res)
    g = vt.voxelize(_dev(c["verts"], torch.float32), _dev(c["tets"], torch.int32), c["origin"], c["voxel_size"], res,
                    workspace=ws, span_rows=span_rows, row_cull=row_cull)
    assert_same(g.cpu().numpy().view(np.uint32), ref, res, f"sliver_60 span_rows={span_rows} row_cull={row_cull}")


def test_full_size_sliver_60_at_1024(vt):
    _slab_check(vt, "sliver_60_1024", n_slabs=4, depth=2, seed=2)


def test_max_resolution_sampled(vt):
    """res = 8192 (a 64 GiB grid): a few tets, checked on the slabs they touch; the rest stays zero."""
    import torch

    res = 8192
    rng = np.random.default_rng(11)
    xyz, tets = random_soup(rng, 6, res, spread=0.01, lo=0.3, hi=0.32)
    g = vt.voxelize_fixed(_dev(xyz, torch.int32), _dev(tets, torch.int32), res)
    s = s_of(res)
    zmin = max(0, int((xyz[:, 2].min() - s) // (2 * s)))
    zmax = min(res, int((xyz[:, 2].max() - s) // (2 * s)) + 2)
    ref = oracle.voxelize_fixed_slab(xyz, tets, res, zmin, zmax)
    got = g[zmin:zmax].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)
    assert int(torch.count_nonzero(g[:zmin])) == 0 and int(torch.count_nonzero(g[zmax:])) == 0
    del g
    torch.cuda.empty_cache()


def test_max_mesh_size_full_lattice(vt):
    """48,000,000 tets (the unjittered 200^3 Kuhn lattice over the grid) at 512^3: a conforming
    tiling of the grid's cube, so its closed union sets every one of the 134 M bits -- a closed
    form at a size that exercises the 32-bit tet queues, tile counters and row queue."""
    import torch

    ijk, tets = mg.kuhn_lattice_int(200)
    verts = torch.from_numpy((ijk.astype(np.float32) / np.float32(200))).cuda()
    del ijk
    dt = torch.from_numpy(tets).cuda()
    del tets
    res = 512
    ws = vt.alloc_workspace(dt.shape[0], verts.shape[0], res)
    g = vt.voxelize(verts, dt, (0, 0, 0), 1.0 / res, res, workspace=ws)
    st = vt.read_stats(ws)
    assert st["degenerate_tets"] == 0
    assert bool((g == -1).all())  # every 32-bit word all ones
    del g, ws, verts, dt
    torch.cuda.empty_cache()


@pytest.mark.parametrize("res", [64, 512])
def test_snap_ties_zero_origin(vt, res):
    """Vertices exactly half a lattice unit off: with origin 0 and h = 1/res the snap runs in
    float and must round half to even exactly as the oracle's double arithmetic does."""
    v, t = mg.kuhn_lattice(4, 0.3, res)
    half = np.rint(v.astype(np.float64) * 2.0 ** 20) + 0.5  # (k + 1/2) lattice units
    v = (half * 2.0 ** -20).astype(np.float32)
    assert (v.astype(np.float64) * 2.0 ** 20 % 1 == 0.5).all()  # every coordinate is a tie
    st, xyz = oracle.snap(v, (0, 0, 0), 1.0 / res, res)
    assert st == 0 and (xyz % 2 == 0).all()  # ties went to even
    got = gpu_world(vt, v, t, (0, 0, 0), 1.0 / res, res)
    ref = oracle.voxelize(v, t, (0, 0, 0), 1.0 / res, res)
    assert (got == ref).all()
