"""Seeded synthetic tetrahedral meshes and job streams.

This module only *generates inputs*: float32 vertex arrays in the unit cube and
int32 tetrahedron index arrays, plus the batch and request-stream recipes built
on them.  It holds none of the voxelizer's arithmetic (no snapping, no
orientation tests, no sample logic), so both the CUDA path and the CPU oracle
can consume its output without sharing any of the method's code.

The meshes stand in for the good-quality tetrahedral meshes the paper
voxelizes (Section 3, "Voxelization": large minimum angle, no overlaps, small
size variance).  A jittered Kuhn lattice has exactly those properties, and the
paper's Thingi10k/ModelNet models are not available here.

Recipes (all seeds explicit; numpy PCG64):

* ``kuhn_lattice(N, jitter, seed)`` -- N^3 unit cells over [0,1]^3, vertex
  (i, j, l) at index (l*(N+1) + j)*(N+1) + i, each cell split into the 6 Kuhn
  tets along its (0,0,0)->(1,1,1) diagonal (one per permutation of the axes, in
  lexicographic order: v0 = cell corner, v_{t+1} = v_t + e_{pi(t)}).  Vertices
  with all three lattice indices strictly inside (1..N-1) move uniformly by up to
  +-jitter cells per axis, so the cube's faces stay flat.  The mesh is conforming.
* ``clip_by_centroid`` keeps the tets whose centroid lies inside an SDF and
  compacts away unreferenced vertices.
* ``add_slivers`` replaces a seeded fraction of tets by near-flat ones: a chosen
  vertex is projected onto the plane of its opposite face and lifted back by a
  tiny distance d, as a *new* vertex referenced by that tet only.
* ``batch_workload`` / ``poisson_stream`` build the many-mesh and served
  workloads (uneven sizes and resolutions).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "kuhn_lattice",
    "kuhn_lattice_int",
    "clip_by_centroid",
    "torus_sdf",
    "sphere_sdf",
    "box_sdf",
    "union_sdf",
    "add_slivers",
    "single_mesh_config",
    "BatchJob",
    "batch_workload",
    "Request",
    "poisson_stream",
    "mesh_pool",
]

# Kuhn subdivision of the unit cube: the 6 axis permutations in lexicographic order.
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _kuhn_cell_offsets() -> np.ndarray:
    """Corner offsets (6 tets x 4 verts x 3 axes) of the Kuhn split of a unit cell."""
    out = np.zeros((6, 4, 3), dtype=np.int64)
    for t, perm in enumerate(_PERMS):
        v = np.zeros(3, dtype=np.int64)
        out[t, 0] = v
        for step, axis in enumerate(perm):
            v = v.copy()
            v[axis] += 1
            out[t, step + 1] = v
    return out


def kuhn_lattice_int(N: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unjittered Kuhn lattice as integer lattice indices.

    Returns (ijk int64 [(N+1)^3, 3], tets int32 [6 N^3, 4]).
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    n1 = N + 1
    g = np.arange(n1, dtype=np.int64)
    l, j, i = np.meshgrid(g, g, g, indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), l.ravel()], axis=1)
    c = np.arange(N, dtype=np.int64)
    cl, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    corners = np.stack([ci.ravel(), cj.ravel(), cl.ravel()], axis=1)  # [N^3, 3]
    offs = _kuhn_cell_offsets()  # [6, 4, 3]
    pts = corners[:, None, None, :] + offs[None, :, :, :]  # [N^3, 6, 4, 3]
    idx = (pts[..., 2] * n1 + pts[..., 1]) * n1 + pts[..., 0]
    tets = idx.reshape(-1, 4).astype(np.int32)
    return ijk, tets


def kuhn_lattice(N: int, jitter: float = 0.0, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Jittered Kuhn lattice over [0,1]^3: (verts float32 [(N+1)^3, 3], tets int32 [6N^3, 4])."""
    ijk, tets = kuhn_lattice_int(N)
    return _jittered_positions(ijk, N, jitter, seed), tets


def _jittered_positions(ijk: np.ndarray, N: int, jitter: float, seed: int) -> np.ndarray:
    pos = ijk.astype(np.float64) / N
    if jitter:
        rng = np.random.Generator(np.random.PCG64(seed))
        interior = np.all((ijk > 0) & (ijk < N), axis=1)
        d = rng.uniform(-jitter, jitter, size=(int(interior.sum()), 3)) / N
        pos[interior] += d
    return pos.astype(np.float32)


def clipped_kuhn_lattice(N: int, jitter: float, seed: int, sdf) -> Tuple[np.ndarray, np.ndarray]:
    """``clip_by_centroid(*kuhn_lattice(N, jitter, seed), sdf)`` without building the
    tets of cells that cannot keep any: a tet's centroid lies within
    (sqrt(3)/2 + sqrt(3) jitter) cells of its cell's centre and the SDF is
    1-Lipschitz, so cells whose centre is farther outside are skipped.  The result
    is identical to the unfiltered recipe."""
    n1 = N + 1
    g = np.arange(n1, dtype=np.int64)
    l, j, i = np.meshgrid(g, g, g, indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), l.ravel()], axis=1)
    pos = _jittered_positions(ijk, N, jitter, seed)
    c = np.arange(N, dtype=np.int64)
    cl, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    corners = np.stack([ci.ravel(), cj.ravel(), cl.ravel()], axis=1)
    centre = (corners.astype(np.float64) + 0.5) / N
    reach = (np.sqrt(3.0) / 2 + np.sqrt(3.0) * abs(jitter) + 1e-6) / N
    corners = corners[sdf(centre) < reach]
    offs = _kuhn_cell_offsets()
    pts = corners[:, None, None, :] + offs[None, :, :, :]
    tets = ((pts[..., 2] * n1 + pts[..., 1]) * n1 + pts[..., 0]).reshape(-1, 4).astype(np.int32)
    return clip_by_centroid(pos, tets, sdf)


# ---------------------------------------------------------------- SDF clipping

def torus_sdf(R: float = 0.3, r: float = 0.12, centre=(0.5, 0.5, 0.5)) -> Callable[[np.ndarray], np.ndarray]:
    cx, cy, cz = centre

    def f(p: np.ndarray) -> np.ndarray:
        q = np.hypot(p[:, 0] - cx, p[:, 1] - cy) - R
        return np.hypot(q, p[:, 2] - cz) - r

    return f


def sphere_sdf(centre, radius: float) -> Callable[[np.ndarray], np.ndarray]:
    c = np.asarray(centre, dtype=np.float64)

    def f(p: np.ndarray) -> np.ndarray:
        return np.linalg.norm(p - c, axis=1) - radius

    return f


def box_sdf(centre, half) -> Callable[[np.ndarray], np.ndarray]:
    c = np.asarray(centre, dtype=np.float64)
    h = np.asarray(half, dtype=np.float64)

    def f(p: np.ndarray) -> np.ndarray:
        q = np.abs(p - c) - h
        outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
        inside = np.minimum(np.max(q, axis=1), 0.0)
        return outside + inside

    return f


def union_sdf(fs: Sequence[Callable[[np.ndarray], np.ndarray]]) -> Callable[[np.ndarray], np.ndarray]:
    def f(p: np.ndarray) -> np.ndarray:
        out = fs[0](p)
        for g in fs[1:]:
            out = np.minimum(out, g(p))
        return out

    return f


def clip_by_centroid(verts: np.ndarray, tets: np.ndarray, sdf) -> Tuple[np.ndarray, np.ndarray]:
    """Keep tets whose centroid has sdf < 0; drop and re-index unreferenced vertices."""
    cent = verts.astype(np.float64)[tets].mean(axis=1)
    keep = sdf(cent) < 0.0
    kept = tets[keep]
    used = np.zeros(len(verts), dtype=bool)
    used[kept.ravel()] = True
    remap = np.full(len(verts), -1, dtype=np.int64)
    remap[used] = np.arange(int(used.sum()))
    return verts[used].copy(), remap[kept].astype(np.int32)


# ---------------------------------------------------------------- slivers

def add_slivers(
    verts: np.ndarray,
    tets: np.ndarray,
    frac: float,
    seed: int,
    d_max: float = 1e-6,
    d_lattice_units: Optional[Sequence[int]] = None,
) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Turn a seeded fraction of tets into near-flat slivers.

    For each chosen tet one vertex (seeded) is replaced by a new vertex: its
    projection onto the plane of the opposite face, lifted back toward its
    original side by d.  d ~ U(0, d_max) in world units, or, when
    ``d_lattice_units`` is given, d = m * 2^-20 with m drawn from that list.
    Neighbouring tets keep the old vertex, so the result is a tet soup.

    Returns (verts, tets, sliver_tet_ids).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(tets)
    k = int(round(frac * n))
    ids = np.sort(rng.choice(n, size=k, replace=False)) if k else np.zeros(0, dtype=np.int64)
    which = rng.integers(0, 4, size=k)
    if d_lattice_units is not None:
        d = rng.choice(np.asarray(d_lattice_units, dtype=np.float64), size=k) * 2.0 ** -20
    else:
        d = rng.uniform(0.0, d_max, size=k)
    P = verts.astype(np.float64)
    T = tets[ids].astype(np.int64)
    moved = T[np.arange(k), which]
    others = np.stack([T[np.arange(k), (which + o) % 4] for o in (1, 2, 3)], axis=1)
    A, B, C = P[others[:, 0]], P[others[:, 1]], P[others[:, 2]]
    nrm = np.cross(B - A, C - A)
    nlen = np.linalg.norm(nrm, axis=1, keepdims=True)
    nlen[nlen == 0] = 1.0
    nrm = nrm / nlen
    X = P[moved]
    h = np.einsum("ij,ij->i", X - A, nrm)
    side = np.where(h >= 0, 1.0, -1.0)
    newp = X - h[:, None] * nrm + (side * d)[:, None] * nrm
    new_idx = len(verts) + np.arange(k)
    out_t = tets.copy()
    out_t[ids, which] = new_idx.astype(np.int32)
    out_v = np.concatenate([verts, newp.astype(np.float32)], axis=0)
    return out_v, out_t, ids


# ---------------------------------------------------------------- single-mesh workloads

def coplanar_face_soup(n_tets: int, res: int, seed: int, spread: int,
                       region: Optional[Sequence[Tuple[int, int]]] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Tie-heavy tet soup on the lattice of a cubic 2^k grid (int32 lattice coordinates, tets).

    Each tet has one face on a plane n . X = n . P through a voxel-centre sample P
    ((2a+1)s per axis, s = 2^(19-k)) with a small integer normal n; that plane holds
    many other samples, so the four orientation values of many samples are exactly
    zero.  The face's three vertices and the fourth vertex lie within ``spread``
    voxels of P at unaligned lattice points, so the zeros only appear after
    cancellation of large products -- the case where inexact arithmetic picks signs
    at random.  All coordinates stay within 2^21.  ``region`` ((x0, x1), (y0, y1), (z0, z1)),
    in sample indices, limits where the planes' samples P are drawn (default: the whole grid).
    """
    k = res.bit_length() - 1
    if res < 1 or (1 << k) != res:
        raise ValueError("res must be a power of two")
    s = 1 << (19 - k)
    rng = np.random.Generator(np.random.PCG64(seed))
    verts: List[np.ndarray] = []
    tets: List[List[int]] = []
    lim = 1 << 21
    while len(tets) < n_tets:
        lo_hi = region if region is not None else ((0, res), (0, res), (0, res))
        P = (2 * np.array([rng.integers(a, b) for a, b in lo_hi], dtype=np.int64) + 1) * s
        nrm = rng.integers(-3, 4, size=3)
        if not nrm.any():
            continue
        c = int(nrm @ P)
        ax = int(np.argmax(np.abs(nrm)))
        face: List[np.ndarray] = []
        for _ in range(50):
            q = P + rng.integers(-spread * s, spread * s + 1, size=3)
            r = c - int(nrm @ q) + int(nrm[ax]) * int(q[ax])
            if r % int(nrm[ax]):
                continue
            q[ax] = r // int(nrm[ax])
            if np.abs(q).max() > lim:
                continue
            face.append(q)
            if len(face) == 3:
                break
        U = P + rng.integers(-spread * s, spread * s + 1, size=3)
        if len(face) < 3 or np.abs(U).max() > lim:
            continue
        b = len(verts)
        verts += face + [U]
        tets.append([b, b + 1, b + 2, b + 3])
    return np.asarray(verts, dtype=np.int32).reshape(-1, 3), np.asarray(tets, dtype=np.int32).reshape(-1, 4)


def single_mesh_config(name: str) -> dict:
    """The single-mesh workloads, by name.

    * ``plain_8``: 8^3 Kuhn lattice (3,072 tets, 729 verts), jitter +-0.2 cell,
      64^3 grid.
    * ``torus_48``: 48^3 lattice, jitter +-0.25, tets with centroid inside the
      torus (R=0.3, r=0.12) kept; 256^3 grid.  ``torus_73`` is the same recipe on
      a 73^3 lattice (about 200k tets).
    * ``sliver_60``: 60^3 lattice (1,296,000 tets), jitter +-0.25, 2% of tets
      turned into slivers with d ~ U(0, 1e-6); 512^3 grid (``sliver_60_1024``:
      1024^3).  ``sliver_60_lattice`` uses d in {1..8} lattice units instead.
    """
    seeds = {"plain_8": 1000, "torus_48": 1001, "torus_73": 1001, "sliver_60": 1002,
             "sliver_60_1024": 1002, "sliver_60_lattice": 1002}
    if name not in seeds:
        raise KeyError(name)
    seed = seeds[name]
    slivers = None
    if name == "plain_8":
        v, t = kuhn_lattice(8, 0.2, seed)
        res = 64
    elif name in ("torus_48", "torus_73"):
        N = 48 if name == "torus_48" else 73
        v, t = clipped_kuhn_lattice(N, 0.25, seed, torus_sdf())
        res = 256
    else:
        v, t = kuhn_lattice(60, 0.25, seed)
        if name == "sliver_60_lattice":
            v, t, slivers = add_slivers(v, t, 0.02, seed + 7, d_lattice_units=range(1, 9))
        else:
            v, t, slivers = add_slivers(v, t, 0.02, seed + 7, d_max=1e-6)
        res = 1024 if name == "sliver_60_1024" else 512
    return {"name": name, "verts": v, "tets": t, "res": res, "origin": (0.0, 0.0, 0.0),
            "voxel_size": 1.0 / res, "seed": seed, "sliver_ids": slivers}


# ---------------------------------------------------------------- many-mesh workloads

@dataclasses.dataclass
class BatchJob:
    verts: np.ndarray
    tets: np.ndarray
    res: int
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    voxel_size: float = 0.0
    seed: int = 0

    def __post_init__(self):
        if not self.voxel_size:
            self.voxel_size = 1.0 / self.res


def _random_union(rng: np.random.Generator):
    shapes = []
    for _ in range(int(rng.integers(1, 4))):
        kind = int(rng.integers(0, 3))
        c = rng.uniform(0.3, 0.7, size=3)
        if kind == 0:
            shapes.append(sphere_sdf(c, float(rng.uniform(0.12, 0.3))))
        elif kind == 1:
            shapes.append(box_sdf(c, rng.uniform(0.08, 0.28, size=3)))
        else:
            R = float(rng.uniform(0.15, 0.3))
            shapes.append(torus_sdf(R, float(rng.uniform(0.05, min(0.15, R - 0.02))), tuple(c)))
    return union_sdf(shapes)


def clipped_mesh(target_tets: int, seed: int, jitter: float = 0.25) -> Tuple[np.ndarray, np.ndarray]:
    """Jittered Kuhn lattice clipped by a seeded union of 1-3 sphere/box/torus SDFs.

    The lattice size N is chosen from a Monte-Carlo estimate of the kept volume
    fraction so that the kept tet count lands near ``target_tets``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sdf = _random_union(rng)
    probe = rng.uniform(0.0, 1.0, size=(20000, 3))
    frac = max(float((sdf(probe) < 0).mean()), 1e-3)
    N = max(2, int(round((target_tets / (6.0 * frac)) ** (1.0 / 3.0))))
    v, t = clipped_kuhn_lattice(N, jitter, seed + 1, sdf)
    if len(t) == 0:  # pathological clip: fall back to the whole lattice
        v, t = kuhn_lattice(N, jitter, seed + 1)
    return v, t


def batch_workload(n_meshes: int = 256, seed: int = 1003, tets_lo: int = 1000, tets_hi: int = 100000,
                   resolutions: Sequence[int] = (32, 64, 128)) -> List[BatchJob]:
    """Many meshes of uneven size: tet counts log-uniform in [tets_lo, tets_hi],
    each grid resolution drawn uniformly from ``resolutions``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    targets = np.exp(rng.uniform(math.log(tets_lo), math.log(tets_hi), size=n_meshes))
    ress = rng.choice(np.asarray(resolutions), size=n_meshes)
    jobs = []
    for m in range(n_meshes):
        v, t = clipped_mesh(int(targets[m]), seed * 1000 + m)
        jobs.append(BatchJob(v, t, int(ress[m]), seed=seed * 1000 + m))
    return jobs


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    mesh_id: int
    res: int


def mesh_pool(n_meshes: int, seed: int, tets_lo: int, tets_hi: int) -> List[Tuple[np.ndarray, np.ndarray]]:
    """A seeded pool of clipped meshes with log-uniform tet counts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    targets = np.exp(rng.uniform(math.log(tets_lo), math.log(tets_hi), size=n_meshes))
    return [clipped_mesh(int(targets[m]), seed * 1000 + m) for m in range(n_meshes)]


def poisson_stream(n_requests: int, rate_per_s: float, n_pool: int, seed: int = 1004,
                   resolutions: Sequence[int] = (64, 128, 256, 512)) -> List[Request]:
    """Poisson arrivals (exponential gaps at ``rate_per_s``); each request names a
    pool mesh (uniform) and a resolution (uniform over ``resolutions``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    mids = rng.integers(0, n_pool, size=n_requests)
    ress = rng.choice(np.asarray(resolutions), size=n_requests)
    return [Request(i, float(t[i]), int(mids[i]), int(ress[i])) for i in range(n_requests)]
