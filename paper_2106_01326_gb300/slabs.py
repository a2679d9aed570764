"""Partition of one grid into z-slabs, one per rank.

Slabs of a grid are disjoint, contiguous runs of slices and, in the z-major bit
layout, disjoint contiguous byte ranges of the output; a rank that voxelizes its
slab (``voxtet.voxelize_grid(..., z_range=...)``) needs no data from any other
rank, so the only collective a caller may want is a gather of the finished slabs.

``slab_cuts`` splits the slices evenly, or, given per-slice weights, so that each
rank's share of the total weight is as even as contiguous runs allow.
``slice_weights`` estimates that weight from a mesh: the number of tetrahedra
whose vertical extent covers each slice (each covering tet costs a slice table
entry and its rows there).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def slab_cuts(rz: int, world: int, weights: Optional[Sequence[float]] = None) -> List[Tuple[int, int]]:
    """[(z0, z1)] for ranks 0..world-1: contiguous, covering [0, rz), possibly empty."""
    if rz < 0 or world < 1:
        raise ValueError("need rz >= 0 and world >= 1")
    if weights is None:
        base, extra = divmod(rz, world)
        cuts, z = [], 0
        for r in range(world):
            n = base + (1 if r < extra else 0)
            cuts.append((z, z + n))
            z += n
        return cuts
    w = np.asarray(weights, dtype=np.float64)
    if w.shape != (rz,) or (w < 0).any():
        raise ValueError("weights must be rz non-negative numbers")
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        z = int(np.searchsorted(cum, target, side="left"))
        bounds.append(min(max(z, bounds[-1]), rz))
    bounds.append(rz)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def _checked(verts: np.ndarray, tets: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """The mesh as arrays, after the checks the library's kernels make on the device: every index
    in [0, n_verts) and every coordinate finite.  A slab's subset must not hide a bad tet or vertex
    (numpy would wrap a negative index, and a NaN fails every comparison), so a bad mesh raises
    here instead of returning a slab the whole-mesh call would have rejected."""
    v = np.asarray(verts)
    t = np.asarray(tets).reshape(-1, 4)
    if t.size and (int(t.min()) < 0 or int(t.max()) >= len(v)):
        raise ValueError("a tetrahedron names a vertex outside [0, n_verts)")
    if not np.isfinite(v).all():
        raise ValueError("a vertex coordinate is NaN or infinite")
    return v, t


def slice_weights(verts: np.ndarray, tets: np.ndarray, origin: Sequence[float], voxel_size: float,
                  rz: int) -> np.ndarray:
    """Tets covering each slice's sample plane (float estimate from world coordinates)."""
    verts, tets = _checked(verts, tets)
    z = np.asarray(verts, dtype=np.float64)[:, 2][tets]
    lo = np.ceil((z.min(axis=1) - float(origin[2])) / float(voxel_size) - 0.5)
    hi = np.floor((z.max(axis=1) - float(origin[2])) / float(voxel_size) - 0.5)
    lo = np.clip(lo, 0, rz).astype(np.int64)
    hi = np.clip(hi + 1, 0, rz).astype(np.int64)  # exclusive
    keep = lo < hi
    lo, hi = lo[keep], hi[keep]
    d = np.zeros(rz + 1, dtype=np.float64)
    np.add.at(d, lo, 1.0)
    np.add.at(d, hi, -1.0)
    return np.cumsum(d)[:rz]


def tets_for_slab(verts: np.ndarray, tets: np.ndarray, origin: Sequence[float], voxel_size: float, z0: int,
                  z1: int) -> np.ndarray:
    """The tets that may have samples in slices [z0, z1): a superset (one slice of margin on each
    side covers the difference between world coordinates and their snapped lattice points), so a
    rank that voxelizes its slab from these alone gets the same bits as from the whole mesh."""
    verts, t = _checked(verts, tets)
    z = np.asarray(verts, dtype=np.float64)[:, 2][t]
    lo = np.floor((z.min(axis=1) - float(origin[2])) / float(voxel_size)) - 1
    hi = np.ceil((z.max(axis=1) - float(origin[2])) / float(voxel_size)) + 1
    keep = (hi >= z0) & (lo <= z1 - 1)
    return np.ascontiguousarray(t[keep])


def slab_mesh(verts: np.ndarray, tets: np.ndarray, origin: Sequence[float], voxel_size: float, z0: int,
              z1: int) -> Tuple[np.ndarray, np.ndarray]:
    """(vertices, tets) of a rank's slab: the tets of ``tets_for_slab`` renumbered onto only the
    vertices they name, so that the rank's call snaps those vertices and no others.  Snapping is
    per vertex, so the slab's bits are unchanged."""
    v = np.asarray(verts)
    sub = tets_for_slab(v, tets, origin, voxel_size, z0, z1)
    used, inv = np.unique(sub.reshape(-1), return_inverse=True)
    return np.ascontiguousarray(v[used]), np.ascontiguousarray(inv.reshape(-1, 4).astype(np.int32))


def rank_slab(rz: int, rank: int, world: int, weights: Optional[Sequence[float]] = None) -> Tuple[int, int]:
    """This rank's (z0, z1)."""
    return slab_cuts(rz, world, weights)[rank]
