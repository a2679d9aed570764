"""Independent pure-Python checker (test infrastructure only).

A second formulation of the same grid, in Python's unbounded integers, used to
pin the C oracle on tiny inputs.  It does not follow Theorem 1's D_a..D_d
patterns; it first orients each tetrahedron to positive signed volume
(Lemma 1.1: swapping two vertices flips the sign of det(AB, AC, AD)) and then
requires the four barycentric orientation values

    lam_0 = orient(P, V1, V2, V3)   lam_1 = orient(V0, P, V2, V3)
    lam_2 = orient(V0, V1, P, V3)   lam_3 = orient(V0, V1, V2, P)

with orient(A, B, C, D) = det[B - A, C - A, D - A], to be >= 0 (closed reading)
or > 0 (the paper's strict statement).  They sum to the tetrahedron's signed
volume times 6, and lam_0 = D_a, lam_1 = -D_b, lam_2 = D_c, lam_3 = -D_d for
the unswapped vertex order, which is why the two formulations must agree.

Snapping follows the same reading as the oracle: each double operation of
((double)v - o) / h is rounded to nearest, the power-of-two scale is exact,
and the result is rounded half to even.  Python floats are IEEE doubles and
``round`` on a float rounds half to even, so this is an independent restatement.
"""
from __future__ import annotations

from typing import Iterable, Sequence, Tuple

import numpy as np

LATTICE_BITS = 20
COORD_LIMIT = 1 << 21


def log2_res(res: int) -> int:
    if res < 1 or res > (1 << 19) or (res & (res - 1)):
        raise ValueError("res must be a power of two in [1, 2^19]")
    return res.bit_length() - 1


def grid_exponent_py(res: Sequence[int]) -> int:
    """Smallest K with 2^K >= every side of the grid (sides in [1, 2^19])."""
    if any(int(r) < 1 or int(r) > (1 << 19) for r in res):
        raise ValueError("grid sides must be in [1, 2^19]")
    K = 0
    while (1 << K) < max(int(r) for r in res):
        K += 1
    return K


def snap_py(verts: np.ndarray, origin: Sequence[float], h: float, res: int) -> np.ndarray:
    return _snap_k(verts, origin, h, log2_res(res))


def snap_grid_py(verts: np.ndarray, origin: Sequence[float], h: float, res: Sequence[int]) -> np.ndarray:
    return _snap_k(verts, origin, h, grid_exponent_py(res))


def _snap_k(verts: np.ndarray, origin: Sequence[float], h: float, k: int) -> np.ndarray:
    scale = float(2 ** (LATTICE_BITS - k))
    out = np.zeros((len(verts), 3), dtype=np.int64)
    for v in range(len(verts)):
        for q in range(3):
            f = float(np.float32(verts[v][q]))
            o = float(np.float32(origin[q]))
            x = ((f - o) / float(np.float32(h))) * scale
            r = round(x)
            if abs(r) > COORD_LIMIT:
                raise ValueError("coordinate out of range")
            out[v, q] = r
    return out


def orient(A, B, C, D) -> int:
    b = [int(B[q]) - int(A[q]) for q in range(3)]
    c = [int(C[q]) - int(A[q]) for q in range(3)]
    d = [int(D[q]) - int(A[q]) for q in range(3)]
    return (b[0] * (c[1] * d[2] - c[2] * d[1])
            - b[1] * (c[0] * d[2] - c[2] * d[0])
            + b[2] * (c[0] * d[1] - c[1] * d[0]))


def voxelize_py(xyz: np.ndarray, tets: np.ndarray, res: int, mode: int = 0) -> np.ndarray:
    """Boolean occupancy [l, j, i] (z, y, x) of the union of closed tets."""
    log2_res(res)
    return voxelize_grid_py(xyz, tets, (res, res, res), mode)


def voxelize_grid_py(xyz: np.ndarray, tets: np.ndarray, res: Sequence[int], mode: int = 0) -> np.ndarray:
    """Boolean occupancy [l, j, i] of a general grid res = (rx, ry, rz)."""
    k = grid_exponent_py(res)
    s = 1 << (19 - k)
    rx, ry, rz = (int(r) for r in res)
    occ = np.zeros((rz, ry, rx), dtype=bool)
    lim = (rx, ry, rz)
    P3 = [[int(c) for c in row] for row in np.asarray(xyz).reshape(-1, 3)]
    for tet in np.asarray(tets).reshape(-1, 4):
        V = [P3[int(i)] for i in tet]
        v6 = orient(*V)
        if v6 == 0:
            continue
        if v6 < 0:
            V = [V[0], V[1], V[3], V[2]]
        lo, hi = [], []
        for q in range(3):
            mn = min(v[q] for v in V)
            mx = max(v[q] for v in V)
            lo.append(max(0, -((-(mn - s)) // (2 * s))))
            hi.append(min(lim[q] - 1, (mx - s) // (2 * s)))
        for l in range(lo[2], hi[2] + 1):
            for j in range(lo[1], hi[1] + 1):
                for i in range(lo[0], hi[0] + 1):
                    P = ((2 * i + 1) * s, (2 * j + 1) * s, (2 * l + 1) * s)
                    lam = (orient(P, V[1], V[2], V[3]), orient(V[0], P, V[2], V[3]),
                           orient(V[0], V[1], P, V[3]), orient(V[0], V[1], V[2], P))
                    if (min(lam) >= 0) if mode == 0 else (min(lam) > 0):
                        occ[l, j, i] = True
    return occ
