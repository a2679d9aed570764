"""CPU oracle for tetrahedral-mesh solid voxelization (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

Two independent oracles live here:

* ``voxtet_oracle.c`` -- plain C, exact 128-bit integer determinants, the
  paper's Theorem 1 sign patterns (Section 4) applied to every voxel-centre
  sample in every tetrahedron's bounding box (Section 3, "Voxelization").
  Loaded through ctypes after ``build()`` compiles it with gcc.
* ``bigint_check`` -- pure Python integers, a different formulation
  (orientation-normalised barycentric signs), for tiny inputs.

``paper_cpu.c`` (same library) is not an oracle: it is the paper's CPU method in
float or double, kept here to count what inexact arithmetic decides differently.

Status codes: 0 ok, -1 bad argument, -2 resolution not a power of two in
[1, 2^19] (general grids: a side outside [1, 2^19]), -3 vertex index out of
range, -4 snapped coordinate beyond 2^21, -5 non-finite vertex coordinate.

General grids (``*_grid`` functions) take res = (rx, ry, rz) of any sizes and a
z-slab [z0, z1); the lattice step per voxel is 2^(20-K), K = ceil(log2(max side)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voxtet_oracle.c")
_SRC_PAPER = os.path.join(_HERE, "paper_cpu.c")
_LIB_PATH = os.path.join(_HERE, "libvoxtet_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_RES, ERR_INDEX, ERR_RANGE, ERR_NAN = 0, -1, -2, -3, -4, -5


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PAPER))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, _SRC_PAPER, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float
            lib.voxtet_oracle_snap.argtypes = [P, i64, P, f32, i32, P]
            lib.voxtet_oracle_snap.restype = ctypes.c_int
            lib.voxtet_oracle_voxelize_fixed.argtypes = [P, i64, P, i64, i32, i32, i32, P, P]
            lib.voxtet_oracle_voxelize_fixed.restype = ctypes.c_int
            lib.voxtet_oracle_voxelize_fixed_slab.argtypes = [P, i64, P, i64, i32, i32, i32, i32, i32, P, P]
            lib.voxtet_oracle_voxelize_fixed_slab.restype = ctypes.c_int
            lib.voxtet_oracle_voxelize.argtypes = [P, i64, P, i64, P, f32, i32, i32, i32, P, P]
            lib.voxtet_oracle_voxelize.restype = ctypes.c_int
            lib.voxtet_oracle_all_pairs.argtypes = [P, i64, P, i64, i32, i32, P]
            lib.voxtet_oracle_all_pairs.restype = ctypes.c_int
            lib.voxtet_oracle_snap_grid.argtypes = [P, i64, P, f32, P, P]
            lib.voxtet_oracle_snap_grid.restype = ctypes.c_int
            lib.voxtet_oracle_voxelize_grid_fixed.argtypes = [P, i64, P, i64, P, i32, i32, i32, i32, P, P]
            lib.voxtet_oracle_voxelize_grid_fixed.restype = ctypes.c_int
            lib.voxtet_oracle_voxelize_grid.argtypes = [P, i64, P, i64, P, f32, P, i32, i32, i32, i32, P, P]
            lib.voxtet_oracle_voxelize_grid.restype = ctypes.c_int
            lib.voxtet_oracle_all_pairs_grid.argtypes = [P, i64, P, i64, P, i32, P]
            lib.voxtet_oracle_all_pairs_grid.restype = ctypes.c_int
            lib.voxtet_paper_cpu.argtypes = [P, i64, P, i64, i32, i32, i32, i32, P]
            lib.voxtet_paper_cpu.restype = ctypes.c_int
            lib.voxtet_paper_cpu_disagreements.argtypes = [P, i64, P, i64, i32, i32, i32, i32, P]
            lib.voxtet_paper_cpu_disagreements.restype = ctypes.c_int
            lib.voxtet_oracle_theorem1_dets.argtypes = [P, P, P, P, P, P]
            lib.voxtet_oracle_theorem1_dets.restype = None
            lib.voxtet_oracle_num_threads.argtypes = []
            lib.voxtet_oracle_num_threads.restype = ctypes.c_int
            lib.voxtet_oracle_last_threads.argtypes = []
            lib.voxtet_oracle_last_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def grid_words(res: int) -> int:
    return res * res * ((res + 31) // 32)


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}")
        self.status = status


def snap(verts: np.ndarray, origin, voxel_size: float, res: int) -> Tuple[int, np.ndarray]:
    lib = _load()
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).reshape(3))
    out = np.zeros((len(v), 3), dtype=np.int32)
    st = lib.voxtet_oracle_snap(_ptr(v), len(v), _ptr(o), float(voxel_size), int(res), _ptr(out))
    return st, out


def voxelize_fixed(xyz: np.ndarray, tets: np.ndarray, res: int, mode: int = 0, n_threads: int = 0,
                   with_stats: bool = False, raise_on_error: bool = True):
    """Grid (uint32 [res, res, W]) of the union of closed tets on lattice coordinates."""
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    W = (res + 31) // 32 if res > 0 else 1
    out = np.zeros(max(res, 1) * max(res, 1) * W, dtype=np.uint32)
    stats = np.zeros(4, dtype=np.int64)
    st = lib.voxtet_oracle_voxelize_fixed(_ptr(x), len(x), _ptr(t), len(t), int(res), int(mode),
                                          int(n_threads), _ptr(out), _ptr(stats))
    if st != OK:
        if raise_on_error:
            raise OracleError(st)
        return (st, None, None) if with_stats else (st, None)
    grid = out.reshape(res, res, W)
    if with_stats:
        return grid, {"degenerate": int(stats[0]), "tested": int(stats[1]), "set": int(stats[2]),
                      "rows_with_samples": int(stats[3])}
    return grid


def voxelize_fixed_slab(xyz: np.ndarray, tets: np.ndarray, res: int, z0: int, z1: int, mode: int = 0,
                        n_threads: int = 0, with_stats: bool = False):
    """Slices z0 <= l < z1 of the grid (uint32 [z1 - z0, res, W]); same semantics as ``voxelize_fixed``."""
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    W = (res + 31) // 32
    out = np.zeros(max(z1 - z0, 1) * res * W, dtype=np.uint32)
    stats = np.zeros(4, dtype=np.int64)
    st = lib.voxtet_oracle_voxelize_fixed_slab(_ptr(x), len(x), _ptr(t), len(t), int(res), int(mode),
                                               int(n_threads), int(z0), int(z1), _ptr(out), _ptr(stats))
    if st != OK:
        raise OracleError(st)
    grid = out[: (z1 - z0) * res * W].reshape(z1 - z0, res, W)
    if with_stats:
        return grid, {"degenerate": int(stats[0]), "tested": int(stats[1]), "set": int(stats[2]),
                      "rows_with_samples": int(stats[3])}
    return grid


def voxelize(verts: np.ndarray, tets: np.ndarray, origin, voxel_size: float, res: int, mode: int = 0,
             n_threads: int = 0, with_stats: bool = False, raise_on_error: bool = True):
    """Grid of float32 vertices snapped to the 2^20 lattice, then voxelized."""
    lib = _load()
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).reshape(3))
    W = (res + 31) // 32 if res > 0 else 1
    out = np.zeros(max(res, 1) * max(res, 1) * W, dtype=np.uint32)
    stats = np.zeros(4, dtype=np.int64)
    st = lib.voxtet_oracle_voxelize(_ptr(v), len(v), _ptr(t), len(t), _ptr(o), float(voxel_size), int(res),
                                    int(mode), int(n_threads), _ptr(out), _ptr(stats))
    if st != OK:
        if raise_on_error:
            raise OracleError(st)
        return (st, None, None) if with_stats else (st, None)
    grid = out.reshape(res, res, W)
    if with_stats:
        return grid, {"degenerate": int(stats[0]), "tested": int(stats[1]), "set": int(stats[2]),
                      "rows_with_samples": int(stats[3])}
    return grid


def all_pairs(xyz: np.ndarray, tets: np.ndarray, res: int, mode: int = 0) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    W = (res + 31) // 32
    out = np.zeros(res * res * W, dtype=np.uint32)
    st = lib.voxtet_oracle_all_pairs(_ptr(x), len(x), _ptr(t), len(t), int(res), int(mode), _ptr(out))
    if st != OK:
        raise OracleError(st)
    return out.reshape(res, res, W)


def _res3(res) -> np.ndarray:
    r = np.ascontiguousarray(np.asarray(res, dtype=np.int32).reshape(3))
    return r


def grid_exponent(res) -> int:
    """K = ceil(log2(max side)) of a general grid: the lattice step is 2^(20-K) per voxel."""
    m = int(max(int(x) for x in res))
    return (m - 1).bit_length()


def snap_grid(verts: np.ndarray, origin, voxel_size: float, res) -> Tuple[int, np.ndarray]:
    """Lattice coordinates of float vertices on the lattice of the general grid ``res`` = (rx, ry, rz)."""
    lib = _load()
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).reshape(3))
    out = np.zeros((len(v), 3), dtype=np.int32)
    st = lib.voxtet_oracle_snap_grid(_ptr(v), len(v), _ptr(o), float(voxel_size), _ptr(_res3(res)), _ptr(out))
    return st, out


def _grid_out(res, z0, z1):
    rx, ry, rz = (int(x) for x in res)
    z1 = rz if z1 is None else int(z1)
    W = (rx + 31) // 32
    n = max(z1 - int(z0), 0) * ry * W
    return np.zeros(max(n, 1), dtype=np.uint32), (max(z1 - int(z0), 0), ry, W), z1


def voxelize_grid_fixed(xyz: np.ndarray, tets: np.ndarray, res, z0: int = 0, z1: Optional[int] = None,
                        mode: int = 0, n_threads: int = 0, with_stats: bool = False):
    """Slices z0 <= l < z1 (default: all) of the general grid res = (rx, ry, rz): uint32 [z1 - z0, ry, W]."""
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    out, shape, z1 = _grid_out(res, z0, z1)
    stats = np.zeros(4, dtype=np.int64)
    st = lib.voxtet_oracle_voxelize_grid_fixed(_ptr(x), len(x), _ptr(t), len(t), _ptr(_res3(res)), int(mode),
                                               int(n_threads), int(z0), int(z1), _ptr(out), _ptr(stats))
    if st != OK:
        raise OracleError(st)
    grid = out[: int(np.prod(shape))].reshape(shape)
    if with_stats:
        return grid, {"degenerate": int(stats[0]), "tested": int(stats[1]), "set": int(stats[2]),
                      "rows_with_samples": int(stats[3])}
    return grid


def voxelize_grid(verts: np.ndarray, tets: np.ndarray, origin, voxel_size: float, res, z0: int = 0,
                  z1: Optional[int] = None, mode: int = 0, n_threads: int = 0, with_stats: bool = False):
    """General-grid voxelization of float32 vertices (snap_grid, then voxelize_grid_fixed)."""
    lib = _load()
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).reshape(3))
    out, shape, z1 = _grid_out(res, z0, z1)
    stats = np.zeros(4, dtype=np.int64)
    st = lib.voxtet_oracle_voxelize_grid(_ptr(v), len(v), _ptr(t), len(t), _ptr(o), float(voxel_size),
                                         _ptr(_res3(res)), int(mode), int(n_threads), int(z0), int(z1), _ptr(out),
                                         _ptr(stats))
    if st != OK:
        raise OracleError(st)
    grid = out[: int(np.prod(shape))].reshape(shape)
    if with_stats:
        return grid, {"degenerate": int(stats[0]), "tested": int(stats[1]), "set": int(stats[2]),
                      "rows_with_samples": int(stats[3])}
    return grid


def all_pairs_grid(xyz: np.ndarray, tets: np.ndarray, res, mode: int = 0) -> np.ndarray:
    """Every sample of the general grid against every tet (no pruning): uint32 [rz, ry, W]."""
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    out, shape, _ = _grid_out(res, 0, None)
    st = lib.voxtet_oracle_all_pairs_grid(_ptr(x), len(x), _ptr(t), len(t), _ptr(_res3(res)), int(mode),
                                          _ptr(out))
    if st != OK:
        raise OracleError(st)
    return out[: int(np.prod(shape))].reshape(shape)


def unpack_grid(grid: np.ndarray, rx: int) -> np.ndarray:
    """Bit grid (uint32 [nz, ry, W]) -> bool [nz, ry, rx] (z, y, x)."""
    g = np.ascontiguousarray(grid, dtype=np.uint32)
    bits = np.unpackbits(g.view(np.uint8), axis=-1, bitorder="little")
    return bits[..., :rx].astype(bool)


def pack_grid(occ: np.ndarray) -> np.ndarray:
    """Inverse of ``unpack_grid``: bool [nz, ry, rx] -> uint32 [nz, ry, ceil(rx / 32)]."""
    nz, ry, rx = occ.shape
    W = (rx + 31) // 32
    pad = np.zeros((nz, ry, W * 32), dtype=np.uint8)
    pad[..., :rx] = occ
    return np.packbits(pad, axis=-1, bitorder="little").view(np.uint32).reshape(nz, ry, W)


def paper_cpu(xyz: np.ndarray, tets: np.ndarray, res: int, precision: str = "float", mode: int = 0,
              n_threads: int = 0) -> np.ndarray:
    """The paper's CPU method in float or double (paper_cpu.c): NOT exact, for counting its
    differences from ``voxelize_fixed``.  Same inputs and grid layout."""
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    W = (res + 31) // 32
    out = np.zeros(res * res * W, dtype=np.uint32)
    st = lib.voxtet_paper_cpu(_ptr(x), len(x), _ptr(t), len(t), int(res), {"float": 0, "double": 1}[precision],
                              int(mode), int(n_threads), _ptr(out))
    if st != OK:
        raise OracleError(st)
    return out.reshape(res, res, W)


def paper_cpu_disagreements(xyz: np.ndarray, tets: np.ndarray, res: int, z0: int = 0, z1: Optional[int] = None,
                            n_threads: int = 0) -> dict:
    """Per-test sign-pattern disagreements of Theorem 1 in float / double with exact integers
    over every (tet, sample in its box) pair in slices [z0, z1)."""
    lib = _load()
    x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    c = np.zeros(6, dtype=np.int64)
    st = lib.voxtet_paper_cpu_disagreements(_ptr(x), len(x), _ptr(t), len(t), int(res), int(z0),
                                            int(res if z1 is None else z1), int(n_threads), _ptr(c))
    if st != OK:
        raise OracleError(st)
    keys = ("tests", "exact_closed_inside", "float_closed", "float_strict", "double_closed", "double_strict")
    return {k: int(v) for k, v in zip(keys, c)}


def mismatches(a: np.ndarray, b: np.ndarray) -> Tuple[int, int]:
    """(samples set in a only, samples set in b only) of two bit grids of the same shape."""
    x = np.ascontiguousarray(a, dtype=np.uint32)
    y = np.ascontiguousarray(b, dtype=np.uint32)
    only_a = np.unpackbits((x & ~y).view(np.uint8)).sum()
    only_b = np.unpackbits((y & ~x).view(np.uint8)).sum()
    return int(only_a), int(only_b)


def dense_to_bricks(grid: np.ndarray, rx: int) -> Tuple[np.ndarray, np.ndarray]:
    """Non-empty 32 x 8 x 8 bricks of a bit grid uint32 [rz, ry, W]: (keys uint64 [n], words
    uint32 [n, 64]) in increasing key order, key = bx | by << 16 | bz << 32, word dz * 8 + dy."""
    g = np.ascontiguousarray(grid, dtype=np.uint32)
    rz, ry, W = g.shape
    assert W == (rx + 31) // 32
    nbz, nby = -(-rz // 8), -(-ry // 8)
    pad = np.zeros((nbz * 8, nby * 8, W), dtype=np.uint32)
    pad[:rz, :ry, :] = g
    b = pad.reshape(nbz, 8, nby, 8, W).transpose(0, 2, 4, 1, 3).reshape(nbz, nby, W, 64)
    nz = b.any(axis=3)
    bz, by, bx = np.nonzero(nz)  # row-major order = increasing (bz, by, bx)
    keys = bx.astype(np.uint64) | (by.astype(np.uint64) << np.uint64(16)) | (bz.astype(np.uint64) << np.uint64(32))
    return keys, b[nz]


def bricks_to_dense(keys: np.ndarray, words: np.ndarray, res) -> np.ndarray:
    """Inverse of ``dense_to_bricks`` for a general grid res = (rx, ry, rz)."""
    rx, ry, rz = (int(x) for x in res)
    W = (rx + 31) // 32
    nbz, nby = -(-rz // 8), -(-ry // 8)
    b = np.zeros((nbz, nby, W, 64), dtype=np.uint32)
    k = np.asarray(keys, dtype=np.uint64)
    bx = (k & np.uint64(0xFFFF)).astype(np.int64)
    by = ((k >> np.uint64(16)) & np.uint64(0xFFFF)).astype(np.int64)
    bz = (k >> np.uint64(32)).astype(np.int64)
    b[bz, by, bx] = np.asarray(words, dtype=np.uint32).reshape(-1, 64)
    dense = b.reshape(nbz, nby, W, 8, 8).transpose(0, 3, 1, 4, 2).reshape(nbz * 8, nby * 8, W)
    return np.ascontiguousarray(dense[:rz, :ry, :])


def theorem1_dets(A, B, C, D, P) -> Tuple[int, int, int, int]:
    """(D_a, D_b, D_c, D_d) of Theorem 1 as Python ints, from the C oracle."""
    lib = _load()
    arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.int64).reshape(3)) for x in (A, B, C, D, P)]
    out = np.zeros(8, dtype=np.int64)
    lib.voxtet_oracle_theorem1_dets(*[_ptr(a) for a in arrs], _ptr(out))
    vals = []
    for m in range(4):
        hi, lo = int(out[2 * m]), int(out[2 * m + 1]) & ((1 << 64) - 1)
        vals.append((hi << 64) | lo)
    return tuple(vals)


def num_threads() -> int:
    """Threads a call with n_threads = 0 uses (the OpenMP default; no call changes it)."""
    return int(_load().voxtet_oracle_num_threads())


def last_threads() -> int:
    """Team size the last voxelization (or paper-method) call actually ran with."""
    return int(_load().voxtet_oracle_last_threads())


def unpack(grid: np.ndarray, res: int) -> np.ndarray:
    """Bit grid (uint32 [res, res, W]) -> bool array indexed [l, j, i] (z, y, x)."""
    g = np.ascontiguousarray(grid, dtype=np.uint32).reshape(res, res, -1)
    bits = np.unpackbits(g.view(np.uint8), axis=-1, bitorder="little")
    return bits[..., :res].astype(bool)


def pack(occ: np.ndarray) -> np.ndarray:
    """Inverse of ``unpack``: bool [res, res, res] (z, y, x) -> uint32 [res, res, W]."""
    res = occ.shape[0]
    W = (res + 31) // 32
    pad = np.zeros((res, res, W * 32), dtype=np.uint8)
    pad[..., :res] = occ
    return np.packbits(pad, axis=-1, bitorder="little").view(np.uint32).reshape(res, res, W)
