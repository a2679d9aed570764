"""Thin ctypes binding of the C ABI in include/voxtet.h (argument marshalling only).

Every step of the voxelization runs in the CUDA library ``libvoxtet.so``; this
module only turns torch tensors (device memory) and streams into the plain
pointers and sizes the C entry points take.  There is no CPU fallback: if the
library is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvoxtet.so")

OK = 0
ERR_ARG, ERR_RES, ERR_INDEX, ERR_RANGE, ERR_NAN = -1, -2, -3, -4, -5
ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM = -6, -7, -8, -9
MAX_RES = 8192

# every symbol include/voxtet.h declares
EXPORTED = (
    "voxtet_default_opts", "voxtet_workspace_size", "voxelize_tets", "voxelize_tets_fixed", "voxelize_tets_grid",
    "voxtet_last_status", "voxtet_read_stats", "voxtet_strerror", "voxtet_launch_count",
    "voxelize_tets_noalloc", "voxtet_batch_workspace_size", "voxelize_tets_batched", "voxtet_plan_create",
    "voxtet_plan_run", "voxtet_plan_query", "voxtet_plan_wait", "voxtet_plan_destroy",
    "voxtet_sparse_scratch_size", "voxelize_tets_sparse", "voxtet_status_async", "voxtet_status_of_word",
    "voxtet_noalloc_status_async",
)
SPARSE_MAX_SIDE = 65536
BRICK_WORDS = 64
NOALLOC_SCRATCH_BYTES = 16 << 20


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("accumulate", ctypes.c_int32), ("use_filter", ctypes.c_int32),
                ("sync", ctypes.c_int32), ("span_rows", ctypes.c_int32), ("block", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("row_cull", ctypes.c_int32), ("kernel", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("spans", ctypes.c_uint64), ("rows", ctypes.c_uint64), ("fallback_rows", ctypes.c_uint64),
                ("degenerate_tets", ctypes.c_uint64), ("wide_tets", ctypes.c_uint64),
                ("kernel_ns", ctypes.c_uint64), ("exact_tets", ctypes.c_uint64), ("reserved", ctypes.c_uint64)]


class Job(ctypes.Structure):
    _fields_ = [("d_verts", ctypes.c_void_p), ("n_verts", ctypes.c_int64), ("d_tets", ctypes.c_void_p),
                ("n_tets", ctypes.c_int64), ("origin", ctypes.c_float * 3), ("voxel_size", ctypes.c_float),
                ("res", ctypes.c_int32), ("span_rows", ctypes.c_int32), ("fixed_point", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("d_out_bits", ctypes.c_void_p)]


class VoxtetError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"voxtet status {status}: {msg or strerror(status)}")


_lock = threading.Lock()
_lib = None


def load(path: Optional[str] = None):
    """Load (once) and return the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libvoxtet.so not built ({p}); run paper_2106_01326_gb300/build.py")
        lib = ctypes.CDLL(p)
        P, i64, i32, f32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_size_t
        lib.voxtet_default_opts.argtypes = [ctypes.POINTER(Opts)]
        lib.voxtet_default_opts.restype = None
        lib.voxtet_workspace_size.argtypes = [i64, i64, i32]
        lib.voxtet_workspace_size.restype = sz
        lib.voxelize_tets.argtypes = [P, i64, P, i64, ctypes.POINTER(f32 * 3), f32, i32, P, P, sz,
                                      ctypes.POINTER(Opts), P]
        lib.voxelize_tets.restype = ctypes.c_int
        lib.voxelize_tets_fixed.argtypes = [P, i64, P, i64, i32, P, P, sz, ctypes.POINTER(Opts), P]
        lib.voxelize_tets_fixed.restype = ctypes.c_int
        lib.voxelize_tets_grid.argtypes = [P, i64, P, i64, ctypes.POINTER(f32 * 3), f32, ctypes.POINTER(i32 * 3),
                                           i32, i32, P, P, sz, ctypes.POINTER(Opts), P]
        lib.voxelize_tets_grid.restype = ctypes.c_int
        lib.voxtet_status_async.argtypes = [P, P, P]
        lib.voxtet_status_async.restype = ctypes.c_int
        lib.voxtet_status_of_word.argtypes = [i32]
        lib.voxtet_status_of_word.restype = ctypes.c_int
        lib.voxtet_sparse_scratch_size.argtypes = [ctypes.POINTER(i32 * 3), i32]
        lib.voxtet_sparse_scratch_size.restype = sz
        lib.voxelize_tets_sparse.argtypes = [P, i64, P, i64, ctypes.POINTER(f32 * 3), f32, ctypes.POINTER(i32 * 3),
                                             i32, P, P, i64, ctypes.POINTER(i64), P, sz, P, sz,
                                             ctypes.POINTER(Opts), P]
        lib.voxelize_tets_sparse.restype = ctypes.c_int
        lib.voxtet_last_status.argtypes = [P, P]
        lib.voxtet_last_status.restype = ctypes.c_int
        lib.voxtet_read_stats.argtypes = [P, ctypes.POINTER(Stats), P]
        lib.voxtet_read_stats.restype = ctypes.c_int
        lib.voxtet_strerror.argtypes = [ctypes.c_int]
        lib.voxtet_strerror.restype = ctypes.c_char_p
        lib.voxtet_launch_count.argtypes = []
        lib.voxtet_launch_count.restype = ctypes.c_uint64
        lib.voxelize_tets_noalloc.argtypes = [P, i64, P, i64, ctypes.POINTER(f32 * 3), f32, i32, P,
                                              ctypes.POINTER(Opts), P]
        lib.voxelize_tets_noalloc.restype = ctypes.c_int
        lib.voxtet_noalloc_status_async.argtypes = [P, P]
        lib.voxtet_noalloc_status_async.restype = ctypes.c_int
        JP = ctypes.POINTER(Job)
        lib.voxtet_batch_workspace_size.argtypes = [JP, i32, i32]
        lib.voxtet_batch_workspace_size.restype = sz
        lib.voxelize_tets_batched.argtypes = [JP, i32, P, sz, ctypes.POINTER(Opts), P, ctypes.POINTER(i32)]
        lib.voxelize_tets_batched.restype = ctypes.c_int
        lib.voxtet_plan_create.argtypes = [P, sz, i32, ctypes.POINTER(Opts), ctypes.POINTER(P)]
        lib.voxtet_plan_create.restype = ctypes.c_int
        lib.voxtet_plan_run.argtypes = [P, JP, i32, P]
        lib.voxtet_plan_run.restype = ctypes.c_int
        lib.voxtet_plan_query.argtypes = [P]
        lib.voxtet_plan_query.restype = ctypes.c_int
        lib.voxtet_plan_wait.argtypes = [P, ctypes.POINTER(i32)]
        lib.voxtet_plan_wait.restype = ctypes.c_int
        lib.voxtet_plan_destroy.argtypes = [P]
        lib.voxtet_plan_destroy.restype = None
        _lib = lib
        return lib


def strerror(status: int) -> str:
    try:
        return load().voxtet_strerror(int(status)).decode()
    except RuntimeError:
        return "library not loaded"


def launch_count() -> int:
    return int(load().voxtet_launch_count())


def grid_words(res: int) -> int:
    return res * res * ((res + 31) // 32)


def workspace_size(n_tets: int, n_verts: int, res: int) -> int:
    return int(load().voxtet_workspace_size(int(n_tets), int(n_verts), int(res)))


KERNEL_AUTO, KERNEL_SPANS, KERNEL_SLICES = 0, 1, 2


def make_opts(mode: int = 0, accumulate: bool = False, use_filter: bool = True, sync: bool = True,
              span_rows: int = 0, block: int = 0, profile: bool = False, row_cull: int = 0,
              kernel: int = 0) -> Opts:
    o = Opts()
    load().voxtet_default_opts(ctypes.byref(o))
    o.mode, o.accumulate, o.use_filter, o.sync = int(mode), int(bool(accumulate)), int(bool(use_filter)), int(bool(sync))
    o.span_rows, o.block, o.profile, o.row_cull = int(span_rows), int(block), int(bool(profile)), int(row_cull)
    o.kernel = int(kernel)
    return o


def _torch():
    import torch

    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check_cuda_tensor(t, name: str, dtype):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def alloc_grid(res: int, device=None):
    """A grid buffer (int32 storage holding the uint32 bit words), shape [res, res, W]."""
    torch = _torch()
    return torch.empty((res, res, (res + 31) // 32), dtype=torch.int32, device=device or "cuda")


def alloc_workspace(n_tets: int, n_verts: int, res: int, device=None):
    torch = _torch()
    return torch.empty(workspace_size(n_tets, n_verts, res), dtype=torch.uint8, device=device or "cuda")


def voxelize(verts, tets, origin: Sequence[float], voxel_size: float, res: int, out=None, workspace=None,
             mode: int = 0, accumulate: bool = False, use_filter: bool = True, sync: bool = True,
             span_rows: int = 0, stream=None, raise_on_error: bool = True, profile: bool = False,
             row_cull: int = 0, kernel: int = 0):
    """Grid (int32 tensor [res, res, W] of uint32 bit words) of a world-space mesh.

    verts: float32 CUDA [n_verts, 3]; tets: int32 CUDA [n_tets, 4].  Returns ``out``
    (or (status, out) when ``raise_on_error`` is False).
    """
    torch = _torch()
    lib = load()
    _check_cuda_tensor(verts, "verts", torch.float32)
    _check_cuda_tensor(tets, "tets", torch.int32)
    n_v, n_t = verts.shape[0], tets.shape[0]
    if out is None:
        out = alloc_grid(res, verts.device)
    _check_cuda_tensor(out, "out", torch.int32)
    if workspace is None:
        workspace = alloc_workspace(n_t, n_v, res, verts.device)
    o = make_opts(mode, accumulate, use_filter, sync, span_rows, profile=profile, row_cull=row_cull, kernel=kernel)
    org = (ctypes.c_float * 3)(*[float(x) for x in origin])
    st = lib.voxelize_tets(verts.data_ptr(), n_v, tets.data_ptr(), n_t, ctypes.byref(org), float(voxel_size),
                           int(res), out.data_ptr(), workspace.data_ptr(), workspace.numel(), ctypes.byref(o),
                           _stream_ptr(stream))
    if raise_on_error:
        if st != OK:
            raise VoxtetError(st)
        return out
    return st, out


def voxelize_fixed(xyz, tets, res: int, out=None, workspace=None, mode: int = 0, accumulate: bool = False,
                   use_filter: bool = True, sync: bool = True, span_rows: int = 0, stream=None,
                   raise_on_error: bool = True, profile: bool = False, row_cull: int = 0, kernel: int = 0):
    """Grid of a mesh whose vertices are already on the 2^20-per-grid lattice (int32 [n, 3])."""
    torch = _torch()
    lib = load()
    _check_cuda_tensor(xyz, "xyz", torch.int32)
    _check_cuda_tensor(tets, "tets", torch.int32)
    n_v, n_t = xyz.shape[0], tets.shape[0]
    if out is None:
        out = alloc_grid(res, xyz.device)
    _check_cuda_tensor(out, "out", torch.int32)
    if workspace is None:
        workspace = alloc_workspace(n_t, n_v, res, xyz.device)
    o = make_opts(mode, accumulate, use_filter, sync, span_rows, profile=profile, row_cull=row_cull, kernel=kernel)
    st = lib.voxelize_tets_fixed(xyz.data_ptr(), n_v, tets.data_ptr(), n_t, int(res), out.data_ptr(),
                                 workspace.data_ptr(), workspace.numel(), ctypes.byref(o), _stream_ptr(stream))
    if raise_on_error:
        if st != OK:
            raise VoxtetError(st)
        return out
    return st, out


def alloc_grid_dims(res3: Sequence[int], z_range: Optional[Tuple[int, int]] = None, device=None):
    """Buffer for a general grid or slab: int32 [z_end - z_begin, ry, ceil(rx / 32)]."""
    torch = _torch()
    rx, ry, rz = (int(x) for x in res3)
    z0, z1 = (0, rz) if z_range is None else (int(z_range[0]), int(z_range[1]))
    return torch.empty((max(z1 - z0, 0), ry, (rx + 31) // 32), dtype=torch.int32, device=device or "cuda")


def voxelize_grid(verts, tets, origin: Sequence[float], voxel_size: float, res3: Sequence[int],
                  z_range: Optional[Tuple[int, int]] = None, out=None, workspace=None, mode: int = 0,
                  accumulate: bool = False, use_filter: bool = True, sync: bool = True, span_rows: int = 0,
                  stream=None, raise_on_error: bool = True, profile: bool = False, row_cull: int = 0,
                  kernel: int = 0):
    """General grid res3 = (rx, ry, rz), any sides in [1, MAX_RES], or its z-slab
    ``z_range`` = (z_begin, z_end): int32 tensor [z_end - z_begin, ry, ceil(rx / 32)]."""
    torch = _torch()
    lib = load()
    _check_cuda_tensor(verts, "verts", torch.float32)
    _check_cuda_tensor(tets, "tets", torch.int32)
    n_v, n_t = verts.shape[0], tets.shape[0]
    rx, ry, rz = (int(x) for x in res3)
    z0, z1 = (0, rz) if z_range is None else (int(z_range[0]), int(z_range[1]))
    if out is None:
        out = alloc_grid_dims(res3, (z0, z1), verts.device)  # an empty slab passes a NULL pointer
    _check_cuda_tensor(out, "out", torch.int32)
    if workspace is None:
        workspace = alloc_workspace(n_t, n_v, max(int(x) for x in res3), verts.device)
    o = make_opts(mode, accumulate, use_filter, sync, span_rows, profile=profile, row_cull=row_cull, kernel=kernel)
    org = (ctypes.c_float * 3)(*[float(x) for x in origin])
    r3 = (ctypes.c_int32 * 3)(rx, ry, rz)
    st = lib.voxelize_tets_grid(verts.data_ptr(), n_v, tets.data_ptr(), n_t, ctypes.byref(org), float(voxel_size),
                                ctypes.byref(r3), z0, z1, out.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                ctypes.byref(o), _stream_ptr(stream))
    if raise_on_error:
        if st != OK:
            raise VoxtetError(st)
        return out
    return st, out


def sparse_scratch_size(res3: Sequence[int], slab_depth: int) -> int:
    r3 = (ctypes.c_int32 * 3)(*[int(x) for x in res3])
    return int(load().voxtet_sparse_scratch_size(ctypes.byref(r3), int(slab_depth)))


def default_slab_depth(res3: Sequence[int], budget_bytes: int = 128 << 20) -> int:
    """Slices per pass so that one dense slab stays within ``budget_bytes`` (a multiple of 8).

    The default keeps a slab about the size of GB300's 129 MB L2, so that zeroing it, the ORs into
    it and the brick count and compaction that read it back mostly stay in L2 instead of HBM
    (torus_73: 4096^3 13.8 -> 11.4 ms, 8192^3 100 -> 77 ms against 2 GiB slabs)."""
    rx, ry, rz = (int(x) for x in res3)
    per_slice = ry * ((rx + 31) // 32) * 4
    fit = budget_bytes // max(per_slice, 1)
    if fit >= rz:  # the whole grid in one slab (rounded up: the last slab is cut at rz)
        return (rz + 7) // 8 * 8
    return max(8, fit // 8 * 8)


def voxelize_sparse(verts, tets, origin: Sequence[float], voxel_size: float, res3: Sequence[int],
                    slab_depth: int = 0, max_bricks: Optional[int] = None, workspace=None, scratch=None,
                    mode: int = 0, use_filter: bool = True, span_rows: int = 0, row_cull: int = 0, stream=None,
                    kernel: int = 0):
    """Brick-sparse grid: (keys int64 [n], words int32 [n, 64]) of the non-empty 32 x 8 x 8 bricks,
    keys bx | by << 16 | bz << 32 in increasing order.  Grows the output and retries once if
    ``max_bricks`` is too small."""
    torch = _torch()
    lib = load()
    _check_cuda_tensor(verts, "verts", torch.float32)
    _check_cuda_tensor(tets, "tets", torch.int32)
    dev = verts.device
    n_v, n_t = verts.shape[0], tets.shape[0]
    r3 = (ctypes.c_int32 * 3)(*[int(x) for x in res3])
    depth = int(slab_depth) or default_slab_depth(res3)
    if scratch is None:
        scratch = torch.empty(max(sparse_scratch_size(res3, depth), 256), dtype=torch.uint8, device=dev)
    if workspace is None:
        workspace = alloc_workspace(n_t, n_v, max(int(x) for x in res3), dev)
    if max_bricks is None:
        rx, ry, rz = (int(x) for x in res3)
        max_bricks = min(((rx + 31) // 32) * ((ry + 7) // 8) * ((rz + 7) // 8), 1 << 20)
    o = make_opts(mode, False, use_filter, True, span_rows, row_cull=row_cull, kernel=kernel)
    org = (ctypes.c_float * 3)(*[float(x) for x in origin])
    for attempt in range(2):
        keys = torch.empty(max(int(max_bricks), 1), dtype=torch.int64, device=dev)
        words = torch.empty((max(int(max_bricks), 1), BRICK_WORDS), dtype=torch.int32, device=dev)
        n = ctypes.c_int64(0)
        st = lib.voxelize_tets_sparse(verts.data_ptr(), n_v, tets.data_ptr(), n_t, ctypes.byref(org),
                                      float(voxel_size), ctypes.byref(r3), depth, keys.data_ptr(), words.data_ptr(),
                                      int(max_bricks), ctypes.byref(n), scratch.data_ptr(), scratch.numel(),
                                      workspace.data_ptr(), workspace.numel(), ctypes.byref(o), _stream_ptr(stream))
        if st == ERR_NOMEM and attempt == 0:
            max_bricks = int(n.value)
            continue
        if st != OK:
            raise VoxtetError(st)
        return keys[: n.value], words[: n.value]
    raise VoxtetError(ERR_NOMEM)


def last_status(workspace, stream=None) -> int:
    return int(load().voxtet_last_status(workspace.data_ptr(), _stream_ptr(stream)))


def read_stats(workspace, stream=None) -> dict:
    s = Stats()
    st = load().voxtet_read_stats(workspace.data_ptr(), ctypes.byref(s), _stream_ptr(stream))
    if st != OK:
        raise VoxtetError(st)
    return {"spans": s.spans, "rows": s.rows, "fallback_rows": s.fallback_rows,
            "degenerate_tets": s.degenerate_tets, "wide_tets": s.wide_tets, "kernel_ns": s.kernel_ns,
            "exact_tets": s.exact_tets}


def voxelize_noalloc(verts, tets, origin: Sequence[float], voxel_size: float, res: int, out, mode: int = 0,
                     use_filter: bool = True, sync: bool = True, stream=None) -> int:
    """Voxelize into ``out`` using the library's fixed device scratch instead of a
    workspace, for callers that cannot allocate device memory when they call (a host
    application that owns the device-memory budget, a loop that must not enter the
    allocator; see voxelize_tets_noalloc in include/voxtet.h).  ``out`` must be
    preallocated; returns the status code (with ``sync`` False, the device-detected
    part comes from ``noalloc_status_async``)."""
    torch = _torch()
    lib = load()
    _check_cuda_tensor(verts, "verts", torch.float32)
    _check_cuda_tensor(tets, "tets", torch.int32)
    _check_cuda_tensor(out, "out", torch.int32)
    o = make_opts(mode, False, use_filter, sync)
    org = (ctypes.c_float * 3)(*[float(x) for x in origin])
    return int(lib.voxelize_tets_noalloc(verts.data_ptr(), verts.shape[0], tets.data_ptr(), tets.shape[0],
                                         ctypes.byref(org), float(voxel_size), int(res), out.data_ptr(),
                                         ctypes.byref(o), _stream_ptr(stream)))


def noalloc_status_async(status_word, stream=None) -> int:
    """Enqueue a copy of the last voxelize_noalloc call's status word into ``status_word``
    (a one-element int32 tensor, pinned host or device) without synchronizing; read it with
    ``status_of_word`` once the stream has passed.  Returns the enqueue status."""
    torch = _torch()
    if not isinstance(status_word, torch.Tensor) or status_word.dtype != torch.int32 or status_word.numel() < 1:
        raise TypeError("status_word must be an int32 tensor with at least one element")
    return int(load().voxtet_noalloc_status_async(status_word.data_ptr(), _stream_ptr(stream)))


def status_of_word(word: int) -> int:
    return int(load().voxtet_status_of_word(int(word)))
