"""Voxelize a stream of host-resident meshes with the copies overlapped.

Each job is three steps on three CUDA streams: the mesh's pinned-host -> device copy
(``h2d``), the library call (``compute``), and the grid's device -> pinned-host copy
(``d2h``), ordered by events.  ``depth`` device slots (mesh buffers, grid, workspace)
rotate, so while job i computes, job i+1's mesh is on its way in and job i-1's grid
on its way out.  Each job's device-detected status is copied out asynchronously
(``voxtet_status_async``) and checked when the job is collected, so no step waits
on the host.

Host buffers must be pinned (``torch.Tensor.pin_memory()``) for the copies to run
asynchronously, and a job's host buffers must stay untouched until ``wait``.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

from . import voxtet as vt


class _Slot:
    def __init__(self, torch, max_verts: int, max_tets: int, res: int, dev):
        self.verts = torch.empty((max_verts, 3), dtype=torch.float32, device=dev)
        self.tets = torch.empty((max_tets, 4), dtype=torch.int32, device=dev)
        self.grid = vt.alloc_grid(res, dev)
        self.ws = vt.alloc_workspace(max_tets, max_verts, res, dev)
        self.copied_in = torch.cuda.Event()
        self.computed = torch.cuda.Event()
        self.copied_out = torch.cuda.Event()
        self.used = False


class HostPipeline:
    """Pipelined voxelization of host meshes into host grids (cubic 2^k grids of one size).

    ``submit(h_verts, h_tets, h_grid, origin, voxel_size)`` enqueues one job and returns
    at once; ``wait()`` waits for all submitted jobs and raises ``VoxtetError`` for the
    first job whose device-detected status is not OK."""

    def __init__(self, max_verts: int, max_tets: int, res: int, depth: int = 3, device=None, mode: int = 0,
                 span_rows: int = 0, row_cull: int = 0, kernel: int = 0):
        import torch

        self._torch = torch
        dev = torch.device(device or "cuda")
        self.res = int(res)
        self.kw = dict(mode=mode, span_rows=span_rows, row_cull=row_cull, kernel=kernel)
        self.slots = [_Slot(torch, max_verts, max_tets, self.res, dev) for _ in range(max(1, int(depth)))]
        self.h2d = torch.cuda.Stream(device=dev)
        self.compute = torch.cuda.Stream(device=dev)
        self.d2h = torch.cuda.Stream(device=dev)
        self._status = torch.zeros(4096, dtype=torch.int32).pin_memory()
        self._jobs = 0
        self._lib = vt.load()

    def submit(self, h_verts, h_tets, h_grid, origin: Sequence[float], voxel_size: float) -> int:
        """Enqueue one job; returns its index.  h_verts float32 [n, 3], h_tets int32 [m, 4],
        h_grid int32 [res, res, W] (all pinned host tensors)."""
        if self._jobs >= self._status.numel():
            raise RuntimeError("wait() before submitting more than 4096 jobs")
        nv, nt = h_verts.shape[0], h_tets.shape[0]
        s = self.slots[self._jobs % len(self.slots)]
        if nv > s.verts.shape[0] or nt > s.tets.shape[0]:
            raise ValueError("mesh larger than the pipeline's slots")
        if s.used:
            self.h2d.wait_event(s.computed)  # the slot's previous job has consumed its mesh
        with self._torch.cuda.stream(self.h2d):
            s.verts[:nv].copy_(h_verts, non_blocking=True)
            s.tets[:nt].copy_(h_tets, non_blocking=True)
            s.copied_in.record(self.h2d)
        self.compute.wait_event(s.copied_in)
        if s.used:
            self.compute.wait_event(s.copied_out)  # the slot's previous grid has left
        vt.voxelize(s.verts[:nv], s.tets[:nt], origin, voxel_size, self.res, out=s.grid, workspace=s.ws,
                    sync=False, stream=self.compute, **self.kw)
        s.computed.record(self.compute)
        self.d2h.wait_event(s.computed)
        with self._torch.cuda.stream(self.d2h):
            h_grid.copy_(s.grid, non_blocking=True)
            st = self._lib.voxtet_status_async(s.ws.data_ptr(),
                                               ctypes.c_void_p(self._status.data_ptr() + 4 * self._jobs),
                                               ctypes.c_void_p(self.d2h.cuda_stream))
            if st != vt.OK:
                raise vt.VoxtetError(st)
            s.copied_out.record(self.d2h)
        s.used = True
        self._jobs += 1
        return self._jobs - 1

    def wait(self) -> List[int]:
        """Wait for every submitted job; returns their statuses and raises on the first failure."""
        self.d2h.synchronize()
        out = [int(self._lib.voxtet_status_of_word(int(w))) for w in self._status[: self._jobs].tolist()]
        self._jobs = 0
        for i, st in enumerate(out):
            if st != vt.OK:
                raise vt.VoxtetError(st, f"job {i}")
        return out
