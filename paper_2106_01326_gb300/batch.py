"""Batched voxelization: many device-resident meshes in one persistent launch.

Thin wrappers over the batch entry points of include/voxtet.h
(``voxelize_tets_batched`` and the CUDA-graph ``voxtet_plan_*`` calls); all
computation runs in the library.  A ``Mesh`` keeps a mesh's vertices and
tetrahedra on the device so repeated jobs pay no host-to-device copy.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence, Tuple

from . import voxtet as vt


@dataclasses.dataclass
class Mesh:
    """A mesh resident in device memory (float32 verts [n, 3], int32 tets [m, 4])."""
    verts: "object"
    tets: "object"

    @classmethod
    def from_numpy(cls, verts, tets, device="cuda") -> "Mesh":
        import torch

        return cls(torch.as_tensor(verts, dtype=torch.float32).to(device).contiguous(),
                   torch.as_tensor(tets, dtype=torch.int32).to(device).contiguous())

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


@dataclasses.dataclass
class JobSpec:
    mesh: Mesh
    res: int
    out: "object"  # int32 grid tensor [res, res, W]
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    voxel_size: float = 0.0
    span_rows: int = 0

    def __post_init__(self):
        if not self.voxel_size:
            self.voxel_size = 1.0 / self.res


_JOB_DTYPE = None


def _job_dtype():
    """numpy view of ``voxtet.Job`` (the C voxtet_job), field for field at its offsets."""
    global _JOB_DTYPE
    if _JOB_DTYPE is None:
        import numpy as np

        formats = {"d_verts": np.uint64, "n_verts": np.int64, "d_tets": np.uint64, "n_tets": np.int64,
                   "origin": (np.float32, 3), "voxel_size": np.float32, "res": np.int32, "span_rows": np.int32,
                   "fixed_point": np.int32, "reserved": np.int32, "d_out_bits": np.uint64}
        names = [f[0] for f in vt.Job._fields_]
        _JOB_DTYPE = np.dtype({"names": names, "formats": [formats[n] for n in names],
                               "offsets": [getattr(vt.Job, n).offset for n in names],
                               "itemsize": ctypes.sizeof(vt.Job)})
    return _JOB_DTYPE


def make_jobs(specs: Sequence[JobSpec]):
    """The job table of a batch (a ctypes ``voxtet.Job`` array), built in one numpy pass: a
    plan rebuilds it every run, so its cost is part of each batch's latency."""
    import numpy as np

    rows = [(sp.mesh.verts.data_ptr(), sp.mesh.verts.shape[0], sp.mesh.tets.data_ptr(), sp.mesh.tets.shape[0],
             sp.origin, sp.voxel_size, sp.res, sp.span_rows, 0, 0, sp.out.data_ptr()) for sp in specs]
    a = np.array(rows, dtype=_job_dtype()) if rows else np.zeros(1, dtype=_job_dtype())
    return (vt.Job * len(a)).from_buffer(a)  # shares a's memory and keeps it alive


def batch_workspace_size(specs: Sequence[JobSpec], max_jobs: Optional[int] = None) -> int:
    jobs = make_jobs(specs)
    return int(vt.load().voxtet_batch_workspace_size(jobs, len(specs), max_jobs or max(len(specs), 1)))


def voxelize_batched(specs: Sequence[JobSpec], workspace=None, mode: int = 0, use_filter: bool = True,
                     sync: bool = True, stream=None, row_cull: int = 0) -> List[int]:
    """One batched call (no graph).  Returns the per-job status codes."""
    import torch

    lib = vt.load()
    jobs = make_jobs(specs)
    n = len(specs)
    if workspace is None:
        workspace = torch.empty(batch_workspace_size(specs), dtype=torch.uint8, device="cuda")
    st_arr = (ctypes.c_int32 * max(n, 1))()
    o = vt.make_opts(mode, False, use_filter, sync, row_cull=row_cull)
    st = lib.voxelize_tets_batched(jobs, n, workspace.data_ptr(), workspace.numel(), ctypes.byref(o),
                                   vt._stream_ptr(stream), st_arr)
    if st != vt.OK:
        raise vt.VoxtetError(st)
    return [int(st_arr[i]) for i in range(n)]


class Plan:
    """A reusable batch plan (CUDA graph captured on the first run, replayed after).

    One plan runs one batch at a time; keep several plans for batches in flight.
    """

    def __init__(self, workspace_bytes: int, max_jobs: int, mode: int = 0, use_filter: bool = True,
                 device=None, row_cull: int = 0):
        import torch

        self.lib = vt.load()
        self.workspace = torch.empty(int(workspace_bytes), dtype=torch.uint8, device=device or "cuda")
        self.max_jobs = int(max_jobs)
        self._handle = ctypes.c_void_p()
        o = vt.make_opts(mode, False, use_filter, sync=False, row_cull=row_cull)
        st = self.lib.voxtet_plan_create(self.workspace.data_ptr(), self.workspace.numel(), self.max_jobs,
                                         ctypes.byref(o), ctypes.byref(self._handle))
        if st != vt.OK:
            raise vt.VoxtetError(st)
        self._n = 0
        self._jobs = None

    def run(self, specs: Sequence[JobSpec], stream=None) -> int:
        """Enqueue a batch; returns the status (ERR_NOMEM if it does not fit)."""
        self._jobs = make_jobs(specs)  # keep alive until the table is built
        self._n = len(specs)
        return int(self.lib.voxtet_plan_run(self._handle, self._jobs, self._n, vt._stream_ptr(stream)))

    def done(self) -> bool:
        r = int(self.lib.voxtet_plan_query(self._handle))
        if r < 0:
            raise vt.VoxtetError(r)
        return r == 1

    def wait(self) -> List[int]:
        arr = (ctypes.c_int32 * max(self._n, 1))()
        st = self.lib.voxtet_plan_wait(self._handle, arr)
        if st != vt.OK:
            raise vt.VoxtetError(st)
        return [int(arr[i]) for i in range(self._n)]

    def close(self):
        if self._handle:
            self.lib.voxtet_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
