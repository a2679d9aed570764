"""Serving loop: continuous batching of voxelization requests on one GPU.

Requests (mesh id + resolution) arrive over time.  Meshes live on the device for
the life of the server (uploaded once).  A request is *admitted* when its output
grid fits in a preallocated device arena (admission by HBM footprint) and a
batch slot can take it; admitted requests are grouped into batches and launched
through ``batch.Plan`` objects (CUDA-graph replays), one CUDA stream per plan, so
batches overlap on the device.  Requests that arrive while earlier batches run
are admitted as soon as arena memory and a plan slot free up -- continuous
batching, not a drain-then-refill queue.

Every result is the same grid the request would get alone (the kernels are
exact and a batch is only a different schedule of the same per-job work); the
test suite checks that.
"""
from __future__ import annotations

import bisect
import dataclasses
import time
from typing import Dict, List, Optional, Sequence

from . import batch as vb
from . import voxtet as vt


class Arena:
    """First-fit allocator over one device buffer (offsets in bytes, 256-aligned)."""

    ALIGN = 256

    def __init__(self, nbytes: int, device=None):
        import torch

        self.nbytes = int(nbytes) // self.ALIGN * self.ALIGN
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device or "cuda")
        self._free: List[List[int]] = [[0, self.nbytes]]  # sorted [offset, size]
        self.used = 0
        self.peak = 0

    def alloc(self, nbytes: int) -> Optional[int]:
        need = (int(nbytes) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for k, (off, size) in enumerate(self._free):
            if size >= need:
                if size == need:
                    self._free.pop(k)
                else:
                    self._free[k] = [off + need, size - need]
                self.used += need
                self.peak = max(self.peak, self.used)
                return off
        return None

    def free(self, off: int, nbytes: int) -> None:
        need = (int(nbytes) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        self.used -= need
        k = bisect.bisect_left(self._free, [off, 0])
        self._free.insert(k, [off, need])
        # coalesce with neighbours
        if k + 1 < len(self._free) and self._free[k][0] + self._free[k][1] == self._free[k + 1][0]:
            self._free[k][1] += self._free.pop(k + 1)[1]
        if k > 0 and self._free[k - 1][0] + self._free[k - 1][1] == self._free[k][0]:
            self._free[k - 1][1] += self._free.pop(k)[1]

    def view_grid(self, off: int, res: int):
        w = (res + 31) // 32
        n = res * res * w * 4
        return self.buf[off:off + n].view(dtype=__import__("torch").int32).view(res, res, w)


def grid_bytes(res: int) -> int:
    return res * res * ((res + 31) // 32) * 4


@dataclasses.dataclass
class Ticket:
    rid: int
    mesh_id: int
    res: int
    arrival_s: float
    admitted_s: float = -1.0
    launched_s: float = -1.0
    done_s: float = -1.0
    status: int = 0
    grid_off: int = -1
    slot: int = -1

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclasses.dataclass
class Report:
    tickets: List[Ticket]
    makespan_s: float
    batches: int
    admission_stalls: int
    peak_arena_bytes: int

    def summary(self) -> Dict[str, float]:
        import numpy as np

        lat = np.array([t.latency_s for t in self.tickets]) * 1e3
        ok = sum(1 for t in self.tickets if t.status == vt.OK)
        return {"requests": len(self.tickets), "ok": ok, "jobs_per_s": len(self.tickets) / self.makespan_s,
                "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                "latency_ms_max": float(lat.max()), "makespan_s": self.makespan_s, "batches": self.batches,
                "mean_batch": len(self.tickets) / max(self.batches, 1), "admission_stalls": self.admission_stalls,
                "peak_arena_MiB": self.peak_arena_bytes / 2**20}


class _Slot:
    def __init__(self, ws_bytes: int, max_jobs: int, mode: int):
        import torch

        self.plan = vb.Plan(ws_bytes, max_jobs, mode=mode)
        self.ws_bytes = ws_bytes
        self.stream = torch.cuda.Stream()
        self.tickets: List[Ticket] = []

    @property
    def busy(self) -> bool:
        return bool(self.tickets)


class Server:
    """Continuous-batching voxelization server over device-resident meshes.

    ``meshes``: device meshes (``batch.Mesh``) requests refer to by index.
    ``arena_bytes``: device memory for output grids; a request is admitted only
    when its grid fits.  ``n_slots`` plans (each with ``slot_workspace_bytes`` of
    workspace and its own stream) keep up to that many batches in flight.
    ``on_result(ticket, grid)`` is called for every finished request before its
    grid's memory is reused (copy the grid out there if it is needed later).
    """

    def __init__(self, meshes: Sequence[vb.Mesh], arena_bytes: int, n_slots: int = 3,
                 slot_workspace_bytes: int = 256 << 20, max_jobs: int = 128, mode: int = 0,
                 span_rows_by_res: Optional[Dict[int, int]] = None, on_result=None):
        self.meshes = list(meshes)
        self.arena = Arena(arena_bytes)
        self.max_jobs = int(max_jobs)
        self.slots = [_Slot(slot_workspace_bytes, self.max_jobs, mode) for _ in range(n_slots)]
        self.table_bytes = vb.batch_workspace_size([], self.max_jobs)
        self._slice = {}
        self.span_rows_by_res = dict(span_rows_by_res or {})
        self.on_result = on_result

    def _slice_bytes(self, mesh_id: int, res: int) -> int:
        key = (mesh_id, res)
        if key not in self._slice:
            m = self.meshes[mesh_id]
            self._slice[key] = (vt.workspace_size(m.n_tets, m.n_verts, res) + 255) // 256 * 256
        return self._slice[key]

    def serve(self, requests, realtime: bool = True) -> Report:
        """Serve ``requests`` (objects with rid, arrival_s, mesh_id, res).  With
        ``realtime`` requests become visible at their arrival times; otherwise all
        are visible at once (saturation)."""
        from collections import deque

        reqs = sorted(requests, key=lambda r: r.arrival_s)
        tickets = [Ticket(r.rid, r.mesh_id, r.res, r.arrival_s if realtime else 0.0) for r in reqs]
        n = len(tickets)
        arrived = deque()
        admitted = deque()
        nxt = 0
        finished = 0
        batches = 0
        stalls = 0
        stalled = False
        self.arena.peak = self.arena.used
        t0 = time.perf_counter()
        while finished < n:
            now = time.perf_counter() - t0
            progressed = False
            # completions free arena memory and slots
            for sl in self.slots:
                if sl.busy and sl.plan.done():
                    st = sl.plan.wait()
                    tdone = time.perf_counter() - t0
                    for tk, s in zip(sl.tickets, st):
                        tk.done_s, tk.status = tdone, s
                        if self.on_result is not None:
                            self.on_result(tk, self.arena.view_grid(tk.grid_off, tk.res))
                        self.arena.free(tk.grid_off, grid_bytes(tk.res))
                        finished += 1
                    sl.tickets = []
                    progressed = True
            # arrivals
            while nxt < n and (tickets[nxt].arrival_s <= now):
                arrived.append(tickets[nxt])
                nxt += 1
            # admission by HBM footprint (FIFO)
            while arrived:
                tk = arrived[0]
                off = self.arena.alloc(grid_bytes(tk.res))
                if off is None:
                    if not stalled:
                        stalls += 1
                        stalled = True
                    break
                stalled = False
                tk.grid_off, tk.admitted_s = off, time.perf_counter() - t0
                arrived.popleft()
                admitted.append(tk)
                progressed = True
            # launch admitted work on free slots
            for si, sl in enumerate(self.slots):
                if sl.busy or not admitted:
                    continue
                specs, group, used = [], [], self.table_bytes
                while admitted and len(group) < self.max_jobs:
                    tk = admitted[0]
                    need = self._slice_bytes(tk.mesh_id, tk.res)
                    if group and used + need > sl.ws_bytes:
                        break
                    admitted.popleft()
                    used += need
                    group.append(tk)
                    specs.append(vb.JobSpec(self.meshes[tk.mesh_id], tk.res, self.arena.view_grid(tk.grid_off, tk.res),
                                            span_rows=self.span_rows_by_res.get(tk.res, 0)))
                st = sl.plan.run(specs, stream=sl.stream)
                if st != vt.OK:
                    raise vt.VoxtetError(st, "a single request does not fit a slot's workspace")
                tl = time.perf_counter() - t0
                for tk in group:
                    tk.launched_s, tk.slot = tl, si
                sl.tickets = group
                batches += 1
                progressed = True
            if not progressed:
                idle = not any(sl.busy for sl in self.slots) and not admitted
                if idle and arrived:  # nothing will free memory: the request can never fit
                    raise MemoryError(f"a {arrived[0].res}^3 grid does not fit the arena")
                if nxt < n and idle and not arrived:
                    gap = tickets[nxt].arrival_s - (time.perf_counter() - t0)
                    if gap > 0:
                        time.sleep(min(gap, 0.002))
                else:
                    time.sleep(0)
        makespan = max(t.done_s for t in tickets) - min(t.arrival_s for t in tickets) if n else 0.0
        return Report(tickets, makespan, batches, stalls, self.arena.peak)

    def close(self):
        for sl in self.slots:
            sl.plan.close()
