"""Autotuner for the voxelizer's launch shape.

The scanline step can distribute its work two ways (``kernel``): spans (a thread walks
whole z-slices of one tet, 512-tet tiles sorted by estimated work; ``span_rows`` sets how
many box rows a span holds) or slice units (one (tet, z-slice) unit per thread, 128-tet
tiles sorted by exact row count).  Both take ``row_cull`` (whether rows outside each
slice's cross-section are skipped).  Their best values depend mostly on the grid
resolution (how many rows a tetrahedron covers), so the tuner times candidates on a
representative mesh per resolution bucket and caches the winner in a JSON file keyed by
device name and resolution.

Every candidate produces the same grid (the tunables only change how work is split), and
the tuner checks that before accepting a result.

Cache location: ``$VOXTET_TUNE_CACHE`` or ``~/.cache/voxtet/tune.json``.
"""
from __future__ import annotations

import json
import os
import statistics
import threading
from typing import Dict, Iterable, Optional, Sequence, Tuple

from . import voxtet as vt

SPAN_CANDIDATES = (64, 128, 256, 512, 1024)
CULL_CANDIDATES = (1, 2)  # 1 = skip rows outside the cross-section, 2 = visit every box row
KERNEL_CANDIDATES = (vt.KERNEL_SPANS, vt.KERNEL_SLICES)
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("VOXTET_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "voxtet",
                                                                  "tune.json")


def _device_key() -> str:
    import torch

    return torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")


def _load_cache() -> Dict[str, dict]:
    p = cache_path()
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(c: Dict[str, dict]) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # a read-only home only loses the cache


def _key(res: int) -> str:
    return f"{_device_key()}/res{int(res)}"


def lookup(res: int) -> Optional[dict]:
    """Cached best settings for this device and resolution, or None."""
    with _lock:
        return _load_cache().get(_key(res))


def time_config(verts, tets, origin, voxel_size, res, span_rows, row_cull, reps=5, workspace=None, out=None,
                kernel=vt.KERNEL_SPANS):
    """Median device time (microseconds) of the main kernel(s) for one setting."""
    import torch

    if workspace is None:
        workspace = vt.alloc_workspace(tets.shape[0], verts.shape[0], res)
    if out is None:
        out = vt.alloc_grid(res)
    kw = dict(out=out, workspace=workspace, span_rows=span_rows, row_cull=row_cull, profile=True, sync=False,
              kernel=kernel)
    vt.voxelize(verts, tets, origin, voxel_size, res, **kw)
    times = []
    for _ in range(reps):
        vt.voxelize(verts, tets, origin, voxel_size, res, **kw)
        times.append(vt.read_stats(workspace)["kernel_ns"] / 1e3)
    torch.cuda.synchronize()
    return statistics.median(times), out


def candidates(spans: Sequence[int] = SPAN_CANDIDATES, culls: Sequence[int] = CULL_CANDIDATES,
               kernels: Sequence[int] = KERNEL_CANDIDATES):
    """(kernel, span_rows, row_cull) settings to time: every span size for the span kernel,
    the span size being irrelevant (0) to slice units."""
    out = []
    for kernel in kernels:
        for cull in culls:
            for span in (spans if kernel == vt.KERNEL_SPANS else (0,)):
                out.append((kernel, span, cull))
    return out


def _label(kernel: int, span: int, cull: int) -> str:
    return f"spans/{span}/{cull}" if kernel == vt.KERNEL_SPANS else f"slices/{cull}"


def tune(verts, tets, origin, voxel_size, res: int, spans: Sequence[int] = SPAN_CANDIDATES,
         culls: Sequence[int] = CULL_CANDIDATES, reps: int = 5, store: bool = True,
         kernels: Sequence[int] = KERNEL_CANDIDATES) -> dict:
    """Time every (kernel, span_rows, row_cull) candidate on this mesh; keep the fastest.

    Returns {"kernel", "span_rows", "row_cull", "us", "table": {label: us}} and, with
    ``store``, records it for the device and resolution."""
    import torch

    ws = vt.alloc_workspace(tets.shape[0], verts.shape[0], res)
    ref = None
    table = {}
    best = None
    for kernel, span, cull in candidates(spans, culls, kernels):
        us, out = time_config(verts, tets, origin, voxel_size, res, span, cull, reps, workspace=ws, kernel=kernel)
        grid = out.clone()
        label = _label(kernel, span, cull)
        if ref is None:
            ref = grid
        elif not torch.equal(grid, ref):
            raise RuntimeError(f"tuning candidate {label} changed the grid")
        table[label] = us
        if best is None or us < best[0]:
            best = (us, kernel, span, cull)
    result = {"kernel": best[1], "span_rows": best[2], "row_cull": best[3], "us": best[0], "table": table,
              "n_tets": int(tets.shape[0])}
    if store:
        with _lock:
            c = _load_cache()
            c[_key(res)] = result
            _store_cache(c)
    return result


def settings_for(res: int) -> Tuple[int, int, int]:
    """(span_rows, row_cull, kernel) to use at this resolution: cached if tuned, else the
    library's automatic choice (0, 0, 0)."""
    hit = lookup(res)
    if hit:
        return int(hit["span_rows"]), int(hit["row_cull"]), int(hit.get("kernel", vt.KERNEL_SPANS))
    return 0, 0, 0


def tune_batch(specs: Iterable, reps: int = 3) -> Dict[int, dict]:
    """Tune each resolution present in a batch on its largest job, then set every
    job's span_rows from the result (jobs are ``batch.JobSpec``)."""
    specs = list(specs)
    by_res: Dict[int, list] = {}
    for sp in specs:
        by_res.setdefault(int(sp.res), []).append(sp)
    out = {}
    for res, group in sorted(by_res.items()):
        big = max(group, key=lambda s: s.mesh.n_tets)
        # batches run the span kernel (one persistent launch over every job's tiles)
        out[res] = tune(big.mesh.verts, big.mesh.tets, big.origin, big.voxel_size, res, culls=(0,), reps=reps,
                        kernels=(vt.KERNEL_SPANS,), store=False)
        for sp in group:
            sp.span_rows = out[res]["span_rows"]
    return out
