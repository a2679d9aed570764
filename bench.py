#!/usr/bin/env python
"""Benchmark: solid voxelization of the 1.3M-tet sliver mesh into a 512^3 bit grid.

One step = one full voxelization (snap + fused tile/scan/scanline/OR kernel,
grid cleared first) of the workload through the C ABI, inputs resident in HBM.
Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded z-slab of the same workload instead.

Multi-GPU: every rank voxelizes its own copy of the mesh (independent jobs, no
collective on the data path); value = tets of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxelized tets/s at 512^3 (bit-exact)"
UNIT = "tets/s"
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sliver_60")
    ap.add_argument("--span-rows", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0, help="scanline work distribution: 0 auto, 1 spans, 2 slice units")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slab", type=int, default=128, help="z-slices in the CPU oracle sample")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-mesh batched comparison")
    ap.add_argument("--no-served", action="store_true", help="skip the served (continuous batching) run")
    ap.add_argument("--no-sparse", action="store_true", help="skip the brick-sparse output run")
    ap.add_argument("--no-slabs", action="store_true", help="skip the one-GPU estimate of z-slab strong scaling")
    ap.add_argument("--requests", type=int, default=10000, help="requests in the served run")
    ap.add_argument("--partition", choices=["replica", "slab"], default="replica",
                    help="N > 1: a replica of the whole job per rank (weak scaling), or one z-slab of the same "
                         "grid per rank (strong scaling, no exchange)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value_ms: float, dist=None, device=None) -> float:
    """The largest per-rank time (the job takes as long as its slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value_ms)
    import torch

    t = torch.tensor([float(value_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, steps: int, total_ms_max: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return world * units_per_rank * steps / (total_ms_max / 1000.0)


def kernel_source_digest() -> str:
    """SHA-256 over the CUDA sources; a recorded ncu traffic figure is valid only for it."""
    import hashlib

    h = hashlib.sha256()
    for name in ("voxtet.cu", "voxtet_slices.cu", "voxtet_device.cuh", "voxtet_slices.cuh", "tet_math.cuh"):
        with open(os.path.join(ROOT, "paper_2106_01326_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(workload: str, kernel: str = "k_voxelize"):
    """DRAM bytes per launch of the main kernel from profiles/<kernel>_traffic.txt (one ncu
    capture of this benchmark's command), or None if it was taken on other sources or
    another workload."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    try:
        kv = {}
        with open(p) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != kernel_source_digest() or kv.get("workload") != workload:
            return None
        return int(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# Algorithmic ALU work per unit: 25 lane-ops per candidate x-row (four affine bounds, their
# rounding and certification, the word mask) and 150 per tetrahedron (box, orientation,
# face data), the minimum counts of the operations the method needs per unit.
ALU_OPS_PER_ROW = 25
ALU_OPS_PER_TET = 150


def alu_roofline(rows: int, tets: int, kernel_ms: float, rows_with_samples=None) -> dict:
    """The main kernel against the FP32/INT32 lane throughput (152 SMs x 128 lanes x
    the maximum SM clock), the bound that actually limits it.  The per-row work is counted
    on the rows that hold a sample when that count is known (the oracle counts them: no
    method can do less), else on the candidate rows the kernel visited (an upper bound)."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    peak = 152 * 128 * mhz * 1e6 / 1e12
    unit_rows = rows if rows_with_samples is None else int(rows_with_samples)
    ops = ALU_OPS_PER_ROW * unit_rows + ALU_OPS_PER_TET * tets
    achieved = ops / (kernel_ms / 1000.0) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s", "frac": achieved / peak,
            "algorithmic_ops": ops, "ops_per_row": ALU_OPS_PER_ROW, "ops_per_tet": ALU_OPS_PER_TET,
            "rows_counted": "rows holding a sample (oracle)" if rows_with_samples is not None
            else "candidate rows visited (kernel)", "rows_candidate": int(rows),
            "rows_with_samples": None if rows_with_samples is None else int(rows_with_samples),
            "peak_source": f"152 SMs x 128 lanes x {mhz:.0f} MHz"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(cfg, slab, n_threads=0):
    """The oracle (as it stands) on z-slab [res/2 - slab/2, res/2 + slab/2) of the workload."""
    import oracle

    res = cfg["res"]
    st, xyz = oracle.snap(cfg["verts"], cfg["origin"], cfg["voxel_size"], res)
    assert st == 0
    z0 = max(0, res // 2 - slab // 2)
    z1 = min(res, z0 + slab)
    t0 = time.perf_counter()
    oracle.voxelize_fixed_slab(xyz, cfg["tets"], res, z0, z1, n_threads=n_threads)
    dt = time.perf_counter() - t0
    frac = (z1 - z0) / res
    value = len(cfg["tets"]) * frac / dt
    return value, dt, (z1 - z0), oracle.num_threads() if n_threads <= 0 else n_threads


def oracle_whole_grid(cfg):
    """The oracle's grid of the whole workload (all host cores), with its time, the threads it
    ran with and its counts (rows holding a sample: the per-row work the method cannot avoid)."""
    import oracle

    res = cfg["res"]
    st, xyz = oracle.snap(cfg["verts"], cfg["origin"], cfg["voxel_size"], res)
    assert st == 0
    t0 = time.perf_counter()
    exact, stats = oracle.voxelize_fixed(xyz, cfg["tets"], res, with_stats=True)
    return exact, xyz, {"s": time.perf_counter() - t0, "threads": oracle.last_threads(), **stats}


def paper_cpu_comparison(cfg, exact, xyz, exact_info):
    """The paper's CPU method in float and double (oracle/paper_cpu.c) on the same snapped mesh:
    whole-grid mismatches against the exact oracle, per-test sign disagreements on the middle
    128 slices, and the same on a tie-heavy soup (faces on planes through samples).  Every time
    carries the threads it ran with."""
    import oracle
    from paper_2106_01326_gb300 import meshgen as mg

    res = cfg["res"]
    out = {"what": "Theorem 1 in binary floating point on the oracle's snapped inputs (not exact)",
           "exact_oracle_s": exact_info["s"], "exact_oracle_threads": exact_info["threads"]}
    for prec in ("float", "double"):
        t0 = time.perf_counter()
        g = oracle.paper_cpu(xyz, cfg["tets"], res, prec, 0)
        out[f"{prec}_s"] = time.perf_counter() - t0
        out[f"{prec}_threads"] = oracle.last_threads()
        extra, missing = oracle.mismatches(g, exact)
        out[f"{prec}_grid_mismatches"] = {"extra": extra, "missing": missing}
    z0 = max(0, res // 2 - 64)
    out["per_test_disagreements_middle_128_slices"] = oracle.paper_cpu_disagreements(xyz, cfg["tets"], res, z0,
                                                                                     min(res, z0 + 128))
    sx, stt = mg.coplanar_face_soup(400, 64, seed=124, spread=60)
    out["per_test_disagreements_coplanar_soup_64"] = oracle.paper_cpu_disagreements(sx, stt, 64)
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2106_01326_gb300 import meshgen as mg
    import oracle

    oracle.build()
    cfg = mg.single_mesh_config(args.workload)
    for _ in range(args.warmup):
        cpu_oracle_sample(cfg, args.slab)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, depth, cores = cpu_oracle_sample(cfg, args.slab)
        vals.append(v)
        secs.append(dt)
    res = cfg["res"]
    total = sum(secs)
    value = len(cfg["tets"]) * (depth / res) * args.steps / total
    sample = (f"z-slab of {depth} of {res} slices (all tets overlapping it) per step; "
              f"tets/s = n_tets x {depth}/{res} / step time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i128",
        "data": "synthetic", "config": {"workload": f"{args.workload} ({len(cfg['tets'])} tets) -> {res}^3"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_section(args, flush, stream):
    """256 meshes (1k-100k tets, grids 32^3-128^3) as one graph-replayed batch vs one
    call per mesh on the same stream: jobs/s, per-job completion latency, exactness."""
    import numpy as np
    import torch

    from paper_2106_01326_gb300 import batch
    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import voxtet as vt

    jobs = mg.batch_workload()
    specs, ref_out = [], []
    for j in jobs:
        m = batch.Mesh.from_numpy(j.verts, j.tets)
        specs.append(batch.JobSpec(m, j.res, vt.alloc_grid(j.res), j.origin, j.voxel_size))
        ref_out.append(vt.alloc_grid(j.res))
    n_tets = sum(len(j.tets) for j in jobs)
    from paper_2106_01326_gb300 import autotune

    tuned = autotune.tune_batch(specs, reps=2)  # per-resolution span size, untimed
    plan = batch.Plan(batch.batch_workspace_size(specs, len(specs)), len(specs))
    ws_single = [vt.alloc_workspace(sp.mesh.n_tets, sp.mesh.n_verts, sp.res) for sp in specs]

    def run_batch():
        st = plan.run(specs, stream=stream)
        if st != vt.OK:
            raise vt.VoxtetError(st)

    def run_single(events=None):
        for i, sp in enumerate(specs):
            vt.voxelize(sp.mesh.verts, sp.mesh.tets, sp.origin, sp.voxel_size, sp.res, out=ref_out[i],
                        workspace=ws_single[i], sync=False, stream=stream, span_rows=sp.span_rows)
            if events is not None:
                events[i].record(stream)

    for _ in range(3):
        run_batch()
        run_single()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b_ms, s_ms, s_lat = [], [], []
    ev = [torch.cuda.Event(enable_timing=True) for _ in specs]
    l0 = vt.launch_count()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0.record(stream)
        run_batch()
        e1.record(stream)
        e1.synchronize()
        b_ms.append(e0.elapsed_time(e1))
    launches_batch = (vt.launch_count() - l0) // max(args.steps, 1)
    status = plan.wait()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0.record(stream)
        run_single(ev)
        e1.record(stream)
        e1.synchronize()
        s_ms.append(e0.elapsed_time(e1))
        s_lat.extend(e0.elapsed_time(e) for e in ev)
    torch.cuda.synchronize()
    exact = all(bool(torch.equal(sp.out, r)) for sp, r in zip(specs, ref_out)) and status == [vt.OK] * len(specs)
    plan.close()
    # every job's batched grid against the oracle's grid of the same mesh and resolution
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    oracle_ok = 0
    for j, sp in zip(jobs, specs):
        ref = oracle.voxelize(j.verts, j.tets, j.origin, j.voxel_size, j.res)
        oracle_ok += int(np.array_equal(sp.out.cpu().numpy().view(np.uint32), ref))
    oracle_s = time.perf_counter() - t0
    bmean, smean = statistics.mean(b_ms), statistics.mean(s_ms)
    q = lambda xs, f: float(np.percentile(np.asarray(xs), f))
    return {
        "workload": f"256 meshes, {n_tets} tets (log-uniform 1k-100k per mesh), grids 32^3/64^3/128^3",
        # every job of a replay is submitted with it and its grid is final when the replay's last
        # kernel (the exact one, which serves all jobs) ends: each job's latency is its replay's
        # duration, measured per replay
        "batched": {"jobs_per_s": len(specs) / (bmean / 1e3), "tets_per_s": n_tets / (bmean / 1e3),
                    "ms_per_batch": bmean, "latency_ms_p50": q(b_ms, 50), "latency_ms_p99": q(b_ms, 99),
                    "latency_samples": len(b_ms) * len(specs),
                    "launches_per_batch": int(launches_batch), "form": "one CUDA-graph replay"},
        "per_mesh": {"jobs_per_s": len(specs) / (smean / 1e3), "tets_per_s": n_tets / (smean / 1e3),
                     "ms_per_batch": smean, "latency_ms_p50": q(s_lat, 50), "latency_ms_p99": q(s_lat, 99),
                     "form": "256 voxelize_tets calls on one stream"},
        "speedup_jobs_per_s": smean / bmean,
        "span_rows_by_res": {str(r): v["span_rows"] for r, v in tuned.items()},
        "bit_identical": exact,
        "oracle_exact": f"{oracle_ok}/{len(specs)}", "oracle_s": oracle_s, "oracle_threads": oracle.last_threads(),
    }


def sparse_section(stream):
    """Brick-sparse output of torus_73 (198,549 tets) at 4096^3 and 8192^3: time, bricks and
    bytes against the dense grid's; at 4096^3 the bricks are scattered back on the device and
    compared bit for bit with the dense path's grid."""
    import torch

    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import voxtet as vt

    cfg = mg.single_mesh_config("torus_73")
    verts = torch.from_numpy(cfg["verts"]).cuda()
    tets = torch.from_numpy(cfg["tets"]).cuda()
    n_t, n_v = len(cfg["tets"]), len(cfg["verts"])
    out = {"workload": f"torus_73: {n_t} tets (torus R=0.3, r=0.12 clipped from a 73^3 jittered Kuhn lattice)"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for res in (4096, 8192):
        res3 = (res, res, res)
        ws = vt.alloc_workspace(n_t, n_v, res)
        depth = vt.default_slab_depth(res3)
        scratch = torch.empty(vt.sparse_scratch_size(res3, depth), dtype=torch.uint8, device="cuda")
        keys, words = vt.voxelize_sparse(verts, tets, (0, 0, 0), 1.0 / res, res3, slab_depth=depth, workspace=ws,
                                         scratch=scratch, stream=stream)
        cap = int(len(keys))
        times = []
        for _ in range(3):
            e0.record(stream)
            keys, words = vt.voxelize_sparse(verts, tets, (0, 0, 0), 1.0 / res, res3, slab_depth=depth,
                                             max_bricks=cap, workspace=ws, scratch=scratch, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        n_b = int(len(keys))
        total_b = (res // 32) * (res // 8) * (res // 8)
        entry = {"ms": ms, "tets_per_s": n_t / (ms / 1000.0), "gvox_per_s": res ** 3 / (ms / 1000.0) / 1e9,
                 "slab_depth": depth, "slabs": -(-res // depth), "bricks": n_b, "bricks_fraction": n_b / total_b,
                 "sparse_bytes": n_b * (8 + 4 * vt.BRICK_WORDS), "dense_bytes": res ** 3 // 8}
        if res == 4096:
            dense = vt.voxelize(verts, tets, (0, 0, 0), 1.0 / res, res, workspace=ws, stream=stream)
            W = res // 32
            b = dense.view(res // 8, 8, res // 8, 8, W).permute(0, 2, 4, 1, 3).reshape(-1, vt.BRICK_WORDS)
            k = keys.view(torch.int64)
            lin = ((k >> 32) * (res // 8) + ((k >> 16) & 0xFFFF)) * W + (k & 0xFFFF)
            nonempty = b.ne(0).any(dim=1)
            entry["bit_identical_to_dense"] = bool(int(nonempty.sum()) == n_b and torch.equal(b[lin], words))
            del dense, b
        entry["uncertain_rows_last_slab"] = int(vt.read_stats(ws)["fallback_rows"])
        out[f"{res}^3"] = entry
        del scratch, keys, words, ws
        torch.cuda.empty_cache()
    return out


def slab_section(verts, tets, cfg, span_rows, row_cull, stream, kernel=0):
    """The benchmark grid cut into 2, 4 and 8 weighted z-slabs (slabs.slab_cuts over the tets per
    slice), each slab voxelized from the tets that can reach it (slabs.tets_for_slab) and timed
    alone on this GPU: the slowest slab against the whole grid estimates the strong scaling of one
    slab per GPU, since ranks exchange nothing."""
    import torch

    from paper_2106_01326_gb300 import slabs
    from paper_2106_01326_gb300 import voxtet as vt

    res = cfg["res"]
    n_t, n_v = len(cfg["tets"]), len(cfg["verts"])
    ws = vt.alloc_workspace(n_t, n_v, res)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    full = vt.alloc_grid(res)
    full_ms = timed(lambda: vt.voxelize(verts, tets, cfg["origin"], cfg["voxel_size"], res, out=full, workspace=ws,
                                        sync=False, span_rows=span_rows, row_cull=row_cull, stream=stream,
                                        kernel=kernel))
    w = slabs.slice_weights(cfg["verts"], cfg["tets"], cfg["origin"], cfg["voxel_size"], res)
    out = {"whole_grid_ms": full_ms}
    for n in (2, 4, 8):
        times, parts, n_sub = [], [], []
        for z0, z1 in slabs.slab_cuts(res, n, w):
            g = vt.alloc_grid_dims((res, res, res), (z0, z1))
            # the rank's tets and only the vertices they name (chosen once per mesh on the host, not
            # timed), so the rank snaps its own vertices only
            sv, st = slabs.slab_mesh(cfg["verts"], cfg["tets"], cfg["origin"], cfg["voxel_size"], z0, z1)
            sub = torch.from_numpy(st).to(tets.device)
            subv = torch.from_numpy(sv).to(tets.device)
            n_sub.append(int(sub.shape[0]))
            times.append(timed(lambda g=g, z0=z0, z1=z1, sub=sub, subv=subv: vt.voxelize_grid(
                subv, sub, cfg["origin"], cfg["voxel_size"], (res, res, res), z_range=(z0, z1), out=g,
                workspace=ws, sync=False, span_rows=span_rows, row_cull=row_cull, stream=stream, kernel=kernel)))
            parts.append(g)
        same = bool(torch.equal(torch.cat(parts, dim=0), full))
        out[f"{n}_slabs"] = {"slab_ms": [round(t, 4) for t in times], "max_slab_ms": max(times), "tets_per_slab": n_sub,
                             "strong_scaling_estimate": full_ms / (n * max(times)), "concatenation_equals_grid": same}
        del parts
    return out


def served_section(args):
    """Continuous batching of a Poisson request stream over a pool of 16 device-resident
    meshes (1k-2M tets, log-uniform) at 64^3-512^3: capacity (all requests queued at
    once) and latency at 80% of that rate; every 25th result is checked bit for bit
    against the same request voxelized alone."""
    import torch

    from paper_2106_01326_gb300 import batch, server
    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import voxtet as vt

    host_pool = mg.mesh_pool(16, seed=1004, tets_lo=1000, tets_hi=2000000)
    pool = [batch.Mesh.from_numpy(v, t) for v, t in host_pool]
    res_set = (64, 128, 256, 512)
    alone = {}
    checked = [0, 0]

    def check(tk, grid):
        if tk.rid % 25:
            return
        key = (tk.mesh_id, tk.res)
        if key not in alone:
            m = pool[tk.mesh_id]
            alone[key] = vt.voxelize(m.verts, m.tets, (0, 0, 0), 1.0 / tk.res, tk.res)
        checked[0] += 1
        checked[1] += int(torch.equal(grid, alone[key]))

    def make_server():
        return server.Server(pool, arena_bytes=4 << 30, n_slots=3, slot_workspace_bytes=512 << 20, max_jobs=64,
                             on_result=check)

    n = args.requests
    sat_reqs = mg.poisson_stream(n, rate_per_s=1.0, n_pool=len(pool), seed=1004, resolutions=res_set)
    srv = make_server()
    srv.serve(sat_reqs[: min(n, 200)], realtime=False)  # warm-up: graph capture, first launches
    torch.cuda.synchronize()
    cap = srv.serve(sat_reqs, realtime=False).summary()
    rate = 0.8 * cap["jobs_per_s"]
    reqs = mg.poisson_stream(n, rate_per_s=rate, n_pool=len(pool), seed=1004, resolutions=res_set)
    rt = srv.serve(reqs, realtime=True).summary()
    srv.close()
    verified = served_oracle_check(pool, host_pool, sat_reqs, res_set)
    return {"workload": f"{n} Poisson requests over 16 pooled meshes ({sum(m.n_tets for m in pool)} tets), "
                        f"grids {res_set}", "capacity": cap, "poisson_at_0.8_capacity": dict(rt, rate_per_s=rate),
            "sampled_exact": f"{checked[1]}/{checked[0]}", "sampled_oracle_exact": verified, "slots": 3,
            "arena_GiB": 4}


def served_oracle_check(pool, host_pool, reqs, res_set, n_check=400):
    """The first ``n_check`` requests of the saturated stream plus the pool's largest mesh at the
    finest grid and its smallest at the coarsest, served again (untimed) through the same
    continuous-batching server, each result compared bit for bit with the oracle's grid."""
    import numpy as np
    import torch

    import oracle
    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import server

    oracle.build()
    sizes = [len(t) for _, t in host_pool]
    sub = list(reqs[:n_check])
    last = sub[-1].arrival_s
    sub.append(mg.Request(len(reqs), last, int(np.argmax(sizes)), max(res_set)))
    sub.append(mg.Request(len(reqs) + 1, last, int(np.argmin(sizes)), min(res_set)))
    ref = {}
    t0 = time.perf_counter()
    for r in sub:
        key = (r.mesh_id, r.res)
        if key not in ref:
            v, t = host_pool[r.mesh_id]
            g = oracle.voxelize(v, t, (0, 0, 0), 1.0 / r.res, r.res)
            ref[key] = torch.from_numpy(g.view(np.int32)).cuda()
    oracle_s = time.perf_counter() - t0
    good = [0, 0]

    def cmp(tk, grid):
        good[0] += 1
        good[1] += int(torch.equal(grid, ref[(tk.mesh_id, tk.res)]))

    srv = server.Server(pool, arena_bytes=4 << 30, n_slots=3, slot_workspace_bytes=512 << 20, max_jobs=64,
                        on_result=cmp)
    try:
        srv.serve(sub, realtime=False)
    finally:
        srv.close()
    del ref
    torch.cuda.empty_cache()
    return {"exact": f"{good[1]}/{good[0]}", "requests": len(sub), "distinct_grids": len(set((r.mesh_id, r.res)
                                                                                           for r in sub)),
            "oracle_s": oracle_s, "oracle_threads": oracle.last_threads(),
            "includes": "largest pool mesh at the finest grid, smallest at the coarsest"}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(local)
    from paper_2106_01326_gb300 import build as vbuild
    from paper_2106_01326_gb300 import meshgen as mg
    from paper_2106_01326_gb300 import voxtet as vt

    if rank == 0:
        vbuild.build()
    if dist is not None:
        dist.barrier()
    vt.load()
    cfg = mg.single_mesh_config(args.workload)
    res = cfg["res"]
    n_t, n_v = len(cfg["tets"]), len(cfg["verts"])
    dev = torch.device("cuda", local)
    verts = torch.from_numpy(cfg["verts"]).to(dev)
    tets = torch.from_numpy(cfg["tets"]).to(dev)
    ws = vt.alloc_workspace(n_t, n_v, res, dev)
    slab = args.partition == "slab" and world > 1
    if slab:  # this rank's z-slab of the one grid, cut by the mesh's per-slice tet counts
        from paper_2106_01326_gb300 import slabs

        w = slabs.slice_weights(cfg["verts"], cfg["tets"], cfg["origin"], cfg["voxel_size"], res)
        z_range = slabs.rank_slab(res, rank, world, w)
        grid = vt.alloc_grid_dims((res, res, res), z_range, dev)
        sv, st = slabs.slab_mesh(cfg["verts"], cfg["tets"], cfg["origin"], cfg["voxel_size"], *z_range)
        verts = torch.from_numpy(sv).to(dev)
        tets = torch.from_numpy(st).to(dev)
    else:
        z_range = (0, res)
        grid = vt.alloc_grid(res, dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # launch shape: the autotuner times span sizes and row culling on this mesh (untimed)
    from paper_2106_01326_gb300 import autotune

    kernel = args.kernel
    if args.span_rows > 0 or kernel:
        span_rows, row_cull, tuned = args.span_rows, 0, None
    else:
        tuned = autotune.tune(verts, tets, cfg["origin"], cfg["voxel_size"], res, reps=3)
        span_rows, row_cull, kernel = tuned["span_rows"], tuned["row_cull"], tuned["kernel"]

    def call(v, t, profile=False):
        if slab:
            vt.voxelize_grid(v, t, cfg["origin"], cfg["voxel_size"], (res, res, res), z_range=z_range, out=grid,
                             workspace=ws, sync=False, span_rows=span_rows, row_cull=row_cull, profile=profile,
                             stream=stream, kernel=kernel)
        else:
            vt.voxelize(v, t, cfg["origin"], cfg["voxel_size"], res, out=grid, workspace=ws, sync=False,
                        span_rows=span_rows, row_cull=row_cull, profile=profile, stream=stream, kernel=kernel)

    def step():
        call(verts, tets, profile=True)

    for _ in range(max(args.warmup, 3)):
        step()
        torch.cuda.synchronize()
    st = vt.last_status(ws)
    if st != vt.OK:
        raise vt.VoxtetError(st)
    stats = vt.read_stats(ws)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    launches0 = vt.launch_count()
    step_ms, kern_ms = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict the mesh and grid from L2 (outside the timed events)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(vt.read_stats(ws)["kernel_ns"] / 1e6)
    launches = vt.launch_count() - launches0
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    if dist is not None:
        dist.barrier()
    st = vt.last_status(ws)
    if st != vt.OK:
        raise vt.VoxtetError(st)

    # end to end through the public API: pinned host mesh -> device, voxelize, grid -> pinned host
    h_verts = verts.cpu().pin_memory()  # this rank's vertices (a slab's own under --partition slab)
    h_tets = tets.cpu().pin_memory()  # this rank's tets (a slab's subset under --partition slab)
    h_grid = torch.empty(grid.shape, dtype=torch.int32).pin_memory()
    d_verts = torch.empty_like(verts)
    d_tets = torch.empty_like(tets)

    def e2e_step():
        d_verts.copy_(h_verts, non_blocking=True)
        d_tets.copy_(h_tets, non_blocking=True)
        call(d_verts, d_tets)
        h_grid.copy_(grid, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_single_total = max_over_ranks(sum(e2e_ms), dist, dev)

    # the same jobs as a stream through the pipelined host API: each job's mesh copy in,
    # kernels and grid copy out on three streams, 4 device slots (each ~54 MB, together
    # larger than L2) rotating, every copy inside the timed region
    e2e_total = None
    if not slab:
        from paper_2106_01326_gb300 import pipeline

        pipe = pipeline.HostPipeline(n_v, n_t, res, depth=4, device=dev, span_rows=span_rows, row_cull=row_cull,
                                     kernel=kernel)
        h_grids = [torch.empty(grid.shape, dtype=torch.int32).pin_memory() for _ in range(4)]
        for k in range(4):
            pipe.submit(h_verts, h_tets, h_grids[k], cfg["origin"], cfg["voxel_size"])
        pipe.wait()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(pipe.h2d)
        for k in range(args.steps):
            pipe.submit(h_verts, h_tets, h_grids[k % 4], cfg["origin"], cfg["voxel_size"])
        p1.record(pipe.d2h)
        pipe.wait()
        e2e_total = max_over_ranks(p0.elapsed_time(p1), dist, dev)
        pipe_ok = all(torch.equal(h_grids[k], h_grids[0]) for k in range(1, 4)) and torch.equal(h_grids[0], h_grid)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    jobs = 1 if slab else world  # meshes voxelized per step across all ranks
    value = whole_job_rate(n_t, jobs, args.steps, total_ms)
    gvox = jobs * (res ** 3) * args.steps / (total_ms / 1000.0) / 1e9
    kmean = statistics.mean(kern_ms)
    grid_bytes = grid.numel() * 4  # this rank's slab (the whole grid unless partitioned)
    alg_bytes = 16 * n_t + 12 * n_v + grid_bytes
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (kmean / 1000.0) / 1e9
    # the launches the library's profile events bracket
    main_kernel = ("k_slices + k_voxelize (list pass over the tets the slice-unit kernel leaves)"
                   if kernel == 2 else "k_voxelize")
    traffic_kernel = "k_slices" if kernel == 2 else "k_voxelize"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if slab else "weak",
        "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: 60^3 jittered Kuhn lattice, 2% slivers, {n_t} tets, {n_v} verts "
                               f"-> {res}^3 bit grid", "res": res, "n_tets": n_t, "n_verts": n_v,
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"z-slabs x{world}" if slab else f"replicas x{world}",
                   "span_rows": span_rows, "row_cull": {0: "auto", 1: "on", 2: "off"}[row_cull],
                   "kernel": {0: "auto", 1: "spans", 2: "slice units"}[kernel],
                   "launch_shape": "autotuned" if tuned else "given",
                   "tuning_table_us": tuned["table"] if tuned else None},
        "gvox_per_s": gvox,
        "e2e": {"value": whole_job_rate(n_t, jobs, args.steps, e2e_total if e2e_total else e2e_single_total),
                "unit": UNIT, "h2d_bytes_per_step": 12 * n_v + 16 * n_t, "d2h_bytes_per_step": grid_bytes,
                "api": "pipeline.HostPipeline (copies of one job overlap the kernels of the next)" if e2e_total
                       else "one voxelize call per step, copies before and after",
                "single_call_value": whole_job_rate(n_t, jobs, args.steps, e2e_single_total),
                "grids_equal_device_path": bool(pipe_ok) if e2e_total else None},
        "gpu_launches": int(launches),
        # the kernel is bound by issued lane operations, not by HBM: its primary roofline is the
        # ALU one; the HBM fraction (algorithmic bytes over the measured copy bandwidth) is kept beside it
        "roofline": dict(alu_roofline(int(stats["rows"]), n_t, kmean), traffic=recorded_traffic(args.workload, traffic_kernel),
                         kernel=main_kernel, kernel_ms=kmean),
        "hbm_roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": recorded_traffic(args.workload, traffic_kernel), "kernel": main_kernel, "kernel_ms": kmean,
                         "algorithmic_bytes": alg_bytes, "peak_source": peak_kind},
        "stats": {"rows": int(stats["rows"]), "spans": int(stats["spans"]),
                  "fallback_rows": int(stats["fallback_rows"]), "degenerate_tets": int(stats["degenerate_tets"]),
                  "wide_tets": int(stats["wide_tets"])},
        "clocks": clocks,
    }
    if not args.no_batched:
        line["batched"] = batched_section(args, flush, stream)
    if not args.no_served:
        line["served"] = served_section(args)
    if not args.no_sparse:
        line["sparse"] = sparse_section(stream)
    if not args.no_slabs and world == 1:
        line["slabs_one_gpu"] = slab_section(verts, tets, cfg, span_rows, row_cull, stream, kernel)
    if not args.no_cpu_baseline:
        import numpy as np

        import oracle

        oracle.build()
        v, dt, depth, cores = cpu_oracle_sample(cfg, args.slab)
        v1, dt1, depth1, _ = cpu_oracle_sample(cfg, max(8, args.slab // 8), n_threads=1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"z-slab of {depth} of {res} slices, all tets overlapping it, {dt:.2f} s; "
                                          f"tets/s = n_tets x {depth}/{res} / time",
                                "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                  "sample": f"z-slab of {depth1} of {res} slices, {dt1:.2f} s"}}
        if not slab:
            # the timed grid against the oracle's, every sample of it
            exact, xyz, info = oracle_whole_grid(cfg)
            got = grid.cpu().numpy().view(np.uint32).reshape(exact.shape)
            line["parity"] = {"bit_identical_to_oracle": bool(np.array_equal(got, exact)),
                              "compared": f"whole {res}^3 grid of the timed call ({res ** 3} samples)",
                              "oracle_s": info["s"], "oracle_threads": info["threads"]}
            # the per-row work the method cannot avoid: rows holding a sample (a property of the mesh
            # and grid, counted by the oracle), beside the candidate rows the kernel visited
            line["roofline"] = dict(line["roofline"], **alu_roofline(int(stats["rows"]), n_t, kmean,
                                                                     rows_with_samples=info["rows_with_samples"]))
            line["cpu_baseline"]["paper_cpu_method"] = paper_cpu_comparison(cfg, exact, xyz, info)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
