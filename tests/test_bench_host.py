"""Host-side arithmetic of bench.py (no GPU): the whole-job rate, the ALU roofline, and the rule
that a recorded ncu traffic figure is reported only for the sources and workload it was taken on."""
import math

import bench


def test_whole_job_rate():
    # 2 ranks x 1000 units x 10 steps in 20 ms (the slowest rank) = 1e6 units/s
    assert math.isclose(bench.whole_job_rate(1000, 2, 10, 20.0), 1.0e6)


def test_alu_roofline_counts_and_peak():
    r = bench.alu_roofline(rows=1000, tets=10, kernel_ms=1.0)
    ops = bench.ALU_OPS_PER_ROW * 1000 + bench.ALU_OPS_PER_TET * 10
    assert r["bound"] == "alu" and r["algorithmic_ops"] == ops
    assert math.isclose(r["achieved"], ops / 1e-3 / 1e12)
    mhz = float(r["peak_source"].split(" x ")[-1].split()[0])
    assert math.isclose(r["peak"], 152 * 128 * mhz * 1e6 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])


def test_recorded_traffic_only_for_matching_sources(monkeypatch):
    rec = bench.recorded_traffic("sliver_60", "k_slices")
    if rec is not None:  # the committed capture matches the committed sources
        assert rec > 40_000_000
    assert bench.recorded_traffic("torus_48", "k_slices") is None  # another workload
    assert bench.recorded_traffic("sliver_60", "k_nonexistent") is None  # no capture of that kernel
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 64)
    assert bench.recorded_traffic("sliver_60", "k_slices") is None  # sources changed since the capture


def test_alu_roofline_counts_rows_with_samples_when_known():
    """With the oracle's count of rows holding a sample, the per-row work is counted on those
    (the work no method avoids), not on the candidate rows the kernel visited."""
    r = bench.alu_roofline(rows=1000, tets=10, kernel_ms=1.0, rows_with_samples=700)
    assert r["algorithmic_ops"] == bench.ALU_OPS_PER_ROW * 700 + bench.ALU_OPS_PER_TET * 10
    assert r["rows_candidate"] == 1000 and r["rows_with_samples"] == 700
    assert r["frac"] < bench.alu_roofline(rows=1000, tets=10, kernel_ms=1.0)["frac"]
