"""Host logic of the autotuner, without a GPU: candidate choice, the equal-grid check and the
per-device, per-resolution cache (timings and grids come from a fake)."""
import json

import pytest
import torch

from paper_2106_01326_gb300 import autotune


@pytest.fixture()
def fake(monkeypatch, tmp_path):
    monkeypatch.setenv("VOXTET_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_device_key", lambda: "FakeGPU")
    monkeypatch.setattr(autotune.vt, "alloc_workspace", lambda *a, **k: None)
    state = {"times": {}, "grids": {}, "calls": []}

    def time_config(verts, tets, origin, voxel_size, res, span, cull, reps, workspace=None, out=None, kernel=1):
        key = (span, cull) if kernel == 1 else ("slices", cull)
        state["calls"].append(key)
        g = state["grids"].get(key, torch.zeros(4, dtype=torch.int32))
        return state["times"][key], g

    monkeypatch.setattr(autotune, "time_config", time_config)
    return state


def _mesh():
    return torch.zeros((4, 3)), torch.zeros((1, 4), dtype=torch.int32)


def _times(f):
    t = {(s, c): f(s, c) for s in autotune.SPAN_CANDIDATES for c in (1, 2)}
    t.update({("slices", c): f(0, c) for c in (1, 2)})
    return t


def test_picks_fastest_and_caches(fake, tmp_path):
    fake["times"] = _times(lambda s, c: 100.0 + s / 64 + 10 * c)
    fake["times"][(512, 1)] = 50.0
    v, t = _mesh()
    r = autotune.tune(v, t, (0, 0, 0), 1 / 512, 512)
    assert (r["kernel"], r["span_rows"], r["row_cull"], r["us"]) == (1, 512, 1, 50.0)
    assert len(r["table"]) == 2 * len(autotune.SPAN_CANDIDATES) + 2
    assert sorted(map(str, fake["calls"])) == sorted(map(str, fake["times"]))  # every candidate timed once
    assert autotune.settings_for(512) == (512, 1, 1)
    assert autotune.settings_for(256) == (0, 0, 0)  # untuned resolution: the library's own choice
    stored = json.load(open(tmp_path / "tune.json"))
    assert set(stored) == {"FakeGPU/res512"}


def test_slice_units_can_win(fake):
    fake["times"] = _times(lambda s, c: 100.0 + c)
    fake["times"][("slices", 1)] = 40.0
    v, t = _mesh()
    r = autotune.tune(v, t, (0, 0, 0), 1 / 1024, 1024)
    assert (r["kernel"], r["span_rows"], r["row_cull"]) == (2, 0, 1)
    assert r["table"]["slices/1"] == 40.0
    assert autotune.settings_for(1024) == (0, 1, 2)


def test_candidate_that_changes_the_grid_is_rejected(fake):
    fake["times"] = _times(lambda s, c: 1.0)
    fake["grids"][(128, 2)] = torch.ones(4, dtype=torch.int32)
    v, t = _mesh()
    with pytest.raises(RuntimeError, match="changed the grid"):
        autotune.tune(v, t, (0, 0, 0), 1 / 64, 64)
    assert autotune.settings_for(64) == (0, 0, 0)  # nothing stored


def test_store_false_leaves_cache_alone(fake, tmp_path):
    fake["times"] = {(s, 1): float(s) for s in autotune.SPAN_CANDIDATES}
    v, t = _mesh()
    r = autotune.tune(v, t, (0, 0, 0), 1 / 128, 128, culls=(1,), store=False, kernels=(1,))
    assert r["span_rows"] == min(autotune.SPAN_CANDIDATES)
    assert not (tmp_path / "tune.json").exists()
