"""Host logic that needs no GPU: in bench.py, which committed ncu summary a
launch may use (source hash, register budget, skip level, multi-scale level
configuration), the issue roofline arithmetic
and the algorithmic-bytes model of the fetch counters; in the binding, the
autotuner cache's key and file."""
import json

import pytest

import bench


def test_occupancy_key_follows_pin_then_autotuner():
    assert bench.occupancy_key("9", None) == "9"
    assert bench.occupancy_key("8", {"engine": 1, "occupancy": 2}) == "8"  # a pin wins
    assert bench.occupancy_key("auto", None) == "8"  # grid default: 8 blocks per SM
    assert bench.occupancy_key("auto", {"engine": 1, "occupancy": 2}) == "9"
    assert bench.occupancy_key("auto", {"engine": 1, "occupancy": 1}) == "8"
    assert bench.occupancy_key("auto", {"engine": 1, "occupancy": 0}) == "8"
    assert bench.occupancy_key("auto", {"engine": 2, "occupancy": 0}) is None  # loop nest: no count


def _profiles(tmp_path, monkeypatch, name, payload):
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / f"render_{name}_traffic.json").write_text(json.dumps(payload))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "render_source_sha", lambda workload="room": "abc")


def test_summary_is_ignored_when_the_kernel_source_changed(tmp_path, monkeypatch):
    _profiles(tmp_path, monkeypatch, "room", {"source_sha": "old", "warp_inst_per_launch": 10,
                                               "dram_bytes_per_launch": 5})
    assert bench.ncu_summary("room") == {}
    assert bench.ncu_traffic("room") is None
    assert bench.issue_roofline("room", 1.0, 2070.0, 152) is None


def test_summary_per_register_budget(tmp_path, monkeypatch):
    _profiles(tmp_path, monkeypatch, "batched", {
        "source_sha": "abc",
        "by_occupancy": {"8": {"warp_inst_per_launch": 100, "dram_bytes_per_launch": 7},
                         "9": {"warp_inst_per_launch": 200, "dram_bytes_per_launch": 9}}})
    assert bench.ncu_traffic("batched", "8") == 7.0
    assert bench.ncu_traffic("batched", "9") == 9.0
    assert bench.ncu_summary("batched") == {}  # a keyed summary needs the budget
    assert bench.ncu_summary("batched", None) == {}


def test_summary_needs_the_skip_level_it_was_taken_at(tmp_path, monkeypatch):
    """Counts depend on the block side the walk skipped with: a summary is
    used only for a launch at the same skip level (one per multi-scale level)."""
    _profiles(tmp_path, monkeypatch, "room", {"source_sha": "abc", "skip_block": 4, "warp_inst_per_launch": 10,
                                               "dram_bytes_per_launch": 5})
    assert bench.ncu_traffic("room", "8", 4) == 5.0
    assert bench.ncu_traffic("room", "8", 8) is None
    assert bench.ncu_traffic("room", "8") is None
    _profiles(tmp_path, monkeypatch, "multiscale", {"source_sha": "abc", "skip_block": [4, 8, 16], "levels": {}})
    assert bench.ncu_summary("multiscale", skip=[4, 8, 16]) != {}
    assert bench.ncu_summary("multiscale", skip=[4, 8, 32]) == {}


def test_level_config_key():
    assert bench.level_config_key("nested", "auto", None) == "nested"
    assert bench.level_config_key("auto", "9", None) == "9"
    assert bench.level_config_key("auto", "auto", {"engine": 1, "occupancy": 2}) == "9"
    assert bench.level_config_key("auto", "auto", {"engine": 2, "tile": [8, 4], "schedule": 2}) == "nested"
    assert bench.level_config_key("auto", "auto", {"engine": 2, "tile": [16, 8], "schedule": 2}) is None
    assert bench.level_config_key("auto", "auto", {"engine": 2, "tile": [8, 4], "schedule": 1}) is None


def test_issue_roofline_arithmetic(tmp_path, monkeypatch):
    # 1258.56 G warp instructions in one second at 2070 MHz on 152 SMs = 100 %
    _profiles(tmp_path, monkeypatch, "room", {"source_sha": "abc", "warp_inst_per_launch": 1258.56e6,
                                               "dram_bytes_per_launch": 1})
    r = bench.issue_roofline("room", 1.0, 2070.0, 152, "8")
    assert r["peak"] == pytest.approx(1258.6, abs=0.05)
    assert r["achieved"] == pytest.approx(1258.6, abs=0.05)
    assert r["frac"] == pytest.approx(1.0, abs=1e-4)
    assert bench.issue_roofline("room", 2.0, 2070.0, 152, "8")["frac"] == pytest.approx(0.5, abs=1e-4)
    assert bench.issue_roofline("room", 1.0, None, 152, "8") is None  # no clock sample, no peak


def test_bytes_model_counts_each_fetch_kind():
    c = {"coarse": 1, "fine": 0, "normal": 0, "radiance": 0, "rays": 0}
    assert bench.bytes_model(c, False, False) == 8  # min + max of a low-resolution texel
    c = {"coarse": 0, "fine": 1, "normal": 0, "radiance": 0, "rays": 0}
    assert bench.bytes_model(c, False, False) == 4  # one distance
    for f16, nb, rb in ((False, 8, 12), (True, 4, 8)):
        assert bench.bytes_model({"coarse": 0, "fine": 0, "normal": 1, "radiance": 0, "rays": 0}, f16, f16) == nb
        assert bench.bytes_model({"coarse": 0, "fine": 0, "normal": 0, "radiance": 1, "rays": 0}, f16, f16) == rb
    # rgb f32 x 3 + class u8 per ray
    assert bench.bytes_model({"coarse": 0, "fine": 0, "normal": 0, "radiance": 0, "rays": 1}, False, False) == 13


def test_committed_summaries_parse():
    """Every committed traffic summary is JSON with a source hash and the
    fields the bench reads."""
    import glob
    import os
    files = glob.glob(os.path.join(os.path.dirname(bench.__file__), "profiles", "render_*_traffic.json"))
    assert files
    for f in files:
        d = json.load(open(f))
        assert "source_sha" in d, f
        assert isinstance(d.get("skip_block"), (int, list)), f
        entries = list(d.get("by_occupancy", {}).values())
        for lv in d.get("levels", {}).values():
            entries += list(lv["by_occupancy"].values())
        if not entries:
            entries = [d]
        for e in entries:
            assert ("warp_inst_per_launch" in e) or ("warp_inst_per_ray" in e), f


def test_autotune_cache_key_and_file(tmp_path):
    """The autotuner's cache key names the GPU, the library build, the grid
    descriptor and the multiset of view sizes; picks round-trip through the
    JSON file."""
    import types
    import paper_2507_14624_gb300 as lfpk
    from paper_2507_14624_gb300 import lfp
    d = lfp.lfp_grid_desc()
    d.nx, d.ny, d.nz, d.spacing, d.N, d.M = 4, 4, 4, 0.5, 256, 16
    grid = types.SimpleNamespace(desc=d)
    V = lambda w, h: types.SimpleNamespace(W=w, H=h)  # noqa: E731
    k1 = lfpk.tune_key(grid, [V(64, 48), V(32, 32)], "GB300")
    assert k1 == lfpk.tune_key(grid, [V(32, 32), V(64, 48)], "GB300")  # order does not matter
    assert k1 != lfpk.tune_key(grid, [V(64, 48), V(32, 33)], "GB300")
    assert k1 != lfpk.tune_key(grid, [V(64, 48), V(32, 32)], "B200")
    d2 = lfp.lfp_grid_desc()
    d2.nx, d2.ny, d2.nz, d2.spacing, d2.N, d2.M = 4, 4, 4, 0.5, 256, 32
    assert k1 != lfpk.tune_key(types.SimpleNamespace(desc=d2), [V(64, 48), V(32, 32)], "GB300")
    path = str(tmp_path / "tune.json")
    pick = {"engine": 2, "tile": (16, 8), "schedule": 2, "occupancy": 0}
    lfpk._write_tune_cache(path, k1, pick)
    lfpk._write_tune_cache(path, "other", dict(pick, engine=1))
    got = lfpk._read_tune_cache(path)
    assert got[k1] == {"engine": 2, "tile": [16, 8], "schedule": 2, "occupancy": 0}
    assert got["other"]["engine"] == 1


def test_adjoint_bytes_and_traffic_summary(tmp_path, monkeypatch):
    # 12 B gradient + 16 B saved state + 4 taps x 3 channels x 8 B read-modify-write
    assert bench.BWD_BYTES_PER_HIT == 124
    (tmp_path / "profiles").mkdir()
    p = tmp_path / "profiles" / "backward_fit_traffic.json"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "backward_source_sha", lambda: "cur")
    p.write_text(json.dumps({"source_sha": "cur", "dram_bytes_per_launch": 123.0}))
    assert bench.backward_traffic("fit") == 123.0
    p.write_text(json.dumps({"source_sha": "old", "dram_bytes_per_launch": 123.0}))
    assert bench.backward_traffic("fit") is None  # taken on another adjoint source
    assert bench.backward_traffic("batched") is None  # no summary
