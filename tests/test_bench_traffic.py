"""Host logic of the benchmark's DRAM-traffic field (no GPU): a record is
used only when it was taken on the current kernel sources, and a per-step
record scales with the shots of the benchmark's launches."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _write(tmp_path, rec):
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    with open(tmp_path / "profiles" / "traffic.json", "w") as f:
        json.dump(rec, f)


def test_record_matches_sources_and_scales_with_launch_shots(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    _write(tmp_path, {"k_fwd": {"source_hash": "abc", "bytes_per_launch_full": 800, "shots_per_launch": 8},
                      "k_adj": {"source_hash": "old", "bytes_per_launch_full": 900, "shots_per_launch": 8},
                      "k_fwd_persist": {"source_hash": "abc", "bytes_per_launch_full": 5000}})
    assert bench.traffic_record("k_fwd") == 800
    assert bench.traffic_record("k_fwd", 16) == 1600          # two lanes of 32 shots: 16 per launch
    assert bench.traffic_record("k_fwd", 8) == 800
    assert bench.traffic_record("k_adj", 8) is None           # taken on other sources
    assert bench.traffic_record("k_fwd_persist", None) == 5000
    assert bench.traffic_record("k_born") is None


def test_committed_record_names_the_per_step_kernels():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for k in ("k_fwd", "k_adj"):
        assert d[k]["bytes_per_launch_full"] > 0 and d[k]["shots_per_launch"] > 0 and d[k]["source_hash"]
