"""Host logic of the benchmark's DRAM-traffic field (no GPU): a record is
used only when it was taken on the current kernel sources, and it scales
with the grid-point updates of the benchmark's launches."""
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


def test_record_matches_sources_and_scales_with_launch_updates(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    _write(tmp_path, {"large": {"k_fwd_traces": {"source_hash": "abc", "dram_bytes_per_update": 5.5},
                                "k_adj": {"source_hash": "old", "dram_bytes_per_update": 20.0}}})
    assert bench.traffic_record("large", "k_fwd_traces", 1000) == 5500.0
    assert bench.traffic_record("large", "k_adj", 1000) is None          # taken on other sources
    assert bench.traffic_record("batched", "k_fwd_traces", 1000) is None  # no record for that workload
    assert bench.traffic_record("large", "k_born", 1000) is None


def test_committed_record_names_the_headline_kernels():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for k in ("k_fwd_traces", "k_fwd_history", "k_adj"):
        r = d["large"][k]
        assert r["dram_bytes_per_update"] > 0 and r["source_hash"] and r["launches"] > 0
