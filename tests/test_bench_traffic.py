"""bench.py reports an ncu DRAM-traffic figure only for the kernel sources it
was captured on."""
import json

import bench

SRC = ["paper_2602_15883_b300/csrc/pinn_kernels.cuh"]


def test_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    rec = {"captures": [{"workload": "tgv", "precision": "fp32", "dram_bytes_per_launch": 123,
                         "sources": SRC, "sources_sha256": bench.kernel_source_sha256(SRC)}]}
    f = tmp_path / "t.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.captured_traffic("tgv", "fp32") == 123
    assert bench.captured_traffic("tgv", "fp32", scale=8) is None   # a reduced profiling run is another workload
    assert bench.captured_traffic("tgv", "tf32x3") is None
    assert bench.captured_traffic("beltrami32", "fp32") is None
    rec["captures"][0]["sources_sha256"] = "0" * 64          # sources changed since the capture
    f.write_text(json.dumps(rec))
    assert bench.captured_traffic("tgv", "fp32") is None
    rec["captures"][0]["sources"] = ["no/such/file.cuh"]
    f.write_text(json.dumps(rec))
    assert bench.captured_traffic("tgv", "fp32") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.captured_traffic("tgv", "fp32") is None


def test_recorded_captures_name_existing_sources():
    import os
    rec = json.load(open(bench.TRAFFIC_FILE))
    root = os.path.dirname(os.path.abspath(bench.__file__))
    for c in rec["captures"]:
        assert c["sources"] and all(os.path.exists(os.path.join(root, f)) for f in c["sources"])
