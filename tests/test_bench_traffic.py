"""bench.py's DRAM-traffic lookup: a stored ncu capture is used only while the sources of the
workload's dominant kernel hash to the value recorded with it, and is scaled per voxel.  CPU only."""
import json

import bench


def test_traffic_needs_matching_sources(tmp_path, monkeypatch):
    f = tmp_path / "t.json"
    good = {"bytes_per_voxel_launch": 200.0, "source_hash": bench.kernel_source_hash("euler3d")}
    f.write_text(json.dumps({"workloads": {"euler3d": good}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("euler3d", 1000) == 200.0 * 1000
    assert bench.measured_traffic("wave3d", 1000) is None
    f.write_text(json.dumps({"workloads": {"euler3d": dict(good, source_hash="0" * 16)}}))
    assert bench.measured_traffic("euler3d", 1000) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("euler3d", 1000) is None


def test_source_hashes():
    for name in bench.WORKLOADS:
        assert bench.kernel_source_hash(name) == bench.kernel_source_hash(name)
        assert len(bench.kernel_source_hash(name)) == 16
    assert bench.kernel_source_hash("wave3d") == bench.kernel_source_hash("gw59")
    assert bench.kernel_source_hash("euler3d") != bench.kernel_source_hash("wave3d")


def test_hash_ignores_comments():
    a = "int f(int x) {  // the answer\n  return x; /* done */\n}\n"
    b = "int f(int x) {\n\n  return x;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(b.replace("x;", "x + 1;"))
