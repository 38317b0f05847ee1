"""bench.py's DRAM-traffic lookup: a stored ncu capture is used only while the kernel sources
hash to the value recorded with it, and is scaled per voxel.  CPU only."""
import json

import bench


def test_traffic_needs_matching_sources(tmp_path, monkeypatch):
    f = tmp_path / "t.json"
    f.write_text(json.dumps({"source_hash": bench.kernel_source_hash(),
                             "workloads": {"euler3d": {"bytes_per_voxel_launch": 200.0}}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("euler3d", 1000) == 200.0 * 1000
    assert bench.measured_traffic("wave3d", 1000) is None
    f.write_text(json.dumps({"source_hash": "0" * 16,
                             "workloads": {"euler3d": {"bytes_per_voxel_launch": 200.0}}}))
    assert bench.measured_traffic("euler3d", 1000) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("euler3d", 1000) is None


def test_source_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16
