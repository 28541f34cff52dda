"""Host logic of the benchmark (no GPU): the per-launch DRAM traffic recorded with
an ncu capture is reported only while the kernel's source is the one captured."""
import hashlib
import json
import os

import bench


def _tree(tmp_path, source_text, recorded_hash):
    src_dir = tmp_path / "paper_2404_14691_b300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "k.cu").write_text(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(
        {"wl": {"kern": {"source": "k.cu", "source_sha256_16": recorded_hash, "dram_bytes_per_launch": 1234,
                         "capture": "test"}}}))


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    text = "__global__ void k() {}\n"
    _tree(tmp_path, text, hashlib.sha256(text.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("kern", "wl") == 1234
    assert bench.traffic_for("kern", "other-workload") is None
    assert bench.traffic_for("other-kernel", "wl") is None
    # the kernel changed since the capture: no traffic figure
    (tmp_path / "paper_2404_14691_b300" / "csrc" / "k.cu").write_text(text + "// edited\n")
    assert bench.traffic_for("kern", "wl") is None


def test_committed_traffic_entries_name_existing_sources():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for wl, kernels in d.items():
        for kind, rec in kernels.items():
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2404_14691_b300", "csrc", rec["source"])), (wl, kind)
            assert rec["dram_bytes_per_launch"] > 0 and len(rec["source_sha256_16"]) == 16
