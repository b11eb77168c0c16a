"""The bench line's DRAM-traffic figures on CPU: a committed ncu figure is reported
only for the kernel sources it was captured from (any edit to them makes the
figure null), and only for its own workload key."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _entries():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)["entries"]


def test_committed_entries_are_well_formed():
    for e in _entries():
        assert e["dram_bytes_per_launch"] == e["dram_read"] + e["dram_write"]
        assert len(e["source_sha256"]) == 64
        assert os.path.exists(os.path.join(ROOT, e["summary"]))


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2605_14035_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text("// " + f + "\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    entry = {"kernel": "k", "workload": "w_tile2304", "source_sha256": h, "dram_bytes_per_launch": 10.0,
             "dram_read": 4.0, "dram_write": 6.0, "summary": "x"}
    (prof / "traffic.json").write_text(json.dumps({"entries": [entry]}))
    assert bench.measured_traffic("k", "w_tile2304") == 10.0
    assert bench.measured_traffic("k", "w_tile2048") is None     # another tiling
    assert bench.measured_traffic("other", "w_tile2304") is None  # another kernel
    (csrc / bench.KERNEL_SOURCES[0]).write_text("// edited\n")
    assert bench.measured_traffic("k", "w_tile2304") is None     # sources changed since the capture


def test_batch_hash_covers_more_sources():
    assert set(bench.KERNEL_SOURCES) < set(bench.BATCH_SOURCES)
    assert bench.kernel_source_hash(bench.BATCH_SOURCES) != bench.kernel_source_hash()
