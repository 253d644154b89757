"""Host logic of bench.py that the JSON line depends on, CPU only: the DRAM traffic of a
kernel is reported only while the committed capture was taken on the current kernel
sources; the source digest covers every CUDA source and nothing else; the command line
offers every workload and path."""
import json
import os
import shutil

import pytest

import bench


def test_source_digest_tracks_the_kernel_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1405_3331_gb300" / "csrc"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1405_3331_gb300", "csrc"), csrc,
                    ignore=shutil.ignore_patterns("*.o", "*.so", "__pycache__"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest()
    assert len(d0) == 16
    (csrc / "notes.txt").write_text("not a source")
    assert bench.source_digest() == d0                      # only .cu / .cuh / .h count
    k = csrc / "k_resident.cu"
    k.write_text(k.read_text() + "\n")
    assert bench.source_digest() != d0                      # any change to a kernel source moves it


def test_recorded_traffic_only_for_the_current_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "source_digest", lambda: "abcdef0123456789")
    (tmp_path / "profiles").mkdir()
    entries = {"fused@c2": {"dram_bytes_per_launch": 123, "source_digest": "abcdef0123456789"},
               "field@c3": {"dram_bytes_per_launch": 456, "source_digest": "0000000000000000"}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entries))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("fused", "c2") == 123.0
    assert bench.recorded_traffic("field", "c3") is None      # taken on other sources
    assert bench.recorded_traffic("step", "c4") is None       # never taken


def test_committed_traffic_entries_are_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        entries = json.load(f)
    for key, e in entries.items():
        kernel, _, work = key.partition("@")
        assert kernel and work in ("c1", "c2", "c2x", "c3", "c4", "c5"), key
        assert e["dram_bytes_per_launch"] > 0 and len(e["source_digest"]) == 16 and e["note"], key


@pytest.mark.parametrize("flag,values", [("--workload", ["c1", "c2", "c2x", "c3", "c4", "c5", "graph"]),
                                         ("--path", ["auto", "plain", "fused", "persist", "resident"])])
def test_command_line_offers_every_workload_and_path(monkeypatch, flag, values):
    for v in values:
        monkeypatch.setattr("sys.argv", ["bench.py", flag, v])
        assert getattr(bench.parse_args(), flag[2:]) == v
