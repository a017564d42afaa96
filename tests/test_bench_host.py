"""Host logic of bench.py that needs no GPU: the committed ncu figures are
used only for the kernel source they were captured on, the right figure is
read for each key, and the issue-rate peak follows the SM count."""
import json
import os

import bench


def write_profile(tmp_path, src_hash):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"source_hash": src_hash, "bytes_per_launch": 1000, "inst_per_launch": 2000}
    (prof / "traffic.json").write_text(json.dumps({"3d_1m": {"fused": entry}}))


def test_figures_only_for_the_captured_source(tmp_path, monkeypatch):
    write_profile(tmp_path, "abc")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.ncu_traffic("3d_1m", "fused") == 1000.0
    assert bench.ncu_traffic("3d_1m", "fused", "inst_per_launch") == 2000.0
    assert bench.ncu_traffic("3d_8m", "fused") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.ncu_traffic("3d_1m", "fused") is None
    assert bench.ncu_traffic("3d_1m", "fused", "inst_per_launch") is None


def test_source_hash_covers_the_search_sources():
    """Every file the tile search is compiled from takes part in the hash."""
    csrc = os.path.join(bench.ROOT, "paper_2401_08586_gb300", "csrc")
    with open(os.path.join(csrc, "nnps_tile.cu")) as f:
        text = f.read()
    local = {line.split('"')[1] for line in text.splitlines() if line.startswith('#include "')}
    hashed = set(bench.KERNEL_SOURCES)
    # launch.cuh declares host launchers only
    assert local - {"launch.cuh"} <= hashed
    assert len(bench.kernel_source_hash()) == 16


def test_issue_peak():
    assert bench.issue_per_clock(152) == 152 * 4
