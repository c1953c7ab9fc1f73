"""The benchmark's DRAM-traffic figure comes only from a committed profile
summary whose capture covered the current kernel sources: a line keyed to
another source hash is ignored (no GPU needed)."""
import os
import shutil

import bench


def test_traffic_line_needs_matching_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1610_07902_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("kernels.cu", "expand_dev.cuh", "spmspv_internal.cuh", "device_util.cuh", "selector_dev.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1610_07902_gb300", "csrc", name), csrc / name)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernels_hash()
    (tmp_path / "profiles" / "k.md").write_text(
        "traffic: k2_expand_scatter 9.5 bytes per product (sources %s)\n"
        "traffic: k3_bucket_merge 1.25 bytes per product (sources 0123456789abcdef)\n" % h)
    assert bench.captured_traffic("k2_expand_scatter") == (9.5, "k.md")
    assert bench.captured_traffic("k3_bucket_merge") == (None, None)  # captured from other sources
    # any change to the sources withdraws the figure
    with open(csrc / "kernels.cu", "a") as fh:
        fh.write("\n// changed\n")
    assert bench.kernels_hash() != h
    assert bench.captured_traffic("k2_expand_scatter") == (None, None)


def test_committed_summary_parses():
    # every traffic line of the committed summaries has the expected form
    import glob
    import re
    n = 0
    for path in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")):
        for line in open(path):
            if line.startswith("traffic:"):
                assert re.match(r"traffic: \S+ [0-9.]+ bytes per \w+ \(sources [0-9a-f]{16}\)$", line.strip()), line
                n += 1
    assert n >= 1
