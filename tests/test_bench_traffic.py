"""The DRAM-traffic figure bench.py reports as roofline.traffic (CPU only).

The figure comes from a committed ncu capture of the pair-convolution passes
(`profiles/pairconv_traffic.json`) and is reported only while the pass
sources hash to the value stored with it; after any change to those sources
the bench reports null with the reason, until the capture is taken again.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402

TRAFFIC = os.path.join(os.path.dirname(HERE), "profiles", "pairconv_traffic.json")


def test_committed_capture_matches_the_pass_sources():
    d = json.load(open(TRAFFIC))
    # a stale capture means: the passes changed, take the capture again
    assert d["kernel_sources_sha256"] == bench.pairconv_sources_sha256()
    traffic, note = bench.committed_traffic()
    assert traffic == d["traffic_bytes_per_step"]
    assert traffic == d["dram_read_bytes_per_step"] + d["dram_write_bytes_per_step"]
    assert note.startswith("ncu capture of")


def test_changed_sources_give_no_traffic(tmp_path, monkeypatch):
    d = json.load(open(TRAFFIC))
    d["kernel_sources_sha256"] = "0" * 64
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "profiles" / "pairconv_traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "pairconv_sources_sha256", lambda: "f" * 64)
    traffic, note = bench.committed_traffic()
    assert traffic is None
    assert note.startswith("stale")


def test_missing_capture_gives_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, note = bench.committed_traffic()
    assert traffic is None and note == "no committed capture"
