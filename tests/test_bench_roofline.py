"""The benchmark's roofline arithmetic on CPU: the committed ncu capture is
read only while the field kernel's source is the captured one, and the
issue roofline follows from its counters, the kernel time and the clock."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_profile_counters_belong_to_the_current_source():
    traffic, counters = bench.read_profile_traffic()
    d = json.load(open(os.path.join(ROOT, "profiles", "k_guide_stream_frame1080p.json")))
    if traffic is None:
        pytest.skip("the field kernel changed since the capture: its counters are withheld")
    assert traffic == d["dram_bytes_per_launch"]
    assert counters["warp_instructions_per_launch"] == d["warp_instructions_per_launch"]


def test_profile_counters_are_withheld_for_another_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    d = json.load(open(os.path.join(ROOT, "profiles", "k_guide_stream_frame1080p.json")))
    src = tmp_path / d["source"]
    src.parent.mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, d["source"]), src)
    with open(src, "a") as f:
        f.write("\n// edited\n")
    (prof / "k_guide_stream_frame1080p.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_profile_traffic() == (None, None)


def test_issue_roofline_arithmetic():
    c = {"warp_instructions_per_launch": 5.2e8, "active_lanes_per_warp_instruction": 16.0}
    r = bench.issue_roofline(c, kernel_ms=1.0, sm_mhz=2000.0, n_sm=152)
    assert r["achieved"] == pytest.approx(520.0)               # G warp instructions per second
    assert r["peak"] == pytest.approx(152 * 4 * 2.0)           # one per scheduler per cycle
    assert r["frac"] == pytest.approx(520.0 / 1216.0)
    assert r["lane_frac"] == pytest.approx(r["frac"] * 0.5)
    assert bench.issue_roofline(None, 1.0, 2000.0, 152) is None
    assert bench.issue_roofline(c, 1.0, None, 152) is None
    assert bench.issue_roofline({"active_lanes_per_warp_instruction": 16.0}, 1.0, 2000.0, 152) is None
