"""Host-side pieces of bench.py's JSON line on CPU: the ncu DRAM-traffic record is reported
only for the exact kernel source it was captured on, and the clock sampler keeps only the
samples taken after the timed region starts and flags the throttle reasons the timing rules
reject."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_reported_for_the_captured_source_only(monkeypatch, tmp_path):
    src = tmp_path / "kernel.cu"
    hdr = tmp_path / "kernel.cuh"
    src.write_text("__global__ void k() {}\n")
    hdr.write_text("#pragma once\n")
    digest = hashlib.sha256(src.read_bytes() + hdr.read_bytes()).hexdigest()
    rels = [os.path.relpath(src, ROOT), os.path.relpath(hdr, ROOT)]
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {
        ("w", "p", 8, 2): {"sources": rels, "sha256": digest, "row_sweep": 111, "col_sweep": 222}})
    assert bench.ncu_traffic("w", "p", 8, 2, "row_sweep") == 111
    assert bench.ncu_traffic("w", "p", 8, 2, "col_sweep") == 222
    assert bench.ncu_traffic("w", "p", 16, 2, "row_sweep") is None  # another size
    hdr.write_text("#pragma once\n// changed\n")
    assert bench.ncu_traffic("w", "p", 8, 2, "row_sweep") is None  # a header of the kernel changed
    hdr.write_text("#pragma once\n")
    assert bench.ncu_traffic("w", "p", 8, 2, "row_sweep") == 111
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.ncu_traffic("w", "p", 8, 2, "row_sweep") is None  # the kernel changed


def test_recorded_traffic_matches_the_committed_sources():
    """Every committed record names an existing source, and a record whose hash no longer
    matches its source reports null rather than a stale figure."""
    for key, rec in bench.NCU_TRAFFIC.items():
        h = hashlib.sha256()
        for rel in rec["sources"]:
            path = os.path.join(ROOT, rel)
            assert os.path.exists(path), key
            with open(path, "rb") as f:
                h.update(f.read())
        current = h.hexdigest()
        value = bench.ncu_traffic(*key, "row_sweep")
        assert (value is not None) == (current == rec["sha256"]), key


def test_clock_sampler_parses_samples_after_mark():
    s = bench.ClockSampler(0)
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    # index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s.lines = ["0, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active"]  # idle, before mark
    s.mark()
    s.lines += [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_flags_thermal_slowdown():
    s = bench.ClockSampler(0)
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    s.mark()
    s.lines = ["0, 1500, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"]
    out = s.stop()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["sm_mhz"] == 1500.0
