"""Host logic of bench.py that needs no GPU: the clock-record parser and the recorded
DRAM-traffic lookup."""
import json

import pytest

import bench


def test_clock_parser_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1201.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 900.0, 0x0, Not Active, Active, Not Active, Not Active",
    ]
    out = bench.ClockSampler.parse(lines)
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2055.0          # median of the numeric SM clocks
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_parser_empty():
    out = bench.ClockSampler.parse([])
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    """The recorded DRAM bytes are returned, scaled to the grid, only while the hash of
    the listed sources matches the record; otherwise (or for an unknown kernel) None."""
    import hashlib
    src = tmp_path / "k.cuh"
    src.write_bytes(b"kernel source v1")
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"source": ["k.cuh"], "sha256": hashlib.sha256(b"kernel source v1").hexdigest(),
                 "bytes_per_launch_per_cell": 96.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k", 1024) == pytest.approx(96.0 * 1024 * 1024)
    assert bench.traffic_for("other", 1024) is None
    src.write_bytes(b"kernel source v2")
    assert bench.traffic_for("k", 1024) is None
