"""Host logic of bench.py that needs no GPU: the clock-record parser, the recorded
DRAM-traffic lookup and the reference arm (the oracle timed on the host)."""
import json
import os

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


def _run_bench(args, env_extra=None):
    import os
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args, capture_output=True,
                         text=True, timeout=600, env=env, cwd=bench.ROOT)
    return out


def test_reference_arm_prints_the_contract_line():
    """`--impl reference` times the oracle on the named workload and prints one JSON line
    with the contract's keys (here on a 64^2 grid to keep it short)."""
    out = _run_bench(["--impl", "reference", "--size", "64", "--steps", "2", "--warmup", "1"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] >= 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and "64x64" in d["config"]["workload"]
    cpu = d["cpu_baseline"]
    # the oracle's OpenMP build on every host core
    assert cpu["kind"] == "oracle" and cpu["cores"] == (os.cpu_count() or 1) and cpu["value"] == d["value"]
    assert cpu["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    out = _run_bench(["--impl", "reference", "--size", "64", "--steps", "1", "--warmup", "0"], {"RANK": "1"})
    assert out.returncode == 0 and not out.stdout.strip()
