"""CPU checks of bench.py's host side: the clock-record summary that decides
whether a run is kept (throttle reasons, median SM clock), and the JSON line
of the reference arm (the oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_median_max_and_reasons():
    quiet = "0, 2070, 2070, 910.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1200.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    s = _sampler([quiet, quiet, capped])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s = _sampler([quiet, hot, hot])
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_thermal_slowdown"]
    # unparsable lines (a driver message) are skipped; no sample at all says so
    s = _sampler(["No devices were found", quiet])
    assert s["samples"] == 1 and s["reasons"] == []
    assert _sampler([])["reasons"] == ["unavailable"]


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` times the oracle on the host cores and
    prints the contract's line (here with 1 timed step, to check its shape)."""
    pytest.importorskip("torch")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "FP64 cell-steps/s per GB300" and d["unit"] == "cell-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["config"]["workload"] == "h2air_detonation_tube_4096x512_9sp19r_cfl0.5"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
