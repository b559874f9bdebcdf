"""Host logic of bench.py (no GPU): the clock record it attaches to the JSON
line, the derived FP64 peak, and the reference arm, which runs the CPU oracle
and prints the contract's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _DoneProc:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _row(mhz, max_mhz, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", power="Not Active"):
    return ["0", str(mhz), str(max_mhz), "900.5", "0x0", hw, thermal, sw_thermal, power]


def test_clock_record_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.proc = _DoneProc()
    s.rows = [_row(2070, 2070), _row(1980, 2070, power="Active"), _row(2070, 2070), ["garbled"],
              _row(1500, 2070, thermal="Active")]
    rec = s.stop()
    assert rec["sm_mhz"] == pytest.approx(2025.0)  # median of 2070, 1980, 2070, 1500
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert rec["samples"] == 4


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_derived_fp64_peak():
    # 152 SMs x 2 FP64 instructions per clock x 2070 MHz
    assert bench.fp64_peak({"sm_max_mhz": 2070.0}) == pytest.approx(0.62928e12)
    assert bench.fp64_peak({}) == pytest.approx(0.62928e12)


def test_reference_arm_prints_the_contract_line():
    """One step of the reference arm: one complete oracle solve of the bench
    problem at 33^3 nodes, timed on the host."""
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600, check=True)
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "s" and line["higher_is_better"] is False
    assert line["value"] > 0 and line["ms_per_step"] == pytest.approx(1e3 * line["value"])
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the oracle solve converges like the GPU arm's (5 Newton steps at 33^3)
    assert "5 Newton" in line["cpu_baseline"]["sample"]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120, check=True)
    assert out.stdout.strip() == ""
