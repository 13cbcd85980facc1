"""bench.py's clock record: the nvidia-smi samples taken during the timed
region are summarised as the median SM clock under load, the maximum clock,
and every throttle reason that was active in any sample."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c


def test_summary_of_clean_samples():
    lines = [f"0, {mhz}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
             for mhz in (2070, 2070, 2055, 2070, 2070)]
    s = _sampler(lines).summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_summary_reports_every_active_reason():
    lines = ["0, 1800, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 1500, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
             "0, 1900, 2070, 1300.0, 0x0, Not Active, Not Active, Active, Not Active",
             "garbage line", "0, [N/A], 2070, 1, 0, a, b, c, d"]
    s = _sampler(lines).summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 1800.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_summary_without_samples():
    assert _sampler([]).summary()["reasons"] == ["unsampled"]
