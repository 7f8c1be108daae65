"""bench.py's clock record, from nvidia-smi lines given as text (no GPU, no
nvidia-smi): the median SM clock under load, the maximum, the throttle reasons
that were active, and only the samples taken from the start of the timed
region on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, mx=2070, power=900.0, cap="Not Active", thermal="Not Active"):
    return "0, %s, %s, %s, 0x0, Not Active, %s, Not Active, %s" % (sm, mx, power, thermal, cap)


def test_summary_of_the_timed_samples():
    c = bench.ClockSampler(0)
    c.lines = [_line(345, thermal="Active")]  # before the timed region: ignored
    c.first = len(c.lines)
    c.lines += [_line(1980), _line(2010, cap="Active"), "garbled", _line("[N/A]"), _line(1995)]
    s = c.summary()
    assert s == {"sm_mhz": 1995.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}


def test_thermal_reasons_are_reported():
    c = bench.ClockSampler(0)
    c.lines = [_line(1500, thermal="Active"), _line(1520)]
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_no_samples_without_nvidia_smi():
    c = bench.ClockSampler(0)
    c.ready(timeout_s=0.1)  # no process: returns at once
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
