"""bench.py's clock record, on fake nvidia-smi lines (CPU): the median SM clock
and every throttle reason seen inside the timed region decide whether a run
stands, so the summary must read them from the right columns and samples."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

IDLE = "0x0000000000000000"


def _line(sm, mx=2070, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, clocks_event_reasons.active,
    # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return [x.strip() for x in f"0, {sm}, {mx}, 812.5, {IDLE}, {hw}, {hw_th}, {sw_th}, {cap}".split(",")]


def _sampler(samples, region=None):
    c = bench.ClockSampler(0)
    c.samples = samples
    if region:
        c.window(*region)
    return c.summary()


def test_median_clock_and_no_reason():
    s = _sampler([(t, _line(sm)) for t, sm in enumerate((2070, 2055, 2070, 2040, 2070))], (0, 4))
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == [] and s["samples"] == 5


def test_each_reason_is_read_from_its_column():
    for kw, name in (("hw", "hw_slowdown"), ("hw_th", "hw_thermal_slowdown"), ("sw_th", "sw_thermal_slowdown"),
                     ("cap", "sw_power_cap")):
        rows = [(0, _line(2070)), (1, _line(1800, **{kw: "Active"})), (2, _line(2070))]
        assert _sampler(rows, (0, 2))["reasons"] == [name]


def test_samples_outside_the_region_are_ignored():
    rows = [(0.0, _line(900, hw="Active"))] + [(1.0 + 0.1 * i, _line(2070)) for i in range(5)] + \
           [(9.0, _line(900, sw_th="Active"))]
    s = _sampler(rows, (1.0, 1.5))
    assert s["sm_mhz"] == 2070 and s["reasons"] == [] and s["samples"] == 5


def test_short_region_takes_the_three_nearest_samples():
    rows = [(0.0, _line(2070)), (1.0, _line(2070)), (1.02, _line(2070, cap="Active")), (5.0, _line(1000, hw="Active"))]
    s = _sampler(rows, (1.005, 1.01))
    assert s["samples"] == 3 and s["reasons"] == ["sw_power_cap"]


def test_no_samples_says_so():
    assert _sampler([])["reasons"] == ["nvidia-smi unavailable"]
