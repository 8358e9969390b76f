"""bench.py's clock record (host logic, no GPU): which nvidia-smi samples
describe the timed region, and which throttle reasons it reports."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

T0 = datetime.datetime(2026, 12, 4, 10, 0, 0)


def _line(dt_s, sm, reasons=()):
    ts = (T0 + datetime.timedelta(seconds=dt_s)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if r in reasons else "Not Active" for r in bench._CLOCK_REASONS]
    return ", ".join([ts, "0", str(sm), "2070", "900.5", "0x0000000000000000"] + flags)


def _t(dt_s):
    return (T0 + datetime.timedelta(seconds=dt_s)).timestamp()


def test_samples_inside_the_region_decide():
    lines = [_line(0.0, 1400, {"hw_slowdown"}), _line(0.1, 2070), _line(0.2, 2070),
             _line(0.3, 2055), _line(0.4, 1000, {"sw_thermal_slowdown"})]
    r = bench.parse_clock_samples(lines, _t(0.05), _t(0.35))
    assert r["samples"] == 3 and r["sampled"] == "inside the timed region"
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == []


def test_reasons_active_inside_the_region_are_reported():
    lines = [_line(0.0, 2070), _line(0.1, 1900, {"sw_power_cap"}), _line(0.2, 1800, {"hw_slowdown"}),
             _line(0.3, 2070)]
    r = bench.parse_clock_samples(lines, _t(0.05), _t(0.25))
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert r["sm_mhz"] == 1850


def test_short_region_uses_the_neighbouring_samples():
    lines = [_line(0.0, 2070), _line(0.1, 2040), _line(0.2, 1500, {"hw_thermal_slowdown"}),
             _line(0.3, 2070)]
    r = bench.parse_clock_samples(lines, _t(0.12), _t(0.18))   # 60 ms, no sample inside
    assert r["samples"] == 2 and r["sampled"].startswith("adjacent")
    assert r["sm_mhz"] == (2040 + 1500) / 2
    assert r["reasons"] == ["hw_thermal_slowdown"]


def test_without_region_or_timestamps_every_sample_counts():
    lines = [_line(0.0, 2000), _line(0.1, 2070)]
    r = bench.parse_clock_samples(lines)
    assert r["samples"] == 2 and r["sampled"] == "all samples"
    bad = [", ".join(["not a time"] + ln.split(", ")[1:]) for ln in lines]
    r = bench.parse_clock_samples(bad, _t(0.0), _t(0.05))
    assert r["samples"] == 2 and r["sampled"] == "all samples"


def test_no_usable_line():
    r = bench.parse_clock_samples(["garbage", "", "a, b, c"], _t(0), _t(1))
    assert r["samples"] == 0 and r["reasons"] == ["unsampled"]
