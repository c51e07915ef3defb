"""bench.py's clock summary: only the nvidia-smi samples inside the timed region count, throttle
reasons are collected from them, and a window with no sample falls back to all samples."""
import datetime

import pytest

import bench


def _row(t, sm, hw="Not Active", cap="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, 2070, 900.00, 0x0, {hw}, Not Active, Not Active, {cap}\n"


def test_samples_inside_the_timed_window(tmp_path):
    p = tmp_path / "clocks.csv"
    t0 = 1_800_000_000.0
    p.write_text(_row(t0 - 1.0, 1000, hw="Active") + _row(t0 + 0.02, 2070) + _row(t0 + 0.07, 2055, cap="Active")
                 + _row(t0 + 2.0, 500))
    c = bench.ClockSampler(0, path=str(p))
    c.mark(t0, t0 + 0.1)
    s = c.summary(running=False)
    assert s["samples"] == 2
    assert s["sm_mhz"] == pytest.approx(2062.5)
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_no_sample_in_window_uses_all(tmp_path):
    p = tmp_path / "clocks.csv"
    t0 = 1_800_000_000.0
    p.write_text(_row(t0 - 5.0, 2070) + _row(t0 + 5.0, 2040))
    c = bench.ClockSampler(0, path=str(p))
    c.mark(t0, t0 + 0.1)
    s = c.summary(running=False)
    assert s["samples"] == 2 and s["reasons"] == []
