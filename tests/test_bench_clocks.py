"""The clock record of bench.py: nvidia-smi samples are kept when their
timestamps fall inside the timed region, with every throttle reason seen."""
import datetime
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module",
                                                  os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def line(ts, sm, reasons=()):
    flags = ["Active" if n in reasons else "Not Active"
             for n in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                       "sw_power_cap")]
    return ", ".join([ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], "0", str(sm), "2070",
                      "900.5", "0x0"] + flags) + "\n"


def test_samples_inside_the_timed_region_only(bench):
    t = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    ms = datetime.timedelta(milliseconds=1)
    lines = [line(t + k * 50 * ms, 1200 if k < 3 else 2070,
                  ("hw_slowdown",) if k == 1 else ()) for k in range(10)]
    # the region covers samples 4..7 (idle samples 0..2 and a slowdown before it)
    out = bench.summarize_clock_samples(lines, t + 190 * ms, t + 360 * ms)
    assert out["window"] == "timed region"
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == []


def test_reasons_in_the_region_are_reported(bench):
    t = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    ms = datetime.timedelta(milliseconds=1)
    lines = [line(t + k * 50 * ms, 2070, ("sw_power_cap",) if k == 2 else ())
             for k in range(5)]
    out = bench.summarize_clock_samples(lines, t, t + 200 * ms)
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 5


def test_short_region_falls_back_to_the_whole_run(bench):
    t = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    ms = datetime.timedelta(milliseconds=1)
    lines = [line(t + k * 50 * ms, 2000 + k) for k in range(3)] + ["garbage\n", "\n"]
    out = bench.summarize_clock_samples(lines, t + 10 * ms, t + 20 * ms)
    assert out["window"] == "run" and out["samples"] == 3 and out["sm_mhz"] == 2001
    assert bench.summarize_clock_samples([], None, None)["reasons"] == ["no samples"]
