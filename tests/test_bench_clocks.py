"""bench.py's clock record on the CPU: the nvidia-smi samples stamped inside
the timed region are the ones counted, their median SM clock and every
throttle reason active in them are reported (a run that saw hw_slowdown,
hw_thermal_slowdown or sw_thermal_slowdown is rejected by the contract, so
these must not be lost), and a region shorter than the sampling interval
takes the nearest sample."""
from __future__ import annotations

import datetime
import importlib.util
import os
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def row(ts, mhz, reasons=("Not Active",) * 4):
    return ", ".join([ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], "0", str(mhz), "2070", "812.5",
                      "0x0000000000000000", *reasons]) + "\n"


def sampler_with(rows, t0, t1):
    bench = load_bench()
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.writelines(rows)
    s.proc = FakeProc()
    s.t0, s.t1 = t0, t1
    return s


def test_samples_inside_region_and_reasons():
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    at = lambda ms: base + datetime.timedelta(milliseconds=ms)
    rows = [row(at(0), 1500, ("Active", "Not Active", "Not Active", "Not Active")),  # before the region
            row(at(100), 2070),
            row(at(150), 2055, ("Not Active", "Not Active", "Not Active", "Active")),
            row(at(200), 2070),
            row(at(400), 1200, ("Not Active", "Active", "Not Active", "Not Active"))]  # after it
    rec = sampler_with(rows, at(90), at(210)).stop()
    assert rec["samples_in_region"] == 3 and rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_thermal_reason_inside_region_is_reported():
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    at = lambda ms: base + datetime.timedelta(milliseconds=ms)
    rows = [row(at(100), 1900, ("Not Active", "Not Active", "Active", "Not Active")),
            row(at(150), 1950, ("Active", "Active", "Not Active", "Not Active"))]
    rec = sampler_with(rows, at(50), at(200)).stop()
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1925.0


def test_short_region_takes_nearest_sample():
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    at = lambda ms: base + datetime.timedelta(milliseconds=ms)
    rows = [row(at(0), 2000), row(at(50), 2070), row(at(100), 1800)]
    rec = sampler_with(rows, at(52), at(58)).stop()
    assert rec["samples_in_region"] == 0 and rec["samples"] == 1
    assert rec["sm_mhz"] == 2070.0
