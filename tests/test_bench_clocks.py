"""Host logic of bench.py that decides whether a timed run is kept: the
nvidia-smi clock sampler's parsing (median SM clock under load, maximum
clock, throttle reasons seen) and the whole-job rate over replicas."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def parse(lines):
    c = bench.Clocks(0)
    c.proc = DoneProc()
    c.lines = list(lines)
    return c.stop()


def row(sm, smax=2070, active="0x0", hw="Not Active", hwt="Not Active", swt="Not Active",
        cap="Not Active"):
    return f"0, {sm}, {smax}, 1100.5, {active}, {hw}, {hwt}, {swt}, {cap}"


def test_median_clock_and_no_reasons():
    r = parse([row(2070), row(2055), row(1980), row(2070), row(2070)])
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == [] and r["samples"] == 5


def test_reasons_are_collected_once_each():
    r = parse([row(1800, cap="Active"), row(1700, hwt="Active", cap="Active"), row(2070)])
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert r["sm_mhz"] == 1800


def test_malformed_and_short_lines_are_skipped():
    r = parse(["", "garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, "
               "Not Active", row(2000)])
    assert r["samples"] == 1 and r["sm_mhz"] == 2000


def test_without_nvidia_smi():
    c = bench.Clocks(0)
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def test_job_rate_sums_replicas_over_slowest_rank():
    # 30 steps on each of 4 replicas, slowest rank 600 ms: 200 iterations/s
    assert bench.job_rate(30, 4, 600.0) == 200.0
    assert bench.job_rate(30, 1, 600.0) == 50.0
