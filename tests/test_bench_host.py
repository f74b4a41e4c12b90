"""Host-side arithmetic of bench.py, no GPU: the roofline figures of the
dominant stage and the parsing of the clock samples taken during the timed
region."""
from __future__ import annotations

import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_of_takes_the_slowest_site_stage():
    """Six stages timed over 10 launches of 2**26 sites: the slowest stage
    that touches every site (stage 3, 2.3 ms in total) is the dominant one;
    achieved = 4 B/site * 2**26 sites / 0.23 ms."""
    names = [f"s{k}" for k in range(6)]
    stage_ms = [1.8, 1.0, 0.9, 2.3, 1.9, 9.9]     # stage 5 is not a site stage
    sites = 1 << 26
    r = bench.roofline_of(stage_ms, names, 10, sites, True, 6000.0, "measured")
    assert r["kernel"] == "s3" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["avg_launch_ms"] == pytest.approx(0.23)
    assert r["bytes_per_launch"] == 4.0 * sites
    assert r["achieved"] == pytest.approx(4.0 * sites / 0.23e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    t = bench.per_stage(bench.TRAFFIC_BYTES_PER_SITE, 3, 0)
    assert r["traffic"] is None if t is None else r["traffic"] == pytest.approx(t * sites)
    assert r["stage_ms_per_launch"]["s5"] == pytest.approx(0.99)
    # a stage whose entry does not depend on the layout
    r = bench.roofline_of([9.0, 1.0, 0.9, 2.3, 1.9, 0.1], names, 10, sites, True, 6000.0, "measured", patch=2)
    assert r["kernel"] == "s0" and r["traffic"] == pytest.approx(bench.TRAFFIC_BYTES_PER_SITE[0] * sites)


class _Done:
    """Stands in for the finished nvidia-smi sampler."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clocks_from(lines):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    c = bench.Clocks(0)
    c.proc, c.path = _Done(), path
    return c.stop()


def test_clock_samples_median_under_load_and_reasons():
    """Idle samples (below half the maximum clock) are left out of the median;
    a throttle reason counts when any sample shows it active."""
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 345, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = _clocks_from(rows)
    assert r["sm_mhz"] == 2040.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 4


def test_clock_samples_report_slowdowns_and_missing_data():
    rows = ["0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Active, Not Active"]
    r = _clocks_from(rows)
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and r["sm_mhz"] == 1500.0
    assert _clocks_from(["garbage"])["reasons"] == ["no samples"]
    assert bench.Clocks(0).stop()["reasons"] == ["unavailable"]
