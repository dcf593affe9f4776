"""bench.py's host logic: the clock record keeps the nvidia-smi samples taken
inside the timed region (else those within 0.25 s of it, else all), reports
the throttle reasons seen there, and the roofline fields follow from the
per-unit byte counts."""
import datetime
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(t, sm, cap="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, {sm}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}"


def test_clock_summary_keeps_the_timed_region():
    now = time.time()
    c = bench.ClockSampler(0)
    c.lines = [_line(now - 2.0, 1000), _line(now, 2070), _line(now + 0.05, 2060, "Active"),
               _line(now + 3.0, 500), "garbage", ""]
    c.t0, c.t1 = now - 0.01, now + 0.1
    s = c.summary()
    assert s["window"] == "timed region" and s["samples"] == 2
    assert s["sm_mhz"] == 2065.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    # a region between samples: the ones within 0.25 s of it
    c.t0, c.t1 = now + 0.2, now + 0.25
    s = c.summary()
    assert s["window"].startswith("within") and s["samples"] == 2
    # no sample near the region, or no region marked: all samples
    c.t0, c.t1 = now + 1.0, now + 1.1
    assert c.summary()["samples"] == 4
    c.t0 = c.t1 = None
    s = c.summary()
    assert s["window"] == "all samples" and s["sm_mhz"] == 1530.0


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_roofline_fields_follow_the_byte_counts():
    ncl, ns, npairs, nact = 1000, 3000, 3300, 2300
    algo = bench.ALGO_PAIRS(ncl, ns, npairs)
    assert algo == 56 * npairs + 8 * ns + 88 * ncl
    assert bench.ALGO_UPDATE(ncl, ns) == 240 * ncl + 8 * ns
    impl = bench.IMPL_PAIRS(ncl, ns, npairs, nact)
    r = bench.roof("k_pairs32", 2.0, algo=algo, impl=impl, peak=5000.0, peak_src="test",
                   full_bed=False)
    assert abs(r["achieved"] - algo / 2e-3 / 1e9) < 1e-12
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-15
    assert r["traffic"] is None and r["impl_bytes"] == impl
    # on a bed of the captured family the traffic scales with the algorithmic bytes
    r = bench.roof("k_pairs32", 2.0, algo=algo, impl=impl, peak=5000.0, peak_src="test",
                   full_bed=True)
    meas, algo_meas = bench.TRAFFIC["k_pairs32"]
    assert abs(r["traffic"] - meas * algo / algo_meas) < 1e-6
