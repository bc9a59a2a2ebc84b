"""Host-side logic of bench.py that needs no GPU: the clock sampler's summary of nvidia-smi lines
(median SM clock under the timed region, throttle reasons that reject a run)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, reasons=("Not Active",) * 4):
    return ", ".join(["0", str(sm), "2070", "700.5", "0x0000000000000000", *reasons])


def test_clock_summary_median_and_no_reason():
    c = bench.ClockSampler(0)
    c.lines = [_line(2070), _line(2040), _line(2070)]
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == [] and s["samples"] == 3


def test_clock_summary_reports_throttle_reasons():
    c = bench.ClockSampler(0)
    c.lines = [_line(1500, ("Not Active", "Active", "Not Active", "Active")), _line(1600)]
    s = c.summary()
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1550


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.lines = ["garbage", ""]
    assert c.summary()["reasons"] == ["unsampled"]


def test_workload_config_names_the_workload(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()          # the defaults: the n = 2M hybrid workload

    class H:
        n = 2_000_000
        nnz = 402_797_883
    cfg = bench.workload_config(args, H)
    assert "n=2,000,000" in cfg["workload"] and "residual 0.01" in cfg["workload"]
    assert cfg["n_ev"] == 8 and cfg["block"] == 16 and cfg["parallelism"] == "single GPU"
