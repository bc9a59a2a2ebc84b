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


def test_roofline_entries_and_traffic_guard(monkeypatch):
    """Per-shape roofline entries from summed solver stats; traffic is reported only for the
    kernel source its capture was taken on."""
    import bench
    st = {"spmm_calls_by_shape": [0] * 12, "spmm_ms_by_shape": [0.0] * 12, "spmm_bytes_by_shape": [0.0] * 12}
    st["spmm_calls_by_shape"][4], st["spmm_ms_by_shape"][4], st["spmm_bytes_by_shape"][4] = 5, 10.0, 5 * 3.5e9
    st["spmm_calls_by_shape"][3], st["spmm_ms_by_shape"][3], st["spmm_bytes_by_shape"][3] = 7, 7.0, 7 * 3.4e9
    pinfo = {"layout": 1, "layout_entries": 1000}
    monkeypatch.setattr(bench, "SPMM_TRAFFIC", {"kernel_sha": "not-this-source", "per_layout_entry": {4: 6.0}})
    ent = bench.roofline_entries(st, 7000.0, "measured", pinfo)
    assert [e["shape"] for e in ent] == ["FP32 vectors, nb 8", "FP32 vectors, nb 16"]
    e16 = ent[1]
    assert e16["launches"] == 5 and e16["avg_launch_ms"] == 2.0
    assert abs(e16["achieved"] - 3.5e9 / 2.0 / 1e6) < 1e-6 and abs(e16["frac"] - e16["achieved"] / 7000.0) < 1e-12
    assert e16["traffic"] is None                              # captured on another kernel source
    monkeypatch.setattr(bench, "SPMM_TRAFFIC", {"kernel_sha": bench.kernel_sha(), "per_layout_entry": {4: 6.0}})
    ent = bench.roofline_entries(st, 7000.0, "measured", pinfo)
    assert ent[1]["traffic"] == 6000.0 and ent[0]["traffic"] is None


def test_oracle_sample_measures_a_converged_oracle_solve():
    """The CPU legs' single model: the oracle hybrid on a leading block, on host threads."""
    import argparse
    import bench
    from gen import ci_matrix
    H = ci_matrix(12000, 60, 64, seed=1, storage="f32")
    args = argparse.Namespace(nb=8, nev=5, tol=1e-6, rmm_precond=1, switch_res=1e-2, switch_tau=0.0, s_max=10,
                              oracle_rows=3000, nnz_per_row=60, block_pattern=64, seed=1, storage="f32",
                              switch_gap=0.03)
    dt, r, Hs = bench.oracle_sample(H, args, 2)
    assert Hs.n == 3000 and dt > 0 and r.converged
    cb = bench.cpu_baseline(H, args)
    assert cb["cores"] >= 1 and cb["kind"] == "oracle" and cb["value"] > 0 and "n = 3,000" in cb["sample"]
