"""The bench line's roofline arithmetic on a synthetic kernel-class profile (CPU).

achieved = algorithmic work / event-measured time, frac = achieved / peak,
traffic = measured DRAM-to-algorithmic ratio x mean algorithmic bytes per
launch; the dominant single-kernel class is the one with the largest time.
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..")))
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1500.0, "sm_max_mhz": 2000.0}


def _entry(name, ms, launches, flops=0.0, bytes_=0.0, issued=0.0):
    return {"name": name, "total_ms": ms, "launches": launches, "flops": flops, "bytes": bytes_,
            "issued_flops": issued}


def test_tensor_class_roofline():
    prof = [_entry("batch_tc", 200.0, 100, flops=4.0e12, bytes_=100 * 4.0 * 1024 ** 2, issued=8.0e12),
            _entry("eig_tridiag", 150.0, 5, flops=1e12),
            _entry("event_row_fp64", 900.0, 50),     # spans several kernels: never the roofline class
            _entry("ingest", 10.0, 100, bytes_=1e9)]
    r = bench.roofline(prof, PEAKS, "measured")
    assert r["kernel"] == "batch_tc" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(4.0e12 / 0.2 / 1e12)          # 20 TFLOP/s
    assert r["frac"] == pytest.approx(20.0 / 1500.0)
    assert r["avg_launch_us"] == pytest.approx(2000.0)
    ratio = bench.TRAFFIC_RATIO["batch_tc"]
    assert r["traffic"] == pytest.approx(ratio * 4.0 * 1024 ** 2)
    assert r["issued_frac"] == pytest.approx(2.0 * r["frac"])
    assert r["algorithmic_flops_per_launch"] == pytest.approx(4.0e10)


def test_df64_and_fp32_peaks():
    fp32 = bench.N_SM * bench.FP32_SIMT_LANES_PER_SM * 2 * 2000.0e6 / 1e12
    r = bench.roofline([_entry("eig_tridiag", 30.0, 1, flops=3e11)], PEAKS, "measured")
    assert r["bound"] == "alu" and r["traffic"] is None
    assert r["peak"] == pytest.approx(fp32 / bench.DF64_FP32_OPS_PER_FMA)
    assert r["achieved"] == pytest.approx(10.0)
    r = bench.roofline([_entry("batch_persist", 10.0, 2, flops=1e11)], PEAKS, "measured")
    assert r["peak"] == pytest.approx(fp32) and r["achieved"] == pytest.approx(10.0)


def test_hbm_class():
    r = bench.roofline([_entry("ingest", 2.0, 4, bytes_=12e9)], PEAKS, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(6000.0) and r["frac"] == pytest.approx(1.0)
