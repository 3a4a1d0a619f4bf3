"""Host logic of bench.py on CPU: the roofline denominators per precision and the parsing of
the nvidia-smi clock log that decides whether a timed run is kept."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


STATS = {"scatter_flops": 8.0e13, "ms_scatter": 100.0, "n_chunks": 10}


def test_fp32_roofline_uses_the_measured_simt_peak():
    probe = {"fp32": (70.0, "measured"), "fp64": (1.2, "measured")}
    r = bench.roofline_for("fp32", STATS, per_launch_traffic=1.0e9, simt_peaks=probe)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == 70.0 and r["peak_source"] == "measured"
    assert r["achieved"] == pytest.approx(8.0e13 / 0.1 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 70.0)
    assert bench.roofline_for("fp64", STATS, simt_peaks=probe)["peak"] == 1.2


def test_fp32_roofline_falls_back_to_the_derived_cuda_core_peak():
    r = bench.roofline_for("fp32", STATS, per_launch_traffic=1.0e9)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["achieved"] == pytest.approx(8.0e13 / 0.1 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == 1.0e9 and "k_scatter_sf" in r["kernel"]


def test_split_rooflines_use_the_bf16_peak_and_the_tf32_ratio():
    mp, _ = bench.peaks()
    a = bench.roofline_for("fp16x3", STATS)
    b = bench.roofline_for("tf32x3", STATS)
    assert a["bound"] == "tensor" and a["peak"] == pytest.approx(mp["bf16_tflops"])
    assert b["peak"] == pytest.approx(0.5 * mp["bf16_tflops"])
    # three split products per pair
    assert a["achieved"] == pytest.approx(3 * 8.0e13 / 0.1 / 1e12)


def test_fp64_roofline_is_the_fp64_alu_peak():
    r = bench.roofline_for("fp64", STATS)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(152 * 4 * 2.07e9 / 1e12)


def test_clock_log_summary(tmp_path):
    f = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 950.3, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1900, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 100.0, 0x8, Active, Not Active, Not Active, Not Active",   # other GPU
    ]
    f.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(str(f))
    s = cs.summary(0)
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]                   # noted, not a reject
    assert bench.ClockSampler(str(tmp_path / "missing.csv")).summary(0)["reasons"] == ["unsampled"]
