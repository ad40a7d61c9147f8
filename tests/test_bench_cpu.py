"""bench.py's measurement arithmetic on synthetic launch records (no GPU):
the dominant kernel family, its achieved rate from algorithmic work per
launch over the average launch time, and the roof it is judged against."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_alu_bound_family_is_judged_against_the_double_float_roof():
    pk = {"hbm_gbs": 6000.0}
    # 4 launches of 20 ms, each 34.36 GB and 120 Tflop of algorithmic work; plus a smaller family
    recs = [("k_seg/df", 20.0, 34.36e9, 120e12)] * 4 + [("k_gate/df", 5.0, 34.36e9, 6e9 * 1024 ** 3 / 1e9)] * 2
    out, fams = bench.roofline(recs, pk)
    assert out["kernel"] == "k_seg/df" and out["launches"] == 4
    assert out["bound"] == "alu" and out["unit"] == "TFLOP/s"
    tfl = 120e12 / 20e-3 / 1e12
    assert out["achieved"] == pytest.approx(tfl)
    assert out["peak"] == pytest.approx(bench.ALU_PEAK_TFLOPS["df"])
    assert out["frac"] == pytest.approx(tfl / bench.ALU_PEAK_TFLOPS["df"])
    assert out["hbm_frac_of_measured"] == pytest.approx(34.36e9 / 20e-3 / 1e9 / 6000.0)
    assert out["share"] == pytest.approx(80.0 / 90.0)
    assert out["ms_per_launch"] == pytest.approx(20.0) and out["bytes_per_launch"] == pytest.approx(34.36e9)
    assert out["traffic"] is None  # no ncu capture is stored for this family
    assert fams["k_gate/df"]["launches"] == 2 and fams["k_gate/df"]["GBps"] == pytest.approx(34.36e9 / 5e-3 / 1e9, rel=1e-3)


def test_memory_bound_family_is_judged_against_measured_hbm():
    pk = {"hbm_gbs": 6691.5}
    recs = [("k_dense1r/df", 5.4, 2 * 17.18e9, 6 * 2 ** 30)] * 3
    out, _ = bench.roofline(recs, pk)
    assert out["bound"] == "hbm" and out["unit"] == "GB/s"
    assert out["achieved"] == pytest.approx(2 * 17.18e9 / 5.4e-3 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 6691.5)
    assert "MEASURED_PEAKS" in out["peak_source"]


def test_derived_double_float_peak():
    # 152 SMs x 128 FP32 lanes x 2.07 GHz, 32 instructions per 6 float64-equivalent flops
    assert bench.ALU_PEAK_TFLOPS["df"] == pytest.approx(152 * 128 * 2.07e9 * 6 / 32 / 1e12)


def test_replicas_value_is_whole_job_throughput():
    assert bench.replicas_value(1490, 1, 1.5) == pytest.approx(1490 / 1.5)
    assert bench.replicas_value(1490, 8, 1.5) == pytest.approx(8 * 1490 / 1.5)


def test_traffic_of_the_dominant_kernel():
    pk = {"hbm_gbs": 6691.5}
    name = "k_fused_reg_jit/df"
    out, _ = bench.roofline([(name, 20.0, 34.36e9, 120e12)], pk)
    t = bench.TRAFFIC[name]
    assert out["traffic_source"] == t["source"]
    if t.get("changed_since"):
        assert out["traffic"] is None and out["traffic_last_capture"] == t["bytes_per_launch"]
    else:
        assert out["traffic"] == t["bytes_per_launch"]
    out, _ = bench.roofline([(name, 20.0, 34.36e9, 120e12)], pk, traffic=1.5e9)
    assert out["traffic"] == 1.5e9
