"""bench.py's measurement arithmetic on synthetic launch records (no GPU):
the dominant kernel family, its achieved rate from algorithmic work per
launch over the average launch time, the measured HBM peak it is judged
against, and the traffic figure's tie to the sources it was captured from."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_dominant_family_is_judged_against_measured_hbm():
    pk = {"hbm_gbs": 6000.0}
    # 4 launches of 20 ms, each 34.36 GB and 120 Tflop of algorithmic work; plus a smaller family
    recs = [("k_seg/df", 20.0, 34.36e9, 120e12)] * 4 + [("k_gate/df", 5.0, 34.36e9, 6e9 * 1024 ** 3 / 1e9)] * 2
    out, fams = bench.roofline(recs, pk, 30)
    assert out["kernel"] == "k_seg/df" and out["launches"] == 4
    assert out["bound"] == "hbm" and out["unit"] == "GB/s" and out["peak"] == 6000.0
    gbs = 34.36e9 / 20e-3 / 1e9
    assert out["achieved"] == pytest.approx(gbs)
    assert out["frac"] == pytest.approx(gbs / 6000.0)
    assert "measured" in out["peak_source"]
    # the double-float figure is secondary and labelled as derived from the code's own instruction count
    alu = out["alu_derived"]
    tfl = 120e12 / 20e-3 / 1e12
    assert alu["achieved_f64eq_tflops"] == pytest.approx(tfl)
    assert alu["figure_tflops"] == pytest.approx(bench.ALU_PEAK_TFLOPS["df"])
    assert alu["frac"] == pytest.approx(tfl / bench.ALU_PEAK_TFLOPS["df"])
    assert "not a chip peak" in alu["basis"]
    assert out["share"] == pytest.approx(80.0 / 90.0)
    assert out["ms_per_launch"] == pytest.approx(20.0) and out["bytes_per_launch"] == pytest.approx(34.36e9)
    assert out["traffic"] is None  # no ncu capture is stored for this family
    assert fams["k_gate/df"]["launches"] == 2 and fams["k_gate/df"]["GBps"] == pytest.approx(34.36e9 / 5e-3 / 1e9, rel=1e-3)


def test_fallback_peak_is_named():
    out, _ = bench.roofline([("k_dense1r/df", 5.4, 2 * 17.18e9, 6 * 2 ** 30)] * 3, {}, 30)
    assert out["peak"] == 6800.0 and "fallback" in out["peak_source"]


def test_derived_double_float_figure():
    # 152 SMs x 128 FP32 lanes x 2.07 GHz, 32 instructions per 6 float64-equivalent flops
    assert bench.ALU_PEAK_TFLOPS["df"] == pytest.approx(152 * 128 * 2.07e9 * 6 / 32 / 1e12)


def test_replicas_value_is_whole_job_throughput():
    assert bench.replicas_value(1490, 1, 1.5) == pytest.approx(1490 / 1.5)
    assert bench.replicas_value(1490, 8, 1.5) == pytest.approx(8 * 1490 / 1.5)


def test_traffic_is_scaled_and_tied_to_the_captured_sources(monkeypatch):
    pk = {"hbm_gbs": 6691.5}
    name = "k_fused_reg_jit/df"
    t = dict(bench.TRAFFIC[name])
    scaled = (t["read"] + t["write"]) * 2.0 ** (30 - t["capture_qubits"])
    # sources as captured: the figure is reported, scaled to a 30-qubit launch
    monkeypatch.setitem(bench.TRAFFIC, name, dict(t, sha=bench.sources_digest(t["files"])))
    out, _ = bench.roofline([(name, 20.0, 34.36e9, 120e12)], pk, 30)
    assert out["traffic"] == pytest.approx(scaled)
    assert t["source"] in out["traffic_source"]
    # sources changed since the capture: null, with the old figure beside it
    monkeypatch.setitem(bench.TRAFFIC, name, dict(t, sha="0" * 16))
    out, _ = bench.roofline([(name, 20.0, 34.36e9, 120e12)], pk, 30)
    assert out["traffic"] is None and out["traffic_last_capture"] == pytest.approx(scaled)
    assert "retake" in out["traffic_note"]


def test_sources_digest_changes_with_content(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    a.write_text("x")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d1 = bench.sources_digest(["a.cu"])
    a.write_text("y")
    assert bench.sources_digest(["a.cu"]) != d1 and len(d1) == 16
