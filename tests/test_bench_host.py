"""Host logic of bench.py's JSON line, without a GPU: the roofline object of
each kind of dominant kernel class (HBM-bound update, tensor-bound product,
ALU-bound panel), the measured peaks taken from the peaks file when present,
and the DRAM traffic reported only for a class (and precision) whose ncu
capture is on record."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"hbm_gbs": 6786.6, "bf16_tflops": 1885.6, "bf16_tflops_sustained": 1689.9, "sm_max_mhz": 2070.0}


def _dom(name, ms=1000.0, gbytes=4000.0, tflop=500.0, launches=500):
    return {"name": name, "ms": ms, "bytes": gbytes * 1e9, "flops": tflop * 1e12, "launches": launches}


def test_update_class_is_hbm_bound_with_its_captured_traffic(bench):
    dom = _dom("tc_update")
    r = bench.roofline(dom, "f16x3", 4000.0, PEAKS)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == PEAKS["hbm_gbs"]
    assert r["achieved"] == pytest.approx(4000.0)  # 4000 GB in 1 s
    assert r["frac"] == pytest.approx(4000.0 / PEAKS["hbm_gbs"])
    assert r["share_of_step"] == pytest.approx(0.25)
    ratio = bench.TRAFFIC_RATIO[("tc_update", "f16x3")]["ratio"]
    assert 0.5 < ratio < 1.5
    assert r["traffic"] == pytest.approx(ratio * dom["bytes"] / dom["launches"])
    assert r["tensor_rate"]["peak"] == PEAKS["bf16_tflops_sustained"]


def test_traffic_is_null_without_a_capture_of_that_kernel(bench):
    # the TF32 update is another kernel than the FP16-split one captured
    assert bench.roofline(_dom("tc_update"), "tf32", 4000.0, PEAKS)["traffic"] is None
    assert bench.roofline(_dom("tc_gemm"), "f16x3", 4000.0, PEAKS)["traffic"] is None


def test_product_class_is_tensor_bound_against_the_precisions_peak(bench):
    r = bench.roofline(_dom("tc_gemm"), "f16x3", 4000.0, PEAKS)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(500.0)
    assert r["peak"] == PEAKS["bf16_tflops_sustained"]
    r = bench.roofline(_dom("tc_gemm"), "tf32", 4000.0, PEAKS)
    assert r["peak"] == bench.TF32_MEASURED_TFLOPS


def test_panel_class_is_alu_bound_against_the_derived_fp64_peak(bench):
    r = bench.roofline(_dom("panel_qr", tflop=0.5), "f16x3", 4000.0, PEAKS)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(0.5 / r["peak"])


def test_fallback_peaks_without_the_peaks_file(bench):
    r = bench.roofline(_dom("tc_update"), "f16x3", 4000.0, {})
    assert r["peak"] == 6800.0 and "fallback" in r["peak_source"]
