"""Host logic of the bench's roofline line (no GPU): the dominant class, the
algorithmic rate against the derived peak, and the DRAM traffic figure,
which comes from a one-launch capture of the bench workload itself, from
the per-cell figure of the 2048^2 capture on other grids, or is withheld for
a kernel that changed since its capture."""
import importlib.util
import os

import pytest

from paper_1610_10053_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def classes(res_ms, pc_ms=0.63, jv_ms=0.58):
    return {"kernels": {"jv": {"ms_per_step": jv_ms, "ms_per_launch": jv_ms / 15, "launches": 150},
                        "precond": {"ms_per_step": pc_ms, "ms_per_launch": pc_ms / 15, "launches": 150},
                        "residual": {"ms_per_step": res_ms, "ms_per_launch": res_ms / 6, "launches": 60},
                        "vector": {"ms_per_step": 5.0, "ms_per_launch": 0.01, "launches": 850},
                        "unattributed": {"ms_per_step": 0.05}}}


def test_dominant_class_and_rate(bench):
    p = I.kelvin_helmholtz(n=512)
    r = bench.roofline(classes(1.02), p, "diff")
    # the vector class has no single roofline even when it takes the most time
    assert r["class"] == "residual" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    per_s = (1.02 / 6) / 1e3
    assert r["achieved"] == pytest.approx(bench.RES_FLOPS_PER_CELL_2D * p.ncells / per_s / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)


def test_traffic_sources(bench):
    p = I.kelvin_helmholtz(n=512)
    pc = bench.roofline(classes(0.1), p, "diff")
    assert pc["class"] == "precond" and pc["traffic"] == bench.TRAFFIC_KH512["precond"]
    res = bench.roofline(classes(1.02), p, "diff")
    assert res["traffic"] == bench.TRAFFIC_KH512["residual"]
    if res["traffic"] is None:
        assert "changed" in res["traffic_note"]
    big = I.kelvin_helmholtz(n=64)  # not the bench grid: the 2048^2 per-cell figure, scaled
    res = bench.roofline(classes(1.02), big, "diff")
    assert res["traffic"] == pytest.approx(bench.RES_TRAFFIC_B_PER_CELL_2D * big.ncells)


def test_fp64_form_product_uses_the_fp64_peak(bench):
    p = I.kelvin_helmholtz(n=512)
    r = bench.roofline(classes(0.1, pc_ms=0.1, jv_ms=2.0), p, "fd")
    assert r["class"] == "jv" and r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    r = bench.roofline(classes(0.1, pc_ms=0.1, jv_ms=2.0), p, "diff")
    assert r["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS)
    assert r["traffic"] == bench.TRAFFIC_KH512["jv"]


def test_job_rate_and_clock_summary(bench):
    # replicas: every rank's cell-steps over the slowest rank's time
    assert bench.job_rate(4, 1000, 10, 2000.0) == pytest.approx(4 * 1000 * 10 / 2.0)
    cs = bench.ClockSampler(0)
    cs.lines = ["2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                "1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "garbage",
                "2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_measured_alu_peak_is_the_denominator(bench):
    """With the FMA throughput measured in the run (music_measure_peaks), the
    FP64 residual's fraction is taken against the measured FP64 figure; the
    unit-count figure is kept in the note only."""
    p = I.kelvin_helmholtz(n=512)
    alu = {"fp64_fma_tflops": 1.058, "fp32_fma_tflops": 76.3, "fp64_div_gops": 61.4, "sms": 152}
    r = bench.roofline(classes(1.02), p, "diff", alu)
    assert r["peak"] == pytest.approx(1.058)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.058)
    assert "measured" in r["peak_note"] and r["measured_alu_peaks"] == alu
    # the FP32 product's class uses the FP32 figure
    r = bench.roofline(classes(0.1, jv_ms=2.0), p, "diff", alu)
    assert r["class"] == "jv" and r["peak"] == pytest.approx(76.3)
