"""The measured arithmetic ceilings (music_measure_peaks) are plausible for
the device: positive, FP32 FMA far faster than FP64 FMA on this part, and a
division slower than an FMA."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_measured_peaks_are_plausible():
    from paper_1610_10053_gb300 import binding as B
    pk = B.measure_peaks()
    assert pk["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.1 < pk["fp64_fma_tflops"] < 100.0
    assert pk["fp32_fma_tflops"] > 4 * pk["fp64_fma_tflops"]
    # one division costs more than one FMA (2 flops)
    assert pk["fp64_div_gops"] < 1e3 * pk["fp64_fma_tflops"] / 2
