"""The device's FMA throughput (md_measure_fma_peak), the denominator of the triplet kernel's roofline
fraction: plausible against the FP32 lanes and clock the device reports, and FP64 far below FP32."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible(gpu_lib):
    import torch
    props = torch.cuda.get_device_properties(0)
    f32, ms = gpu_lib.md_measure_fma_peak(0, 20.0)
    f32x2, _ = gpu_lib.md_measure_fma_peak(1, 20.0)
    f64, _ = gpu_lib.md_measure_fma_peak(2, 20.0)
    assert ms >= 20.0
    # 128 FP32 lanes per SM, 2 flop per FMA, at most a 2.2 GHz clock
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9
    assert 0.3 * ceiling < max(f32, f32x2) <= 1.02 * ceiling
    assert 0.0 < f64 < 0.5 * max(f32, f32x2)
