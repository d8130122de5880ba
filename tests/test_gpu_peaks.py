"""Calibration of the ALU roofline: measured FMA throughput against the
derived figure (SMs x 128 FP32 lanes x 2 flop x clock)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_measured_fp32_peak_is_near_the_derived_one(gpu):
    f32, f64 = gpu.measure_peaks(0)
    props = torch.cuda.get_device_properties(0)
    # a GB300 SM runs at most 2070 MHz; the loaded clock may sit below it
    derived = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.5 * derived < f32 <= 1.02 * derived
    assert 0.0 < f64 < f32


def test_measure_peaks_rejects_null_outputs(gpu):
    assert gpu.nb_measure_peaks(0, None, None) == gpu.NB_EINVAL
