"""The multiply-add throughput probe (fsmc_probe_fma_peaks) through the C ABI: it runs on the
device and returns rates of the right order against the B300's unit counts (148 SMs x 128 FP32
lanes x 2 flops per clock, at most 77 TFLOP/s at 2032 MHz; FP64 a small fraction of that)."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_returns_plausible_fma_rates():
    import torch
    from paper_2503_17405_b300 import build, fsmc
    build.build()
    torch.cuda.set_device(0)
    f32, f64 = fsmc.probe_fma_peaks(0)
    print("FFMA %.1f TFLOP/s, DFMA %.2f TFLOP/s" % (f32, f64))
    assert 20.0 < f32 < 85.0
    assert 0.05 < f64 < f32
    assert torch.cuda.current_device() == 0


def test_probe_rejects_null_outputs():
    import ctypes
    from paper_2503_17405_b300 import fsmc
    st = fsmc.load().fsmc_probe_fma_peaks(0, None, None)
    assert st == fsmc.EINVAL
