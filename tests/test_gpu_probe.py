"""The benchmark's throughput probe (libfsmc_probe.so, not part of the C ABI) runs on the device
and returns rates of the right order against the B300's unit counts: 148 SMs x 128 FP32 lanes x 2
flops per clock (at most 77 TFLOP/s at 2032 MHz), FP64 a small fraction of that, and the
multi-function unit's ex2 / lg2 at 16 to 32 results per clock per SM (4.8 to 9.6 T/s)."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def _probe():
    from paper_2503_17405_b300 import build
    build.build()
    lib = ctypes.CDLL(build.PROBE_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.fsmc_bench_probe.argtypes = [ctypes.c_int, dp, dp, dp, dp]
    lib.fsmc_bench_probe.restype = ctypes.c_int
    return lib


def test_probe_returns_plausible_rates():
    import torch
    torch.cuda.set_device(0)
    lib = _probe()
    r = [ctypes.c_double(0.0) for _ in range(4)]
    assert lib.fsmc_bench_probe(0, *[ctypes.byref(x) for x in r]) == 0
    f32, f64, ex2, lg2 = (x.value for x in r)
    print("FFMA %.1f TFLOP/s, DFMA %.2f TFLOP/s, ex2 %.2f T/s, lg2 %.2f T/s" % (f32, f64, ex2, lg2))
    assert 20.0 < f32 < 85.0
    assert 0.05 < f64 < f32
    assert 1.0 < ex2 < 12.0 and 1.0 < lg2 < 12.0
    assert torch.cuda.current_device() == 0


def test_probe_rejects_null_outputs():
    lib = _probe()
    assert lib.fsmc_bench_probe(0, None, None, None, None) == -1
