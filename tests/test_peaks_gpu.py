"""The FP64 rate diagnostic (moa_measure_fp64_rate): both kinds run, report a
plausible rate and leave the device status clean; the native FP64 GEMM does
not exceed the measured FMA rate by more than measurement noise."""
import ctypes

import pytest
import torch

from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu


def _rate(kind):
    out = ctypes.c_double(0.0)
    moa.check(moa.lib().moa_measure_fp64_rate(kind, moa._stream_handle(None), ctypes.byref(out)))
    return out.value


def test_fp64_rates_are_plausible():
    fma, mma = _rate(0), _rate(1)
    print(f"FP64 FMA {fma:.3f} TFLOP/s, FP64 MMA {mma:.3f} TFLOP/s")
    assert 0.1 < fma < 200 and 0.1 < mma < 200
    moa.sync_status()


def test_native_fp64_gemm_within_measured_rate():
    N = 2048
    A, B = inputs.square_uniform(N, torch.float64, seed=0)
    A, B = A.cuda(), B.cuda()
    moa.gemm(A, B, moa.MOA_F64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    moa.gemm(A, B, moa.MOA_F64)
    e1.record()
    torch.cuda.synchronize()
    gemm = 2.0 * N ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    fma = _rate(0)
    print(f"native FP64 GEMM {gemm:.3f} TFLOP/s = {gemm / fma:.3f} of the measured FMA rate")
    assert gemm < 1.1 * fma
