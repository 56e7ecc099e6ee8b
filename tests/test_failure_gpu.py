"""Failure detection without a GPU fault.

Every pipeline wait in the tensor-core kernels is bounded; on expiry the
kernel records MOA_ERR_TIMEOUT in the per-device status word and returns.
Here a one-CTA self-test kernel waits on an mbarrier that nothing arrives at,
with a short limit; the host must read MOA_ERR_TIMEOUT, the status must clear,
and the context must stay usable (a GEMM right after is correct).
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_context_survives():
    L = moa.lib()
    sh = moa._stream_handle(None)
    moa.check(moa.moa_sync_status(sh))                 # clean start
    t0 = time.perf_counter()
    moa.check(L.moa_selftest_wait_timeout(50_000_000, sh))   # 50 ms
    assert moa.moa_sync_status(sh) == moa.MOA_ERR_TIMEOUT
    dt = time.perf_counter() - t0
    assert 0.04 <= dt < 5.0
    assert moa.moa_sync_status(sh) == moa.MOA_OK       # cleared by the read
    A, B = inputs.integer_pair(200, 300, 100, dtype=torch.bfloat16, seed=1)
    C = moa.gemm(A.cuda(), B.cuda(), moa.MOA_BF16)
    moa.sync_status()
    assert np.array_equal(C.double().cpu().numpy(),
                          oracle.gemm(A.double().numpy(), B.double().numpy()))


def test_selftest_rejects_bad_limits():
    from paper_2306_11148_b300 import build as moa_build
    moa_build.build()
    L = moa.lib()
    assert L.moa_selftest_wait_timeout(0, None) == moa.MOA_ERR_ARG
    assert L.moa_selftest_wait_timeout(20_000_000_000, None) == moa.MOA_ERR_ARG
