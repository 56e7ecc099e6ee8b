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


@pytest.mark.gpu
def test_workspace_canary_stays_intact():
    """MOA_DEBUG_CANARY=1 (read once per process, so in a child process):
    every mode's plain moa_gemm call guards the bytes past its workspace and
    checks them after its kernels; none may be overwritten, and the results
    stay exact on integer inputs."""
    import os
    import subprocess
    import sys
    code = r'''
import numpy as np, torch, oracle
from paper_2306_11148_b300 import inputs, moa
L = moa.lib()
for dt in (moa.MOA_F32_TF32, moa.MOA_BF16, moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN,
           moa.MOA_F64_SPLIT_F64IN_E4M3, moa.MOA_F64_CRT_F32IN, moa.MOA_F64_CRT_F64IN):
    for (m, n, p) in ((33, 127, 129), (70, 4200, 140), (257, 1000, 200)):
        A, B = inputs.integer_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m + n)
        Ad, Bd = A.cuda(), B.cuda()
        C = torch.empty((m, p), dtype=moa.out_dtype(dt), device="cuda")
        moa.check(L.moa_gemm(m, n, p, dt, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr()))
        moa.check(L.moa_sync_status(None))
        assert np.array_equal(C.double().cpu().numpy(),
                              oracle.gemm(A.double().numpy(), B.double().numpy())), (dt, m, n, p)
print("canary ok")
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MOA_DEBUG_CANARY="1", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "canary ok" in r.stdout
