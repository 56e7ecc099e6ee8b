"""moa_gemm_f32split_noalloc: the FP32-accuracy split GEMM for callers that
may not allocate device memory at all (real-time or safety-certified hosts
whose device memory is fixed at start-up, plugins inside another runtime's
memory pool, static memory plans).  Its scratch is a static 32 MiB device
array inside libmoa.so instead of a caller workspace.

The GPU test calls it through the C ABI three times in a row with different
shapes and inputs: a large one first, then a few-tile shape that takes the
split-K path (its counters and FP32 partial tiles then live in the shared
array, on top of the first call's leftovers), then a small ragged one.  Each
result is checked against the workspace entry point (moa_gemm_ex,
MOA_F32_SPLIT) and against the FP64 oracle, within the split mode's
tolerance, and the device's free memory is the same before and after the
calls.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import build as moa_build
from paper_2306_11148_b300 import inputs, moa

LIMIT = 32 << 20
TOL = 1e-5   # relative Frobenius, the FP32-accuracy split mode's tolerance


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_oversized_problem_rejected_before_any_launch():
    moa_build.build()
    L = moa.lib()
    # 2048^3 needs 3 * 2 * 2 * 2048^2 bytes of BF16 slices: 48 MiB > 32 MiB
    assert moa.moa_gemm_workspace_size(2048, 2048, 2048, moa.MOA_F32_SPLIT, 0) > LIMIT
    rc = L.moa_gemm_f32split_noalloc(2048, 2048, 2048, 256, 512, 1024, None)
    assert rc == moa.MOA_ERR_WORKSPACE
    assert "static no-alloc scratch" in moa.last_error()
    # sizes whose byte counts would not fit 64 bits are refused the same way
    big = 1 << 31
    rc = L.moa_gemm_f32split_noalloc(big, big, big, 256, 512, 1024, None)
    assert rc == moa.MOA_ERR_WORKSPACE
    assert L.moa_gemm_f32split_noalloc(-1, 4, 4, 256, 512, 1024, None) == moa.MOA_ERR_ARG
    assert L.moa_gemm_f32split_noalloc((1 << 31) + 1, 4, 4, 256, 512, 1024, None) == \
        moa.MOA_ERR_ARG


# (m, n, p), seed: a large call, then a split-K call (few tiles, long K) that
# starts on the first call's leftovers, then a small ragged one
CASES = [((700, 1100, 650), 11), ((256, 4096, 256), 13), ((130, 257, 90), 12)]


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_two_calls():
    L = moa.lib()
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    # the split-K case keeps counters and partial tiles in the scratch too
    m, n, p = CASES[1][0]
    planes = 6 * (m * n + n * p)
    assert moa.moa_gemm_workspace_size(m, n, p, moa.MOA_F32_SPLIT, 0) >= planes + 2 * m * p * 4
    data = []
    for (m, n, p), seed in CASES:
        assert moa.moa_gemm_workspace_size(m, n, p, moa.MOA_F32_SPLIT, 0) <= LIMIT
        A, B = inputs.normal_pair(m, n, p, dtype=torch.float32, seed=seed, scaled="rows")
        Ad, Bd = A.cuda(), B.cuda()
        ref = moa.gemm(Ad, Bd, moa.MOA_F32_SPLIT).cpu().numpy()
        exact = oracle.gemm(A.double().numpy(), B.double().numpy())
        C = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
        data.append(((m, n, p), Ad, Bd, C, ref, exact))
    torch.cuda.synchronize()

    def call(k):
        (m, n, p), Ad, Bd, C, _, _ = data[k]
        moa.check(L.moa_gemm_f32split_noalloc(m, n, p, Ad.data_ptr(), Bd.data_ptr(),
                                              C.data_ptr(), sh))

    call(0)   # the first call on the device sets up the scratch address
    moa.check(moa.moa_sync_status(sh))
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 0, 1):
        call(k)
    moa.check(moa.moa_sync_status(sh))
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, "the no-alloc entry point changed the device's free memory"
    for shape, _, _, C, ref, exact in data:
        got = C.cpu().numpy()
        assert _rel(got, ref) <= TOL, shape
        assert _rel(got, exact) <= TOL, shape
