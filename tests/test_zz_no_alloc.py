"""moa_gemm_f32split_noalloc: the FP32-accuracy split GEMM for callers that
cannot allocate device memory (graph-capture regions, fixed start-up memory
plans, plugins confined to another runtime's pool).  Its scratch is a static
32 MiB device array inside libmoa.so instead of a caller workspace.

The GPU test calls it through the C ABI twice in a row, with different shapes
and inputs (the second call finds the first call's slices in the shared
scratch), and checks each result against the workspace entry point
(moa_gemm_ex, MOA_F32_SPLIT) within the split mode's tolerance.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2306_11148_b300 import build as moa_build
from paper_2306_11148_b300 import inputs, moa

LIMIT = 32 << 20
TOL = 1e-5   # relative Frobenius, the FP32-accuracy split mode's tolerance


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_oversized_problem_rejected_before_any_launch():
    moa_build.build()
    L = moa.lib()
    # 2048^3 needs 3 * 2 * 2 * 2048^2 bytes of BF16 slices: 48 MiB > 32 MiB
    assert moa.moa_gemm_workspace_size(2048, 2048, 2048, moa.MOA_F32_SPLIT, 0) > LIMIT
    rc = L.moa_gemm_f32split_noalloc(2048, 2048, 2048, 256, 512, 1024, None)
    assert rc == moa.MOA_ERR_WORKSPACE
    assert "static no-alloc scratch" in moa.last_error()
    assert L.moa_gemm_f32split_noalloc(-1, 4, 4, 256, 512, 1024, None) == moa.MOA_ERR_ARG


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_two_calls():
    L = moa.lib()
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    for (m, n, p), seed in [((700, 1100, 650), 11), ((130, 257, 90), 12)]:
        assert moa.moa_gemm_workspace_size(m, n, p, moa.MOA_F32_SPLIT, 0) <= LIMIT
        A, B = inputs.normal_pair(m, n, p, dtype=torch.float32, seed=seed, scaled="rows")
        A, B = A.cuda(), B.cuda()
        ref = moa.gemm(A, B, moa.MOA_F32_SPLIT)
        C = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
        moa.check(L.moa_gemm_f32split_noalloc(m, n, p, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                              sh))
        moa.check(moa.moa_sync_status(sh))
        assert _rel(C, ref) <= TOL
