"""CUDA-graph capture of the single-GEMM entry point: after one warm-up call
(tensor maps, kernel attributes and the status word are set up on first use),
moa_gemm_ex records only stream work, so a call can be captured once and
replayed; each replay recomputes C from the current contents of A and B."""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu

MODES = [moa.MOA_F32_TF32, moa.MOA_BF16, moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN,
         moa.MOA_F64_SPLIT_F32IN_E4M3, moa.MOA_F64, moa.MOA_F32_SIMT]
NAMES = {v: k for k, v in moa.MODES.items()}


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
def test_captured_gemm_replays_on_new_inputs(dt):
    m, n, p = 300, 520, 260
    tdt = moa.in_dtype(dt)
    A1, B1 = inputs.integer_pair(m, n, p, dtype=tdt, seed=1)
    A2, B2 = inputs.integer_pair(m, n, p, dtype=tdt, seed=2)
    A = A1.cuda()
    B = B1.cuda()
    C = torch.empty((m, p), dtype=moa.out_dtype(dt), device="cuda")
    ws = moa.Workspace(torch.device("cuda"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        moa.gemm(A, B, dt, C=C, stream=s, workspace=ws)          # warm-up, set-up on first use
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        moa.gemm(A, B, dt, C=C, stream=s, workspace=ws)
    for Ah, Bh in ((A1, B1), (A2, B2), (A1, B1)):
        A.copy_(Ah.cuda())
        B.copy_(Bh.cuda())
        C.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        moa.sync_status()
        ref = oracle.gemm(Ah.double().numpy(), Bh.double().numpy())
        assert np.array_equal(C.double().cpu().numpy(), ref)   # integer inputs: exact
