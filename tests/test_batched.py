"""Batched 3-D contraction C[b, i, j] = sum_k A[b, i, k] B[b, k, j]
(moa_gemm_batched), the higher-dimensional extension of the inner product.

Each entry must equal the same GEMM alone (bit for bit) and the oracle; a
stride of 0 broadcasts one operand; argument errors are refused on the host."""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import build as moa_build
from paper_2306_11148_b300 import inputs, moa


@pytest.fixture(scope="module")
def L():
    moa_build.build()
    return moa.lib()


def test_batched_argument_errors(L):
    assert L.moa_gemm_batched(-1, 4, 4, 4, moa.MOA_BF16, 256, 16, 256, 16, 256, 16, None, 0,
                              None) == moa.MOA_ERR_ARG
    # C entries would overlap
    assert L.moa_gemm_batched(2, 4, 4, 4, moa.MOA_BF16, 256, 16, 256, 16, 256, 8, None, 0,
                              None) == moa.MOA_ERR_ARG
    assert L.moa_gemm_batched(2, 4, 4, 4, 42, 256, 16, 256, 16, 256, 16, None, 0,
                              None) == moa.MOA_ERR_DTYPE
    assert L.moa_gemm_batched(0, 4, 4, 4, moa.MOA_BF16, 0, 0, 0, 0, 0, 0, None, 0,
                              None) == moa.MOA_OK


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_BF16, moa.MOA_F32_TF32, moa.MOA_F64_SPLIT_F32IN,
                                moa.MOA_F64_SPLIT_F32IN_E4M3])
@pytest.mark.parametrize("broadcast_b", [False, True])
def test_batched_matches_single_and_oracle(dt, broadcast_b):
    batch, m, n, p = 6, 192, 320, 256
    tdt = moa.in_dtype(dt)
    A = torch.stack([inputs.integer_pair(m, n, p, dtype=tdt, seed=b)[0] for b in range(batch)])
    if broadcast_b:
        B = inputs.integer_pair(m, n, p, dtype=tdt, seed=99)[1]
    else:
        B = torch.stack([inputs.integer_pair(m, n, p, dtype=tdt, seed=50 + b)[1]
                         for b in range(batch)])
    A, B = A.cuda(), B.cuda()
    C = moa.gemm_batched(A, B, dt)
    moa.sync_status()
    for b in range(batch):
        Bb = B if broadcast_b else B[b]
        alone = moa.gemm(A[b].contiguous(), Bb.contiguous(), dt)
        torch.cuda.synchronize()
        assert torch.equal(C[b], alone)
        ref = oracle.gemm(A[b].double().cpu().numpy(), Bb.double().cpu().numpy())
        assert np.array_equal(C[b].double().cpu().numpy(), ref)   # integer inputs: exact
