"""GPU parity of the Kronecker and Hadamard products against the oracle.

Each output element is one product rounded once, in FP64 or FP32 on both
sides (BF16 inputs give exact FP32 products), so the results must be
bit-identical to the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import build as moa_build
from paper_2306_11148_b300 import inputs, moa


def test_products_reject_bad_arguments():
    moa_build.build()
    L = moa.lib()
    assert L.moa_kronecker(2, 2, 2, 2, moa.MOA_F32_SPLIT, 256, 256, 256, None) == moa.MOA_ERR_DTYPE
    assert L.moa_kronecker(-1, 2, 2, 2, moa.MOA_F64, 256, 256, 256, None) == moa.MOA_ERR_ARG
    assert L.moa_hadamard(2, 2, moa.MOA_F64, 256 + 4, 256, 256, None) == moa.MOA_ERR_ALIGN
    assert L.moa_hadamard(0, 5, moa.MOA_F64, None, None, None, None) == moa.MOA_OK


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_F64, moa.MOA_F32_SIMT, moa.MOA_BF16])
@pytest.mark.parametrize("shape", [(3, 5, 7, 2), (16, 16, 16, 16), (33, 9, 17, 31), (1, 64, 300, 1)])
def test_kronecker_bit_exact(dt, shape):
    m, n, p, q = shape
    A, _ = inputs.uniform_pair(m, n, 1, dtype=moa.in_dtype(dt), seed=m + n)
    B, _ = inputs.uniform_pair(p, q, 1, dtype=moa.in_dtype(dt), seed=p + q + 1)
    C = moa.kronecker(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    ref = oracle.kronecker(A.double().numpy(), B.double().numpy())
    if dt == moa.MOA_F32_SIMT:
        ref = ref.astype(np.float32).astype(np.float64)   # the FP32 product, rounded once
    assert np.array_equal(C.double().cpu().numpy(), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_F64, moa.MOA_F32_SIMT, moa.MOA_BF16])
def test_hadamard_bit_exact(dt):
    A, _ = inputs.uniform_pair(257, 1031, 1, dtype=moa.in_dtype(dt), seed=1)
    B, _ = inputs.uniform_pair(257, 1031, 1, dtype=moa.in_dtype(dt), seed=2)
    C = moa.hadamard(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    ref = oracle.hadamard(A.double().numpy(), B.double().numpy())
    if dt == moa.MOA_F32_SIMT:
        ref = ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(C.double().cpu().numpy(), ref)
