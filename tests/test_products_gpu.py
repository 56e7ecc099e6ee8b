"""GPU parity of the outer-product family (moa_product: Hadamard, Kronecker
and matrix products through one kernel) against the oracle.

A Kronecker or Hadamard output element is one product rounded once, in FP64
or FP32 on both sides (BF16 inputs give exact FP32 products), so the results
must be bit-identical to the oracle's.  The matrix product through the same
kernel adds the rounded products in k order from zero, as the oracle's
i-k-j loop does, so in FP64 it must be bit-identical to oracle.gemm."""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import build as moa_build
from paper_2306_11148_b300 import inputs, moa


def test_products_reject_bad_arguments():
    moa_build.build()
    L = moa.lib()
    # shape rules of the one-kernel form, checked before any launch
    assert L.moa_product(moa.MOA_PRODUCT_HADAMARD, 2, 3, 2, 4, moa.MOA_F64, 256, 256, 256,
                         None) == moa.MOA_ERR_ARG
    assert L.moa_product(moa.MOA_PRODUCT_MATMUL, 2, 3, 4, 5, moa.MOA_F64, 256, 256, 256,
                         None) == moa.MOA_ERR_ARG
    assert L.moa_product(7, 2, 2, 2, 2, moa.MOA_F64, 256, 256, 256, None) == moa.MOA_ERR_ARG
    assert L.moa_product(moa.MOA_PRODUCT_MATMUL, 0, 3, 3, 5, moa.MOA_F64, 256, 256, 256,
                         None) == moa.MOA_OK
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


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (64, 64, 64), (37, 129, 21), (130, 1000, 9),
                                   (5, 1, 300)])
def test_matmul_through_outer_product_kernel_bit_exact(shape):
    """The contraction of the outer product, FP64, equals the oracle's i-k-j
    loop bit for bit (same rounded products, same order)."""
    m, n, q = shape
    A, B = inputs.uniform_pair(m, n, q, dtype=torch.float64, seed=m + n + q)
    C = moa.product(moa.MOA_PRODUCT_MATMUL, A.cuda(), B.cuda(), moa.MOA_F64)
    moa.sync_status()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm(A.numpy(), B.numpy()))


@pytest.mark.gpu
@pytest.mark.parametrize("dt,tol", [(moa.MOA_F32_SIMT, 1e-5), (moa.MOA_BF16, 1e-5)])
def test_matmul_through_outer_product_kernel_fp32(dt, tol):
    A, B = inputs.uniform_pair(100, 300, 70, dtype=moa.in_dtype(dt), seed=3)
    C = moa.product(moa.MOA_PRODUCT_MATMUL, A.cuda(), B.cuda(), dt)
    moa.sync_status()
    ref = oracle.gemm(A.double().numpy(), B.double().numpy())
    got = C.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol


@pytest.mark.gpu
def test_matmul_empty_contraction_gives_zero():
    A = torch.empty((4, 0), dtype=torch.float64, device="cuda")
    B = torch.empty((0, 6), dtype=torch.float64, device="cuda")
    C = moa.product(moa.MOA_PRODUCT_MATMUL, A, B, moa.MOA_F64)
    moa.sync_status()
    assert torch.equal(C.cpu(), torch.zeros((4, 6), dtype=torch.float64))


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_F64, moa.MOA_F32_SIMT, moa.MOA_BF16])
@pytest.mark.parametrize("kind", [moa.MOA_PRODUCT_KRONECKER, moa.MOA_PRODUCT_HADAMARD])
@pytest.mark.parametrize("shape", [(8, 16, 8, 16), (5, 7, 5, 7), (33, 12, 33, 12)])
def test_one_kernel_kron_and_hadamard_bit_exact(dt, kind, shape):
    """Both no-reduction members through moa_product, with the 16-byte load
    and store paths (widths that are multiples of 4) and the scalar ones."""
    m, n, p, q = shape
    A, _ = inputs.uniform_pair(m, n, 1, dtype=moa.in_dtype(dt), seed=m * n)
    B, _ = inputs.uniform_pair(p, q, 1, dtype=moa.in_dtype(dt), seed=p * q + 5)
    C = moa.product(kind, A.cuda(), B.cuda(), dt)
    moa.sync_status()
    f = oracle.kronecker if kind == moa.MOA_PRODUCT_KRONECKER else oracle.hadamard
    ref = f(A.double().numpy(), B.double().numpy())
    if dt == moa.MOA_F32_SIMT:
        ref = ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(C.double().cpu().numpy(), ref)
