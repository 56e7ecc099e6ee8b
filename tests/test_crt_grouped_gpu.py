"""Grouped modular-slice problems (moa_gemm_grouped with MOA_F64_CRT_*).

The modular-slice problems of a grouped call run as one exponent and one
residue launch per input type, one persistent residue-GEMM launch over every
(problem, modulus, tile) unit and one reconstruction launch.  Each problem's
result must be bit-identical to the same problem run alone (the method
reaches the exact integer product of the scaled operands, rounded once, so
tiling and scheduling cannot change it) and bit-exact against the oracle's
exact integer product; problems of other modes in the same call still run.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu


def default_moduli(n):
    for M in (14, 15):
        if oracle.crt_bits(max(n, 1), M) >= 47:
            return M
    return 16


def _crt_problem(m, n, p, dt, seed, kind="rows"):
    A, B = inputs.normal_pair(m, n, p, dtype=torch.float64, seed=seed, scaled=kind)
    if dt == moa.MOA_F64_CRT_F32IN:
        A, B = A.float(), B.float()
    C = torch.full((m, p), float("nan"), dtype=torch.float64, device="cuda")
    return A.cuda(), B.cuda(), C, dt


def test_grouped_crt_mixed_batch_bit_exact():
    shapes = [(1, 1, 1), (37, 300, 45), (256, 1024, 256), (130, 2100, 520), (64, 40000, 48),
              (300, 64, 700), (513, 777, 129), (16, 16, 16)]
    probs = []
    for i, (m, n, p) in enumerate(shapes):
        dt = moa.MOA_F64_CRT_F32IN if i % 3 else moa.MOA_F64_CRT_F64IN
        probs.append(_crt_problem(m, n, p, dt, seed=50 + i, kind=[None, "rows", "rowcol"][i % 3]))
    # other modes ride along in the same call
    Ab, Bb = inputs.uniform_pair(128, 256, 192, dtype=torch.bfloat16, seed=7)
    probs.append((Ab.cuda(), Bb.cuda(), torch.empty((128, 192), device="cuda"), moa.MOA_BF16))
    As, Bs = inputs.normal_pair(100, 300, 90, dtype=torch.float32, seed=8)
    probs.append((As.cuda(), Bs.cuda(), torch.empty((100, 90), device="cuda"), moa.MOA_F32_SPLIT))
    moa.gemm_grouped(probs)
    moa.sync_status()
    for A, B, C, dt in probs:
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone), (tuple(A.shape), tuple(B.shape), dt)
        if dt in moa.CRT:
            want = oracle.crt_gemm(A.double().cpu().numpy(), B.double().cpu().numpy(),
                                   default_moduli(A.shape[1]))
            assert np.array_equal(C.cpu().numpy(), want)


def test_grouped_crt_serving_shape_mix():
    """The serving stream's shapes (m, p log-uniform in [64, 4096], n in
    [64, 8192]), scaled down by 4 so that the oracle check stays short: 48
    FP64-accuracy problems in one call, each bit-identical to its lone run,
    every 6th also against the oracle."""
    arr = inputs.serve_arrivals(rate=200.0, seconds=1.0, seed=3)[:48]
    probs = []
    for i, (_, m, n, p, _) in enumerate(arr):
        m, n, p = max(1, m // 4), max(1, n // 4), max(1, p // 4)
        probs.append(_crt_problem(m, n, p, moa.MOA_F64_CRT_F32IN, seed=200 + i))
    moa.gemm_grouped(probs)
    moa.sync_status()
    for i, (A, B, C, dt) in enumerate(probs):
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone)
        if i % 6 == 0:
            want = oracle.crt_gemm(A.double().cpu().numpy(), B.double().cpu().numpy(),
                                   default_moduli(A.shape[1]))
            assert np.array_equal(C.cpu().numpy(), want)


def test_grouped_crt_nonfinite_flagged():
    probs = [_crt_problem(64, 96, 80, moa.MOA_F64_CRT_F32IN, seed=1),
             _crt_problem(32, 64, 48, moa.MOA_F64_CRT_F32IN, seed=2)]
    probs[1][0][3, 5] = float("inf")
    moa.gemm_grouped(probs)
    assert moa.moa_sync_status(0) == moa.MOA_ERR_NONFINITE
    assert moa.moa_sync_status(0) == moa.MOA_OK


def test_grouped_crt_repeat_same_workspace():
    probs = [_crt_problem(200, 500, 150, moa.MOA_F64_CRT_F32IN, seed=i) for i in range(3)]
    descs = moa.make_descs(probs)
    ws = moa.Workspace(torch.device("cuda"))
    moa.gemm_grouped(probs, descs=descs, workspace=ws)
    first = [p[2].clone() for p in probs]
    for p in probs:
        p[2].fill_(float("nan"))
    moa.gemm_grouped(probs, descs=descs, workspace=ws)
    moa.sync_status()
    for a, p in zip(first, probs):
        assert torch.equal(a, p[2])
