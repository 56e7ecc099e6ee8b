"""GPU parity of the grouped persistent launch (moa_gemm_grouped).

Each problem of a grouped call must equal the same problem run alone through
moa_gemm_ex bit for bit (same K-block order per output element), be bit-exact
against the oracle on integer inputs, and match the oracle within the BF16
tolerance on the grouped workload's shape mix (log-uniform in [32, 2048],
multiples of 16).  Problems the persistent path does not take (TF32, rows that
are not 16-byte multiples) run through the single-GEMM path in the same call.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu


def _problem(m, n, p, seed, integer=False, dt=moa.MOA_BF16):
    tdt = moa.in_dtype(dt)
    A, B = (inputs.integer_pair if integer else inputs.uniform_pair)(m, n, p, dtype=tdt, seed=seed)
    C = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
    return A.cuda(), B.cuda(), C, dt


def test_grouped_equals_single_and_oracle_integer():
    shapes = [(128, 64, 128), (16, 16, 16), (200, 96, 48), (300, 512, 520), (64, 2048, 256),
              (33, 64, 24), (512, 128, 1024)]
    probs = [_problem(m, n, p, seed=i, integer=True) for i, (m, n, p) in enumerate(shapes)]
    moa.gemm_grouped(probs)
    torch.cuda.synchronize()
    moa.sync_status()
    for A, B, C, dt in probs:
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone)
        ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
        assert np.array_equal(C.double().cpu().numpy(), ref)


def test_grouped_mixed_paths():
    """Unaligned and TF32 problems ride along through the single-GEMM path."""
    probs = [_problem(100, 40, 72, 1), _problem(37, 41, 43, 2),        # unaligned n, p
             _problem(64, 96, 80, 3, dt=moa.MOA_F32_TF32), _problem(256, 256, 256, 4)]
    moa.gemm_grouped(probs)
    moa.sync_status()
    for A, B, C, dt in probs:
        ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
        got = C.double().cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= (5e-3 if dt == moa.MOA_F32_TF32 else 1e-2)


def test_grouped_workload_shape_mix():
    shapes = inputs.grouped_shapes(96, seed=0)
    probs = [_problem(m, n, p, seed=100 + i) for i, (m, n, p) in enumerate(shapes)]
    moa.gemm_grouped(probs)
    moa.sync_status()
    for i in range(0, len(probs), 8):
        A, B, C, dt = probs[i]
        ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
        got = C.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5   # BF16-given inputs
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone)


def test_grouped_repeat_reuses_plan_and_skips_empty():
    probs = [_problem(64, 64, 64, 5), _problem(128, 256, 64, 6)]
    Z = (torch.empty((0, 16), dtype=torch.bfloat16, device="cuda"),
         torch.empty((16, 8), dtype=torch.bfloat16, device="cuda"),
         torch.empty((0, 8), dtype=torch.float32, device="cuda"), moa.MOA_BF16)
    descs = moa.make_descs(probs + [Z])
    ws = moa.Workspace(torch.device("cuda"))
    moa.gemm_grouped(probs + [Z], descs=descs, workspace=ws)
    c1 = [p[2].clone() for p in probs]
    for p in probs:
        p[2].fill_(float("nan"))
    moa.gemm_grouped(probs + [Z], descs=descs, workspace=ws)   # same plan, tables reused
    torch.cuda.synchronize()
    moa.sync_status()
    for a, p in zip(c1, probs):
        assert torch.equal(a, p[2])
