"""Parity at the configured workload sizes (GPU).

* The split-precision workload: m = n = p = 8192 FP32 operands drawn N(0, 1)
  (seed 0), plain and scaled by 10^U(-4,4) per row of A and of B ("rows") or
  per row of A and column of B ("rowcol").  Every precision mode of that
  workload (FP32-accuracy split; FP64-accuracy integer digits in BF16 and in
  E4M3; FP64-accuracy modular slices) is checked on 64 seed-chosen rows
  against the oracle: relative Frobenius error within the mode's tolerance,
  and elementwise |C - C_oracle| <= tol * (|A| |B|) (the componentwise form
  of the same bound).
* Native FP64 at N = 8192 (uniform[-1,1) inputs) on 64 sampled rows.
* The grouped batch: all 512 problems of the configured shape mix (m, n, p
  log-uniform in [32, 2048], multiples of 16, BF16 inputs, FP32 output) in one
  launch, every problem checked in full against the oracle and bit for bit
  against the same problem run alone.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu

N = 8192
KINDS = {"plain": None, "rows": "rows", "rowcol": "rowcol"}
TOL = {moa.MOA_F32_SPLIT: 1e-5, moa.MOA_F64_SPLIT_F32IN: 1e-12,
       moa.MOA_F64_SPLIT_F32IN_E4M3: 1e-12, moa.MOA_F64_CRT_F32IN: 1e-12, moa.MOA_F64: 1e-12}
NAMES = {v: k for k, v in moa.MODES.items()}


@pytest.fixture(scope="module")
def workload():
    """Per input kind: the operands (host), the sampled rows and the oracle's
    rows of A.B and of |A|.|B|."""
    rows = inputs.sample_rows(N, 64, seed=3)
    out = {}
    for name, scaled in KINDS.items():
        A, B = inputs.normal_pair(N, N, N, dtype=torch.float32, seed=0, scaled=scaled)
        Ad = A.double().numpy()
        Bd = B.double().numpy()
        ref, _ = oracle.gemm_omp(Ad[rows], Bd)
        absref, _ = oracle.gemm_omp(np.abs(Ad[rows]), np.abs(Bd))
        out[name] = (A, B, ref, absref)
    return rows, out


def _check(got, ref, absref, tol):
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= tol, rel
    bad = np.abs(got - ref) > tol * absref
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - ref) / np.maximum(absref, 1e-300))))


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("dt", [moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN,
                                moa.MOA_F64_SPLIT_F32IN_E4M3, moa.MOA_F64_CRT_F32IN],
                         ids=lambda d: NAMES[d])
def test_split_workload_sampled_rows(workload, dt, kind):
    rows, data = workload
    A, B, ref, absref = data[kind]
    C = moa.gemm(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    got = C[torch.from_numpy(rows).cuda()].cpu().double().numpy()
    del C
    _check(got, ref, absref, TOL[dt])


def test_native_f64_workload_sampled_rows():
    A, B = inputs.square_uniform(N, torch.float64, seed=0)
    C = moa.gemm(A.cuda(), B.cuda(), moa.MOA_F64)
    moa.sync_status()
    rows = inputs.sample_rows(N, 64, seed=4)
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
    Ad = A.numpy()
    Bd = B.numpy()
    ref, _ = oracle.gemm_omp(Ad[rows], Bd)
    absref, _ = oracle.gemm_omp(np.abs(Ad[rows]), np.abs(Bd))
    _check(got, ref, absref, TOL[moa.MOA_F64])


def test_grouped_all_configured_problems():
    shapes = inputs.grouped_shapes(512, seed=0)
    probs = []
    for i, (m, n, p) in enumerate(shapes):
        A, B = inputs.uniform_pair(m, n, p, dtype=torch.bfloat16, seed=1000 + i)
        C = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
        probs.append((A.cuda(), B.cuda(), C, moa.MOA_BF16))
    moa.gemm_grouped(probs)
    moa.sync_status()
    worst = 0.0
    for A, B, C, dt in probs:
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone)
        Ad = A.double().cpu().numpy()
        Bd = B.double().cpu().numpy()
        ref, _ = oracle.gemm_omp(Ad, Bd)
        absref, _ = oracle.gemm_omp(np.abs(Ad), np.abs(Bd))
        got = C.double().cpu().numpy()
        # BF16-given inputs: exact products, FP32 accumulation over n terms
        n = A.shape[1]
        assert np.all(np.abs(got - ref) <= n * 2.0 ** -23 * absref)
        worst = max(worst, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    assert worst <= 1e-5, worst
