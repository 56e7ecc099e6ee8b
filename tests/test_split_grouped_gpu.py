"""Grouped FP32-accuracy split problems (moa_gemm_grouped with MOA_F32_SPLIT).

FP32-accuracy split problems that a lone call would run without split K
share one slice pre-pass launch and one persistent slice-GEMM launch over all
their tiles, each at its lone call's tile width.  The slice products of every
output are summed in the same order as alone, so each result must equal the
lone call's bit for bit, and lie within the mode's tolerance (1e-5 relative
Frobenius) of the FP64 oracle; few-tile long-K problems keep their own
split-K launches in the same call.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu


def _problem(m, n, p, seed, kind=None):
    A, B = inputs.normal_pair(m, n, p, dtype=torch.float32, seed=seed, scaled=kind)
    C = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
    return A.cuda(), B.cuda(), C, moa.MOA_F32_SPLIT


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# tile widths 128 and 256 (the lone planner's), ragged rows and columns,
# one and several K chunks, one tile and many
SHAPES = [(1, 1, 1), (37, 300, 45), (256, 1024, 256), (130, 2100, 520), (300, 64, 700),
          (513, 777, 129), (16, 16, 16), (1000, 1500, 1300), (2048, 512, 2048), (129, 3000, 2000)]


def test_grouped_f32_split_bit_identical_to_lone_calls():
    probs = [_problem(m, n, p, seed=70 + i, kind=[None, "rows", "rowcol"][i % 3])
             for i, (m, n, p) in enumerate(SHAPES)]
    grouped = [moa.grouped_path(*pr) for pr in probs]
    assert grouped.count(moa.MOA_GROUPED_F32_SPLIT) >= len(SHAPES) - 2, grouped
    moa.gemm_grouped(probs)
    moa.sync_status()
    for (A, B, C, dt), path in zip(probs, grouped):
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone), (tuple(A.shape), tuple(B.shape), path)
    for A, B, C, dt in probs[::3]:
        want = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
        assert _rel(C.double().cpu().numpy(), want) <= 1e-5


def test_grouped_call_mixes_every_path():
    """BF16, modular-slice, grouped FP32-split and one few-tile long-K
    FP32-split problem (its lone call splits K, so it runs alone) in one
    call: every result equals its lone call."""
    probs = [_problem(200, 700, 300, seed=1), _problem(64, 16384, 64, seed=2)]
    Ab, Bb = inputs.uniform_pair(128, 256, 192, dtype=torch.bfloat16, seed=3)
    probs.append((Ab.cuda(), Bb.cuda(), torch.empty((128, 192), device="cuda"), moa.MOA_BF16))
    Ac, Bc = inputs.normal_pair(150, 500, 260, dtype=torch.float32, seed=4)
    probs.append((Ac.cuda(), Bc.cuda(), torch.empty((150, 260), dtype=torch.float64, device="cuda"),
                  moa.MOA_F64_CRT_F32IN))
    paths = [moa.grouped_path(*pr) for pr in probs]
    assert paths == [moa.MOA_GROUPED_F32_SPLIT, moa.MOA_GROUPED_ALONE, moa.MOA_GROUPED_BF16,
                     moa.MOA_GROUPED_CRT]
    moa.gemm_grouped(probs)
    moa.sync_status()
    for A, B, C, dt in probs:
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        assert torch.equal(C, alone), dt


def test_grouped_f32_split_nonfinite_flagged():
    probs = [_problem(96, 200, 80, seed=10 + i) for i in range(3)]
    probs[1][0][4, 9] = float("nan")
    moa.check(moa.moa_sync_status(moa._stream_handle(None)))
    moa.gemm_grouped(probs)
    assert moa.moa_sync_status(moa._stream_handle(None)) == moa.MOA_ERR_NONFINITE
    assert moa.moa_sync_status(moa._stream_handle(None)) == moa.MOA_OK
