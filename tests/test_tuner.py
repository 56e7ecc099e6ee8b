"""Tile widths of the dense tensor-core GEMMs: forced widths, the measured
autotuner and its table file.

Every tile width sums each output element over the same K blocks in the same
order, so the result must not depend on the width (bit-identical), and the
tuner's choice must be one of the widths and be reused for the shape bucket."""
import ctypes
import os

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


def test_block_n_argument_checked(L):
    assert L.moa_set_block_n(96) == moa.MOA_ERR_ARG
    assert L.moa_set_block_n(0) == moa.MOA_OK


def test_tune_table_file_round_trip(L, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text("3 20 20 20 128\n1 16 18 16 64\n1 2 2 2 99\n")   # last line invalid
    assert L.moa_tune_clear() == moa.MOA_OK
    assert L.moa_tune_load(str(src).encode()) == moa.MOA_OK
    out = tmp_path / "out.txt"
    assert L.moa_tune_save(str(out).encode()) == moa.MOA_OK
    assert sorted(out.read_text().split("\n")[:-1]) == ["1 16 18 16 64", "3 20 20 20 128"]
    assert L.moa_tune_load(str(tmp_path / "missing.txt").encode()) == moa.MOA_ERR_ARG
    L.moa_tune_clear()


def test_tune_rejects_modes_without_tiles(L):
    assert L.moa_tune_dense(8, 8, 8, moa.MOA_F64, 256, 256, 256, None, 0, None, None, None) == \
        moa.MOA_ERR_DTYPE


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_BF16, moa.MOA_F32_TF32])
def test_every_tile_width_gives_the_same_bits(L, dt):
    A, B = inputs.uniform_pair(300, 700, 520, dtype=moa.in_dtype(dt), seed=3)
    A, B = A.cuda(), B.cuda()
    outs = []
    try:
        for w in (64, 128, 256):
            assert L.moa_set_block_n(w) == moa.MOA_OK
            C, st = moa.gemm(A, B, dt, stats=True)
            torch.cuda.synchronize()
            assert st.block_n == w
            outs.append(C)
    finally:
        L.moa_set_block_n(0)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])
    ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
    got = outs[0].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= (5e-3 if dt == moa.MOA_F32_TF32 else 1e-5)


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_BF16, moa.MOA_F32_TF32])
@pytest.mark.parametrize("m", [129, 515, 1024])
def test_widest_tiles_exact_with_ragged_rows_and_columns(L, dt, m):
    """256-wide tiles forced on 2, 5 and 8 row tiles (the last one ragged for
    m = 129 and 515) and a ragged last column tile (p = 1100): integer inputs,
    exact against the oracle."""
    n, p = 1000, 1100
    A, B = inputs.integer_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m)
    try:
        assert L.moa_set_block_n(256) == moa.MOA_OK
        C, st = moa.gemm(A.cuda(), B.cuda(), dt, stats=True)
        moa.sync_status()
        assert st.block_n == 256
    finally:
        L.moa_set_block_n(0)
    ref = oracle.gemm(A.double().numpy(), B.double().numpy())
    assert np.array_equal(C.double().cpu().numpy(), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_BF16, moa.MOA_F32_TF32])
def test_tall_tiles_ragged_edges_exact(L, dt):
    """256 x 256 tiles (two M = 128 MMAs per K step) are the planner's choice
    here: 16 x 9 of them make one wave on 148 SMs, against two waves of
    128 x 256 tiles.  The last row and column tiles are ragged
    (m = 16 * 256 - 50, p = 9 * 256 - 7).  Integer inputs: the rows around
    every tile boundary and the ragged edge are exact against the oracle."""
    m, n, p = 16 * 256 - 50, 1000, 9 * 256 - 7
    A, B = inputs.integer_pair(m, n, p, dtype=moa.in_dtype(dt), seed=77)
    C, st = moa.gemm(A.cuda(), B.cuda(), dt, stats=True)
    moa.sync_status()
    assert st.block_m == 256 and st.block_n == 256
    rows = np.array(sorted({0, 1, 127, 128, 255, 256, 1000, 2047, 2048, 3071, 3072, 3839, 3840,
                            m - 50, m - 2, m - 1}), dtype=np.int64)
    got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    ref = oracle.gemm_rows(A.double().numpy(), B.double().numpy(), rows)
    assert np.array_equal(got, ref)


@pytest.mark.gpu
def test_tuner_records_and_reuses_choice(L, tmp_path):
    L.moa_tune_clear()
    m, n, p = 1024, 2048, 1536
    A, B = inputs.uniform_pair(m, n, p, dtype=torch.bfloat16, seed=4)
    A, B = A.cuda(), B.cuda()
    C = torch.empty((m, p), dtype=torch.float32, device="cuda")
    best = ctypes.c_int()
    ms = ctypes.c_float()
    moa.check(L.moa_tune_dense(m, n, p, moa.MOA_BF16, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                               None, 0, moa._stream_handle(None), ctypes.byref(best),
                               ctypes.byref(ms)))
    assert best.value in (64, 128, 256) and ms.value > 0
    _, st = moa.gemm(A, B, moa.MOA_BF16, stats=True)
    assert st.block_n == best.value
    out = tmp_path / "tune.txt"
    moa.check(L.moa_tune_save(str(out).encode()))
    assert out.read_text().strip().endswith(str(best.value))
    L.moa_tune_clear()


@pytest.mark.gpu
@pytest.mark.parametrize("dt,widths", [(moa.MOA_F32_SPLIT, (128, 256)),
                                       (moa.MOA_F64_SPLIT_F32IN, (128, 192, 256)),
                                       (moa.MOA_F64_SPLIT_F32IN_E4M3, (128, 192, 256))])
def test_split_tile_widths_agree(L, dt, widths):
    """Every slice-GEMM tile width sums the same chunks in the same order, so
    the results are bit-identical; each is within the mode's tolerance."""
    A, B = inputs.normal_pair(300, 900, 700, dtype=torch.float32, seed=9, scaled="rows")
    A, B = A.cuda(), B.cuda()
    outs = []
    try:
        for w in widths:
            assert L.moa_set_block_n(w) == moa.MOA_OK
            C, st = moa.gemm(A, B, dt, stats=True)
            torch.cuda.synchronize()
            moa.sync_status()
            assert st.block_n == w
            outs.append(C)
    finally:
        L.moa_set_block_n(0)
    for o in outs[1:]:
        assert torch.equal(outs[0], o)
    ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
    got = outs[1].double().cpu().numpy()
    tol = 1e-5 if dt == moa.MOA_F32_SPLIT else 1e-12
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol


def test_grouped_planner_reads_the_measured_table(L, tmp_path):
    """The grouped launch's per-problem tile width comes from the measured
    table when its shape bucket has an entry (half-octave buckets: 1024 ->
    round(2 log2 1024) = 20), else from the cost model; moa_set_block_n forces it."""
    L.moa_tune_clear()
    model = L.moa_grouped_block_n(1024, 1024, 1024)
    assert model in (64, 128, 256)
    want = 64 if model != 64 else 128
    src = tmp_path / "t.txt"
    src.write_text(f"3 20 20 20 {want}\n")
    assert L.moa_tune_load(str(src).encode()) == moa.MOA_OK
    assert L.moa_grouped_block_n(1024, 1024, 1024) == want
    assert L.moa_grouped_block_n(1000, 1100, 1024) == want          # same buckets
    assert L.moa_grouped_block_n(2048, 1024, 1024) == L.moa_grouped_block_n(2048, 1024, 1024)
    assert L.moa_set_block_n(256) == moa.MOA_OK
    assert L.moa_grouped_block_n(1024, 1024, 1024) == 256
    assert L.moa_set_block_n(0) == moa.MOA_OK
    L.moa_tune_clear()
    assert L.moa_grouped_block_n(1024, 1024, 1024) == model
    assert L.moa_grouped_block_n(0, 5, 5) == 0


@pytest.mark.gpu
def test_grouped_tuned_widths_bit_identical(L, tmp_path):
    """A grouped call planned with measured widths gives the same bits as the
    cost-model plan and as the problems run alone (integer inputs: exact)."""
    import numpy as np
    import torch

    import oracle
    from paper_2306_11148_b300 import inputs
    shapes = [(1024, 1024, 1024), (1000, 1100, 1024), (256, 512, 384)]
    probs = []
    for i, (m, n, p) in enumerate(shapes):
        A, B = inputs.integer_pair(m, n, p, dtype=torch.bfloat16, seed=40 + i)
        probs.append((A.cuda(), B.cuda(), torch.empty((m, p), device="cuda"), moa.MOA_BF16))
    L.moa_tune_clear()
    moa.gemm_grouped(probs)
    moa.sync_status()
    base = [p[2].clone() for p in probs]
    model = L.moa_grouped_block_n(1024, 1024, 1024)
    want = 64 if model != 64 else 128
    src = tmp_path / "t.txt"
    src.write_text(f"3 20 20 20 {want}\n")
    assert L.moa_tune_load(str(src).encode()) == moa.MOA_OK
    try:
        assert L.moa_grouped_block_n(1024, 1024, 1024) == want
        for p in probs:
            p[2].fill_(float("nan"))
        moa.gemm_grouped(probs, workspace=moa.Workspace(torch.device("cuda")))
        moa.sync_status()
    finally:
        L.moa_tune_clear()
    for b, (A, B, C, dt) in zip(base, probs):
        assert torch.equal(C, b)
        ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
        assert np.array_equal(C.double().cpu().numpy(), ref)
