"""Parity of the FP64-accuracy modular-slice modes (MOA_F64_CRT_F32IN,
MOA_F64_CRT_F64IN) against the oracle.

The mode reaches exactly fl(2^(eA_i + eB_j - 2t) * (A'B')[i,j]) for the
operands scaled per row / column to t-bit integers, which ``oracle.crt_gemm``
computes with 128-bit integer sums: the GPU result must match it bit for bit
at every shape (ragged tiles, K chunk boundaries, split K, both tile widths,
8..16 moduli), and lie within the FP64 tolerance (1e-12 relative Frobenius)
of the FP64 GEMM oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu

MODES = [moa.MOA_F64_CRT_F32IN, moa.MOA_F64_CRT_F64IN]
NAMES = {v: k for k, v in moa.MODES.items()}


def default_moduli(n):
    """The documented default: the fewest moduli from 14 with t >= 47."""
    for M in (14, 15):
        if oracle.crt_bits(max(n, 1), M) >= 47:
            return M
    return 16


def _pair(m, n, p, dt, kind, seed):
    A, B = inputs.normal_pair(m, n, p, dtype=torch.float64, seed=seed, scaled=kind)
    if dt == moa.MOA_F64_CRT_F32IN:
        A, B = A.float(), B.float()
    return A, B


def _run(A, B, dt, slices=0):
    C = moa.gemm(A.cuda(), B.cuda(), dt, slices=slices)
    moa.sync_status()
    return C.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SHAPES = [(1, 1, 1), (3, 17, 5), (130, 257, 300), (257, 1030, 260), (300, 2100, 520),
          (64, 4096, 64), (129, 3000, 385)]


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("kind", [None, "rows", "rowcol"], ids=["plain", "rows", "rowcol"])
def test_bit_exact_against_exact_integer_product(dt, shape, kind):
    m, n, p = shape
    A, B = _pair(m, n, p, dt, kind, seed=m + n + p)
    got = _run(A, B, dt)
    Ad, Bd = A.double().numpy(), B.double().numpy()
    want = oracle.crt_gemm(Ad, Bd, default_moduli(n))
    assert np.array_equal(got, want)
    assert _rel(got, oracle.gemm(Ad, Bd)) <= 1e-12


@pytest.mark.parametrize("M", [8, 10, 12, 13, 14, 15, 16])
def test_every_modulus_count_bit_exact(M):
    m, n, p = 200, 700, 190
    A, B = _pair(m, n, p, moa.MOA_F64_CRT_F32IN, "rows", seed=M)
    got = _run(A, B, moa.MOA_F64_CRT_F32IN, slices=M)
    assert np.array_equal(got, oracle.crt_gemm(A.double().numpy(), B.double().numpy(), M))


@pytest.mark.parametrize("bn", [128, 256])
def test_both_tile_widths_bit_exact(bn):
    m, n, p = 300, 1500, 700
    A, B = _pair(m, n, p, moa.MOA_F64_CRT_F32IN, "rowcol", seed=5)
    L = moa.lib()
    moa.check(L.moa_set_block_n(bn))
    try:
        C, st = moa.gemm(A.cuda(), B.cuda(), moa.MOA_F64_CRT_F32IN, stats=True)
        moa.sync_status()
    finally:
        moa.check(L.moa_set_block_n(0))
    assert st.block_n == bn
    assert np.array_equal(C.cpu().numpy(),
                          oracle.crt_gemm(A.double().numpy(), B.double().numpy(), 14))


def _run_tiles(A, B, dt, block_m, slices=0, block_n=0):
    L = moa.lib()
    moa.check(L.moa_set_block_m(block_m))
    moa.check(L.moa_set_block_n(block_n))
    try:
        C, st = moa.gemm(A.cuda(), B.cuda(), dt, slices=slices, stats=True)
        moa.sync_status()
    finally:
        moa.check(L.moa_set_block_m(0))
        moa.check(L.moa_set_block_n(0))
    return C.cpu().numpy(), st


# ragged rows (the odd CTA's rows partly or wholly past m), ragged columns
# (its B half past p), one and several K chunks, 7- and 8-limb moduli counts
PAIR_CASES = [((1, 1, 1), 14), ((3, 17, 5), 14), ((129, 3000, 385), 14), ((257, 1030, 260), 16),
              ((300, 2100, 520), 15), ((640, 700, 900), 8), ((1000, 64, 3000), 14)]


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("case", PAIR_CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_pair_tiles_bit_exact(dt, case):
    """256 x 256 tiles on CTA pairs (moa_set_block_m(256)) equal the exact
    integer product bit for bit."""
    (m, n, p), M = case
    A, B = _pair(m, n, p, dt, "rowcol", seed=m + 2 * n + p)
    got, st = _run_tiles(A, B, dt, 256, slices=M)
    assert st.block_m == 256 and st.block_n == 256 and st.grid % 2 == 0
    assert np.array_equal(got, oracle.crt_gemm(A.double().numpy(), B.double().numpy(), M))


def test_pair_and_one_sm_tiles_agree_on_many_tiles():
    """3000 x 1500 x 5000 (12 x 20 pair tiles x 14 moduli, several units per
    cluster): CTA-pair tiles, 128 x 256 and 128 x 128 tiles give the same
    bits, and sampled rows equal the exact integer product."""
    m, n, p = 3000, 1500, 5000
    A, B = _pair(m, n, p, moa.MOA_F64_CRT_F32IN, "rows", seed=21)
    pair, st2 = _run_tiles(A, B, moa.MOA_F64_CRT_F32IN, 256)
    one, st1 = _run_tiles(A, B, moa.MOA_F64_CRT_F32IN, 128, block_n=256)
    narrow, st0 = _run_tiles(A, B, moa.MOA_F64_CRT_F32IN, 128, block_n=128)
    assert (st2.block_m, st1.block_m, st1.block_n, st0.block_n) == (256, 128, 256, 128)
    assert np.array_equal(pair, one) and np.array_equal(pair, narrow)
    rows = inputs.sample_rows(m, 6, seed=4)
    want = oracle.crt_gemm(A.double().numpy()[rows], B.double().numpy(), 14)
    assert np.array_equal(pair[rows], want)


def test_planner_pair_tiles_only_while_planes_fit_l2():
    """The planner takes CTA-pair tiles while one modulus plane of A and of B
    fits in the L2 (1024^3), one-SM tiles once a plane does not (8192 x 8192
    x 256: A's plane is 128 MiB); both give the forced other shape's bits."""
    small = _pair(1024, 1024, 1024, moa.MOA_F64_CRT_F32IN, "rows", seed=31)
    got, st = _run_tiles(*small, moa.MOA_F64_CRT_F32IN, 0)
    forced, _ = _run_tiles(*small, moa.MOA_F64_CRT_F32IN, 128)
    assert st.block_m == 256 and np.array_equal(got, forced)
    A, B = _pair(8192, 8192, 256, moa.MOA_F64_CRT_F32IN, "rows", seed=32)
    got, st = _run_tiles(A, B, moa.MOA_F64_CRT_F32IN, 0)
    forced, st2 = _run_tiles(A, B, moa.MOA_F64_CRT_F32IN, 256)
    assert st.block_m == 128 and st2.block_m == 256 and np.array_equal(got, forced)
    rows = inputs.sample_rows(8192, 4, seed=5)
    want = oracle.crt_gemm(A.double().numpy()[rows], B.double().numpy(), 14)
    assert np.array_equal(got[rows], want)


def test_block_m_setter_rejects_bad_values():
    L = moa.lib()
    assert L.moa_set_block_m(64) == moa.MOA_ERR_ARG
    assert L.moa_set_block_m(512) == moa.MOA_ERR_ARG
    assert L.moa_set_block_m(0) == moa.MOA_OK


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
def test_integer_inputs_bit_exact_against_gemm_oracle(dt):
    A, B = inputs.integer_pair(257, 1000, 200, dtype=moa.in_dtype(dt), seed=3)
    got = _run(A, B, dt)
    assert np.array_equal(got, oracle.gemm(A.double().numpy(), B.double().numpy()))


def test_default_moduli_for_long_k():
    m, n, p = 16, 40000, 24
    assert default_moduli(n) == 15
    A, B = _pair(m, n, p, moa.MOA_F64_CRT_F32IN, None, seed=8)
    C, st = moa.gemm(A.cuda(), B.cuda(), moa.MOA_F64_CRT_F32IN, stats=True)
    moa.sync_status()
    assert st.slices == 15 and st.products == 15
    want = oracle.crt_gemm(A.double().numpy(), B.double().numpy(), 15)
    assert np.array_equal(C.cpu().numpy(), want)


def test_wide_exponent_ranges_fp64():
    """Rows of A and columns of B spread over 10^-200 .. 10^200, zero rows and
    columns, subnormal entries: the scaling is per row / column, so every
    result still matches the exact integer product."""
    rng = np.random.default_rng(17)
    m, n, p = 40, 300, 36
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-200, 200, (m, 1))
    B = rng.standard_normal((n, p)) * 10.0 ** rng.uniform(-100, 100, (1, p))
    A[3, :] = 0.0
    B[:, 5] = 0.0
    A[7, 11] = 5e-324
    B[13, 2] = -4e-320
    got = _run(torch.from_numpy(A), torch.from_numpy(B), moa.MOA_F64_CRT_F64IN)
    assert np.array_equal(got, oracle.crt_gemm(A, B, 14))


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("where", ["A", "B"])
def test_nonfinite_input_flagged(dt, where):
    A, B = _pair(64, 96, 80, dt, None, seed=1)
    if where == "A":
        A[5, 7] = float("nan")
    else:
        B[9, 3] = float("inf")
    moa.gemm(A.cuda(), B.cuda(), dt)
    assert moa.moa_sync_status(0) == moa.MOA_ERR_NONFINITE
    assert moa.moa_sync_status(0) == moa.MOA_OK


def test_full_size_sampled_rows():
    """m = n = p = 8192 FP32 inputs, row-scaled (each row of A and of B times
    10^U(-4,4)), in the launch configuration the benchmark times: 8 sampled
    rows of C equal the exact integer product of those rows."""
    N = 8192
    A, B = inputs.normal_pair(N, N, N, dtype=torch.float32, seed=0, scaled="rows")
    C = moa.gemm(A.cuda(), B.cuda(), moa.MOA_F64_CRT_F32IN)
    moa.sync_status()
    rows = inputs.sample_rows(N, 8, seed=2)
    got = C[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    Ad = A.double().numpy()[rows]
    Bd = B.double().numpy()
    # A's scaling is per row, so a subset of rows scales as in the full call
    want = oracle.crt_gemm(Ad, Bd, 14)
    assert np.array_equal(got, want)
    assert _rel(got, oracle.gemm(Ad, Bd)) <= 1e-12


def test_empty_shapes():
    for m, n, p in [(0, 5, 7), (5, 0, 7), (5, 7, 0)]:
        A = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        B = torch.zeros((n, p), dtype=torch.float32, device="cuda")
        C = torch.full((m, p), float("nan"), dtype=torch.float64, device="cuda")
        moa.gemm(A, B, moa.MOA_F64_CRT_F32IN, C=C)
        moa.sync_status()
        assert torch.equal(C.cpu(), torch.zeros((m, p), dtype=torch.float64))
