"""GPU parity of every precision mode of the ONF GEMM against the FP64 oracle.

C[(i*p)+j] := sum_k A[(i*n)+k] * B[(k*p)+j]  (Eq. eq:dnf, Sec. 2).

Two kinds of check per mode, through the C ABI (moa_gemm_ex):
* integer-valued inputs in {-8..8}: every partial sum is an integer below
  2^24, so every mode must be bit-exact against the oracle;
* random inputs (the workloads' distributions): relative Frobenius error
  against the oracle within the mode's stated tolerance.
Shapes span several 128-row tiles, ragged M/N/K tails, single rows/columns and
row pitches that are not a multiple of 16 bytes (padded by the library).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs
from paper_2306_11148_b300 import moa

pytestmark = pytest.mark.gpu

# Relative Frobenius tolerance per mode against the FP64 oracle.
TOL = {
    moa.MOA_F64: 1e-12,
    moa.MOA_F32_TF32: 5e-3,
    moa.MOA_F32_SIMT: 1e-5,
    moa.MOA_BF16: 1e-2,
    moa.MOA_F32_SPLIT: 1e-5,
    moa.MOA_F64_SPLIT_F32IN: 1e-12,
    moa.MOA_F64_SPLIT_F64IN: 1e-12,
    moa.MOA_F64_SPLIT_F32IN_E4M3: 1e-12,
    moa.MOA_F64_SPLIT_F64IN_E4M3: 1e-12,
}
ALL_MODES = list(TOL)
NAMES = {v: k for k, v in moa.MODES.items()}

SHAPES = [
    (1, 1, 1),
    (15, 17, 31),
    (33, 127, 129),
    (128, 64, 128),
    (129, 65, 257),
    (256, 256, 256),
    (300, 200, 520),
    (257, 1000, 200),
    (64, 4096, 96),
]


def _rel(C, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(C - ref) / (den if den > 0 else 1.0)


def _run(A, B, dt, slices=0):
    C = moa.gemm(A.cuda(), B.cuda(), dt, slices=slices)
    moa.sync_status()
    return C.cpu().double().numpy()


@pytest.mark.parametrize("dt", ALL_MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("m,n,p", SHAPES)
def test_integer_inputs_bit_exact(dt, m, n, p):
    A, B = inputs.integer_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m + 7 * n + 13 * p)
    C = _run(A, B, dt)
    ref = oracle.gemm(A.double().numpy(), B.double().numpy())
    assert np.array_equal(C, ref), f"max diff {np.abs(C - ref).max()}"


@pytest.mark.parametrize("dt", ALL_MODES, ids=lambda d: NAMES[d])
def test_small_shape_sweep_bit_exact(dt):
    """48 shapes drawn (seed 0) from m, n, p in 1..40 -- every tile is ragged
    in every direction -- on integer inputs: bit-exact against the oracle."""
    rng = np.random.default_rng(0)
    for m, n, p in rng.integers(1, 41, size=(48, 3)):
        m, n, p = int(m), int(n), int(p)
        A, B = inputs.integer_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m * 1600 + n * 40 + p)
        C = _run(A, B, dt)
        ref = oracle.gemm(A.double().numpy(), B.double().numpy())
        assert np.array_equal(C, ref), f"{m}x{n}x{p}: max diff {np.abs(C - ref).max()}"


@pytest.mark.parametrize("dt", ALL_MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("m,n,p", SHAPES)
def test_uniform_inputs_within_tolerance(dt, m, n, p):
    A, B = inputs.uniform_pair(m, n, p, dtype=moa.in_dtype(dt), seed=1)
    C = _run(A, B, dt)
    ref = oracle.gemm(A.double().numpy(), B.double().numpy())
    assert _rel(C, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", [moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN, moa.MOA_F32_TF32,
                                moa.MOA_F64_SPLIT_F32IN_E4M3], ids=lambda d: NAMES[d])
@pytest.mark.parametrize("scaled", [None, "rows", "rowcol"])
def test_normal_scaled_inputs(dt, scaled):
    A, B = inputs.normal_pair(200, 1536, 160, dtype=torch.float32, seed=3, scaled=scaled)
    C = _run(A, B, dt)
    ref = oracle.gemm(A.double().numpy(), B.double().numpy())
    assert _rel(C, ref) <= TOL[dt]


@pytest.mark.parametrize("dt,S", [pytest.param(dt, S, id=f"{NAMES[dt]}-S{S}")
                                  for dt, Ss in ((moa.MOA_F64_SPLIT_F64IN, (3, 4, 5, 6, 7, 8)),
                                                 (moa.MOA_F64_SPLIT_F64IN_E4M3, (4, 6, 8, 10, 12)))
                                  for S in Ss])
def test_f64_split_matches_exact_slice_product(dt, S):
    """The FP64-accuracy mode reaches the exact triangular slice product of
    the oracle's digits (radix 2^7 for BF16 planes; radix 2^5 with one
    headroom bit for E4M3 planes), up to the final FP64 rounding and the
    int64 total's dropped low bits (relative 2^-46 of the scale)."""
    beta, h = moa.DIGITS[dt]
    A, B = inputs.normal_pair(130, 700, 140, dtype=torch.float64, seed=5, scaled="rows")
    C = _run(A, B, dt, slices=S)
    eA, dA = oracle.slice_fixed(A.numpy(), 0, beta, S, headroom=h)
    eB, dB = oracle.slice_fixed(B.numpy(), 1, beta, S, headroom=h)
    exact = oracle.split_gemm_exact(dA, eA, dB, eB, beta, S)
    scale = np.outer(2.0 ** eA.astype(np.float64), 2.0 ** eB.astype(np.float64))
    assert np.all(np.abs(C - exact) <= scale * 2.0 ** -46 + np.abs(exact) * 2.0 ** -52)


@pytest.mark.parametrize("dt", [moa.MOA_F64_SPLIT_F64IN, moa.MOA_F64_SPLIT_F64IN_E4M3,
                                moa.MOA_F64_SPLIT_F32IN], ids=lambda d: NAMES[d])
@pytest.mark.parametrize("m,n,p", [(70, 4200, 140), (33, 4100, 257), (1, 8192, 3)])
def test_f64_split_k_exact_and_deterministic(dt, m, n, p):
    """Few output tiles and a long K: the slice GEMM cuts every tile's K range
    into slices run on separate SMs whose int64 folds add atomically into C.
    Integer adds are exact and order-free, so the result is still the exact
    slice product of the oracle's digits (to the final FP64 rounding and the
    dropped low bits) and bit-identical from call to call."""
    beta, h = moa.DIGITS[dt]
    A, B = inputs.normal_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m + p, scaled="rows")
    C1 = _run(A, B, dt)
    C2 = _run(A, B, dt)
    assert np.array_equal(C1, C2)
    S = moa.DEFAULT_SLICES[dt]
    eA, dA = oracle.slice_fixed(A.double().numpy(), 0, beta, S, headroom=h)
    eB, dB = oracle.slice_fixed(B.double().numpy(), 1, beta, S, headroom=h)
    exact = oracle.split_gemm_exact(dA, eA, dB, eB, beta, S)
    scale = np.outer(2.0 ** eA.astype(np.float64), 2.0 ** eB.astype(np.float64))
    assert np.all(np.abs(C1 - exact) <= scale * 2.0 ** -46 + np.abs(exact) * 2.0 ** -52)


def test_f64_split_k_many_slices_ragged():
    """Two output tiles and K = 32768: the K range is cut into 32 slices whose
    int64 folds meet in C; an odd p takes the scalar (non-vector) fold and
    convert paths.  Exact slice product of the oracle's digits, as above."""
    dt = moa.MOA_F64_SPLIT_F32IN
    beta, h = moa.DIGITS[dt]
    A, B = inputs.normal_pair(200, 32768, 23, dtype=moa.in_dtype(dt), seed=11, scaled="rows")
    C = _run(A, B, dt)
    S = moa.DEFAULT_SLICES[dt]
    eA, dA = oracle.slice_fixed(A.double().numpy(), 0, beta, S, headroom=h)
    eB, dB = oracle.slice_fixed(B.double().numpy(), 1, beta, S, headroom=h)
    exact = oracle.split_gemm_exact(dA, eA, dB, eB, beta, S)
    scale = np.outer(2.0 ** eA.astype(np.float64), 2.0 ** eB.astype(np.float64))
    assert np.all(np.abs(C - exact) <= scale * 2.0 ** -46 + np.abs(exact) * 2.0 ** -52)


@pytest.mark.parametrize("dt,m,n,p", [(moa.MOA_F64_SPLIT_F64IN, 300, 700, 520),
                                      (moa.MOA_F64_SPLIT_F32IN, 129, 1000, 777),
                                      (moa.MOA_F64_SPLIT_F64IN_E4M3, 300, 700, 520),
                                      (moa.MOA_F64_SPLIT_F32IN_E4M3, 129, 1000, 777)],
                         ids=["f64in-300x700x520", "f32in-129x1000x777",
                              "f64in-e4m3-300x700x520", "f32in-e4m3-129x1000x777"])
def test_f64_level_groups_exact_and_deterministic(dt, m, n, p):
    """K too short to cut (n < 1024) and few output tiles: the S levels of
    every tile are dealt onto separate work units (more units than tiles in
    the launch) whose int64 folds meet in C by atomic adds.  The result is
    still the exact slice product of the oracle's digits, to the final FP64
    rounding and the dropped low bits, and bit-identical from call to call."""
    beta, h = moa.DIGITS[dt]
    A, B = inputs.normal_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m + n, scaled="rows")
    Ad, Bd = A.cuda(), B.cuda()
    C1, st = moa.gemm(Ad, Bd, dt, stats=True)
    C2 = moa.gemm(Ad, Bd, dt)
    moa.sync_status()
    assert st.grid > st.tiles
    C1 = C1.cpu().double().numpy()
    assert np.array_equal(C1, C2.cpu().double().numpy())
    S = moa.DEFAULT_SLICES[dt]
    eA, dA = oracle.slice_fixed(A.double().numpy(), 0, beta, S, headroom=h)
    eB, dB = oracle.slice_fixed(B.double().numpy(), 1, beta, S, headroom=h)
    exact = oracle.split_gemm_exact(dA, eA, dB, eB, beta, S)
    scale = np.outer(2.0 ** eA.astype(np.float64), 2.0 ** eB.astype(np.float64))
    assert np.all(np.abs(C1 - exact) <= scale * 2.0 ** -46 + np.abs(exact) * 2.0 ** -52)


@pytest.mark.parametrize("m,n,p", [(48, 20000, 40), (130, 9000, 300)])
def test_f32_split_k_deterministic_and_accurate(m, n, p):
    """FP32-accuracy split with few tiles and a long K: the K range is cut
    into slices whose FP32 partial tiles are summed in slice order, so the
    result is bit-identical from call to call, exact on integer inputs and
    within the mode's tolerance on normal ones."""
    dt = moa.MOA_F32_SPLIT
    A, B = inputs.integer_pair(m, n, p, dtype=torch.float32, seed=m + n)
    C = _run(A, B, dt)
    assert np.array_equal(C, oracle.gemm(A.double().numpy(), B.double().numpy()))
    A, B = inputs.normal_pair(m, n, p, dtype=torch.float32, seed=m + p)
    C1 = _run(A, B, dt)
    C2 = _run(A, B, dt)
    assert np.array_equal(C1, C2)
    assert _rel(C1, oracle.gemm(A.double().numpy(), B.double().numpy())) <= TOL[dt]


def test_f32_split_slices_match_oracle_split():
    """The FP32-accuracy mode's result equals the six-product sum of the
    oracle's BF16 slices up to FP32 accumulation error: each of the 6n terms
    passes through at most 6n FP32 additions (unit roundoff 2^-24, taken twice
    for accumulators that truncate), so |C - six| <= 2 * 6n * 2^-24 * sum|s||t|."""
    A, B = inputs.normal_pair(96, 512, 80, dtype=torch.float32, seed=8)
    s = oracle.split3_bf16(A.numpy())
    t = oracle.split3_bf16(B.numpy())
    pairs = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]
    six = sum(oracle.gemm(s[i], t[j]) for i, j in pairs)
    abs_six = sum(oracle.gemm(np.abs(s[i]), np.abs(t[j])) for i, j in pairs)
    C = _run(A, B, moa.MOA_F32_SPLIT)
    n = A.shape[1]
    assert np.all(np.abs(C - six) <= 2 * 6 * n * 2.0 ** -24 * abs_six)


def test_zero_inner_dimension_gives_zero():
    for dt in ALL_MODES:
        C = torch.full((5, 7), 3.0, dtype=moa.out_dtype(dt), device="cuda")
        A = torch.empty((5, 0), dtype=moa.in_dtype(dt), device="cuda")
        B = torch.empty((0, 7), dtype=moa.in_dtype(dt), device="cuda")
        moa.gemm(A, B, dt, C=C)
        moa.sync_status()
        assert torch.all(C == 0)


def test_empty_outer_dimensions_touch_nothing():
    for dt in ALL_MODES:
        A = torch.ones((0, 5), dtype=moa.in_dtype(dt), device="cuda")
        B = torch.ones((5, 3), dtype=moa.in_dtype(dt), device="cuda")
        C = moa.gemm(A, B, dt)
        assert C.shape == (0, 3)


def test_nonfinite_input_reported_by_split_modes():
    for dt in (moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN, moa.MOA_F64_SPLIT_F32IN_E4M3):
        A, B = inputs.uniform_pair(64, 64, 64, dtype=torch.float32, seed=2)
        A[3, 5] = float("nan")
        moa.gemm(A.cuda(), B.cuda(), dt)
        assert moa.moa_sync_status(moa._stream_handle(None)) == moa.MOA_ERR_NONFINITE
        moa.sync_status()   # cleared


def test_plain_moa_gemm_entry_point():
    """moa_gemm (library-owned workspace, legacy default stream)."""
    A, B = inputs.uniform_pair(77, 131, 45, dtype=torch.float32, seed=4)
    Ad, Bd = A.cuda(), B.cuda()
    ref = oracle.gemm(A.double().numpy(), B.double().numpy())
    for dt in (moa.MOA_F32_TF32, moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN):
        C = torch.empty((77, 45), dtype=moa.out_dtype(dt), device="cuda")
        torch.cuda.synchronize()
        moa.check(moa.moa_gemm(77, 131, 45, dt, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr()))
        moa.check(moa.moa_sync_status(0))
        assert _rel(C.cpu().double().numpy(), ref) <= TOL[dt]


def test_deterministic_repeat():
    """Two runs give bit-identical results (catches pipeline races)."""
    A, B = inputs.uniform_pair(384, 2048, 512, dtype=torch.float32, seed=6)
    Ad, Bd = A.cuda(), B.cuda()
    for dt in (moa.MOA_F32_TF32, moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN,
               moa.MOA_F64_SPLIT_F32IN_E4M3):
        c1 = moa.gemm(Ad, Bd, dt).clone()
        c2 = moa.gemm(Ad, Bd, dt)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2)


@pytest.mark.parametrize("dt,N", [(moa.MOA_F32_TF32, 8192), (moa.MOA_BF16, 8192),
                                  (moa.MOA_F32_SPLIT, 8192), (moa.MOA_F64_SPLIT_F32IN, 8192),
                                  (moa.MOA_F64_SPLIT_F32IN_E4M3, 8192),
                                  (moa.MOA_F64, 2048), (moa.MOA_F32_SIMT, 4096)],
                         ids=lambda x: NAMES.get(x, str(x)) if isinstance(x, int) and x < 10 else str(x))
def test_full_size_sampled_rows(dt, N):
    """Workload sizes: 64 seed-chosen rows recomputed by the oracle."""
    if dt in (moa.MOA_F64,):
        A, B = inputs.square_uniform(N, torch.float64)
    else:
        A, B = inputs.normal_pair(N, N, N, dtype=moa.in_dtype(dt), seed=0)
    C = moa.gemm(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    rows = inputs.sample_rows(N, 64)
    got = C[torch.from_numpy(rows).cuda()].cpu().double().numpy()
    ref = oracle.gemm_rows(A.double().numpy(), B.double().numpy(), rows)
    assert _rel(got, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", [moa.MOA_BF16, moa.MOA_F32_TF32, moa.MOA_F32_SPLIT,
                                moa.MOA_F64_SPLIT_F32IN, moa.MOA_F64_SPLIT_F32IN_E4M3],
                         ids=lambda d: NAMES[d])
@pytest.mark.parametrize("m,n,p", [(1, 8192, 8192), (8192, 1, 8192), (8192, 8192, 1),
                                   (2, 3, 16384), (16384, 7, 5)])
def test_extreme_aspect_ratios(dt, m, n, p):
    """Single-row, single-column and K = 1 problems: one ragged tile edge in
    each direction; rows sampled against the oracle."""
    A, B = inputs.normal_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m + n + p)
    C = moa.gemm(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    rows = inputs.sample_rows(m, 16)
    got = C[torch.from_numpy(rows).cuda()].cpu().double().numpy()
    ref = oracle.gemm_rows(A.double().numpy(), B.double().numpy(), rows)
    assert _rel(got, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", [moa.MOA_F32_TF32, moa.MOA_F64_SPLIT_F64IN,
                                moa.MOA_F64_SPLIT_F64IN_E4M3], ids=lambda d: NAMES[d])
def test_largest_square_size(dt):
    """N = 16384, the largest size of the square sweep (FP64 operands: 3 x 2 GiB),
    on 8 sampled rows."""
    N = 16384
    A, B = inputs.square_uniform(N, moa.in_dtype(dt), seed=0)
    C = moa.gemm(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    rows = inputs.sample_rows(N, 8)
    got = C[torch.from_numpy(rows).cuda()].cpu().double().numpy()
    ref = oracle.gemm_omp(A[torch.from_numpy(rows)].double().numpy(), B.double().numpy())[0]
    assert _rel(got, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", ALL_MODES, ids=lambda d: NAMES[d])
def test_gpu_matches_golden_records(dt):
    """The CUDA path against the frozen oracle records of tests/golden:
    bit-exact on the integer record in every mode; the FP64 modes also on
    the uniform record within their tolerance."""
    from golden_io import read_record
    r = read_record("gemm_int_7x9x5.txt")
    tdt = moa.in_dtype(dt)
    C = _run(torch.from_numpy(r["A"]).to(tdt), torch.from_numpy(r["B"]).to(tdt), dt)
    assert np.array_equal(C, r["C"])
    if moa.in_dtype(dt) == torch.float64:
        r = read_record("gemm_uniform_6x10x4.txt")
        C = _run(torch.from_numpy(r["A"]), torch.from_numpy(r["B"]), dt)
        assert _rel(C, r["C"]) <= TOL[dt]

