"""Pins for the CPU oracle (CPU only).

The oracle states Eq. (eq:dnf) (Sec. 2) in the i-k-j order of Fig. ip.c.  The
paper prints no worked numeric example, so these tests pin it to what the
mathematics fixes instead: exact integer arithmetic, identity and permutation
matrices, the transpose identity, associativity on integers, exact rational
evaluation within Higham's dot-product bound, the n = 1 and n = 0 special
cases, and the dimension-lifted loop orders of Sec. 3.1 (Figs. ip_rows.c,
ip_cols.c), which visit the same products in the same order per element.

Each pin is also run against deliberately broken variants of the oracle
(dropped term, wrong sign, transposed operand, swapped operands, off-by-one
index) to show that every such mistake fails at least one pin.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs

RNG = np.random.default_rng(1234)
SHAPES = [(1, 1, 1), (3, 5, 7), (17, 33, 9), (64, 64, 64), (31, 129, 15), (8, 1, 8)]


# --------------------------------------------------------------------------
# Pin checks, written as predicates over a GEMM function f(A, B) -> C so that
# the same checks can be run on the oracle and on broken variants of it.
# --------------------------------------------------------------------------

def pin_integer_exact(f, m=17, n=33, p=9, seed=0):
    A, B = inputs.integer_pair(m, n, p, seed=seed)
    A = A.numpy()
    B = B.numpy()
    exact = A.astype(np.int64) @ B.astype(np.int64)   # integer arithmetic, exact
    C = f(A, B)
    return C.shape == exact.shape and np.array_equal(C, exact.astype(np.float64))


def pin_identity_permutation(f, n=12, seed=3):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (n, n + 3))
    I_l = np.eye(n)
    I_r = np.eye(n + 3)
    perm = rng.permutation(n)
    P = np.eye(n)[perm]                        # (P A)[i] = A[perm[i]]
    q = rng.permutation(n + 3)
    Q = np.eye(n + 3)[:, q]                    # (A Q)[:, j] = A[:, q[j]]
    return (np.array_equal(f(I_l, A), A) and np.array_equal(f(A, I_r), A)
            and np.array_equal(f(P, A), A[perm]) and np.array_equal(f(A, Q), A[:, q]))


def pin_transpose(f, m=7, n=11, p=5, seed=5):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (m, n))
    B = rng.uniform(-1, 1, (n, p))
    # (B^T A^T)^T multiplies the same pairs in the same k order: bit-identical.
    return np.array_equal(f(B.T.copy(), A.T.copy()).T, f(A, B))


def pin_associative_integers(f, seed=7):
    rng = np.random.default_rng(seed)
    A = rng.integers(-8, 9, (6, 9)).astype(np.float64)
    B = rng.integers(-8, 9, (9, 4)).astype(np.float64)
    Cm = rng.integers(-8, 9, (4, 10)).astype(np.float64)
    return np.array_equal(f(f(A, B), Cm), f(A, f(B, Cm)))


def pin_rational_bound(f, m=6, n=8, p=5, seed=11):
    """|C - C_exact| <= gamma_n |A||B| elementwise (Higham, Thm 3.5), with the
    exact product evaluated in rational arithmetic from the FP64 inputs."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (m, n)) * 2.0 ** rng.integers(-20, 20, (m, n))
    B = rng.uniform(-1, 1, (n, p)) * 2.0 ** rng.integers(-20, 20, (n, p))
    C = f(A, B)
    if C.shape != (m, p):
        return False
    u = 2.0 ** -53
    gamma = n * u / (1 - n * u)
    absAB = np.abs(A) @ np.abs(B)
    for i in range(m):
        for j in range(p):
            exact = sum((Fraction(A[i, k]) * Fraction(B[k, j]) for k in range(n)), Fraction(0))
            if abs(Fraction(C[i, j]) - exact) > Fraction(gamma) * Fraction(absAB[i, j]) * 1.0000001:
                return False
    return True


PINS = [pin_integer_exact, pin_identity_permutation, pin_transpose,
        pin_associative_integers, pin_rational_bound]


# --------------------------------------------------------------------------
# The oracle passes every pin.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_passes_pin(pin):
    assert pin(oracle.gemm)


@pytest.mark.parametrize("m,n,p", SHAPES)
def test_integer_exact_shapes(m, n, p):
    assert pin_integer_exact(oracle.gemm, m, n, p, seed=m * 1000 + n)


def test_integer_exact_largest_partial_sum():
    # All entries -8 or 8 with n = 4096: |partial sums| reach 64 * 4096 = 2^18.
    n = 4096
    A = np.full((2, n), 8.0)
    A[1, ::2] = -8.0
    B = np.full((n, 3), 8.0)
    B[:, 1] = -8.0
    C = oracle.gemm(A, B)
    exact = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C, exact.astype(np.float64))


def test_rational_bound_square_small():
    for N in range(1, 9):
        assert pin_rational_bound(oracle.gemm, N, N, N, seed=100 + N)


def test_summation_order_and_unfused_products():
    """Reading of Eq. (eq:dnf)/Fig. ip.c: products rounded separately, summed
    for k = 0..n-1 ascending starting from 0.0.  Python floats are IEEE FP64
    and never fuse, so the expected value is fixed by that reading alone."""
    rng = np.random.default_rng(99)
    for _ in range(200):
        n = int(rng.integers(2, 6))
        a = rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-8, 8, n)
        b = rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-8, 8, n)
        expected = 0.0
        for k in range(n):
            expected = expected + float(a[k]) * float(b[k])
        got = oracle.gemm(a[None, :], b[:, None])[0, 0]
        assert got == expected


def test_outer_product_n1():
    rng = np.random.default_rng(2)
    a = rng.uniform(-1, 1, (9, 1))
    b = rng.uniform(-1, 1, (1, 13))
    C = oracle.gemm(a, b)
    for i in range(9):
        for j in range(13):
            assert C[i, j] == float(a[i, 0]) * float(b[0, j])   # one rounding


def test_empty_inner_dimension_gives_zero():
    C = oracle.gemm(np.zeros((4, 0)), np.zeros((0, 6)))
    assert C.shape == (4, 6) and np.all(C == 0.0)


def test_empty_outer_dimensions():
    assert oracle.gemm(np.zeros((0, 5)), np.ones((5, 3))).shape == (0, 3)
    assert oracle.gemm(np.ones((3, 5)), np.ones((5, 0))).shape == (3, 0)


def test_dimension_lifted_forms_bit_identical():
    """Figs. ip_rows.c (i = ip + (m/np)*k over np processors) and ip_cols.c
    (j = jp*rsize + kp) visit, for each C element, the same products in the
    same sigma order, so they reproduce the generic form bit for bit."""
    rng = np.random.default_rng(4)
    m, n, p, np_, rsize = 8, 5, 16, 4, 8
    A = rng.uniform(-1, 1, (m, n))
    B = rng.uniform(-1, 1, (n, p))
    Af, Bf = A.ravel(), B.ravel()
    rows = np.zeros(m * p)
    for k in range(np_):
        for ip in range(m // np_):
            i = ip + (m // np_) * k
            for sigma in range(n):
                for j in range(p):
                    rows[j + i * p] = rows[j + i * p] + Af[i * n + sigma] * Bf[sigma * p + j]
    cols = np.zeros(m * p)
    for i in range(m):
        for sigma in range(n):
            for jp in range(p // rsize):
                for kp in range(rsize):
                    j = jp * rsize + kp
                    cols[j + i * p] = cols[j + i * p] + Af[i * n + sigma] * Bf[sigma * p + j]
    C = oracle.gemm(A, B).ravel()
    assert np.array_equal(rows, C)
    assert np.array_equal(cols, C)


def test_omp_and_rows_bit_identical():
    A, B = inputs.uniform_pair(37, 50, 23, seed=0)
    A, B = A.numpy(), B.numpy()
    C = oracle.gemm(A, B)
    Comp, used = oracle.gemm_omp(A, B, threads=3)
    assert used >= 1 and np.array_equal(Comp, C)
    rows = inputs.sample_rows(37, 10)
    assert np.array_equal(oracle.gemm_rows(A, B, rows), C[rows])


def test_oracle_matches_float128_reference_within_rounding():
    # A second, independent evaluation route: numpy longdouble (x87 80-bit on
    # x86) summation of the same products; differences stay within gamma_n.
    A, B = inputs.uniform_pair(20, 300, 10, seed=2)
    A, B = A.numpy(), B.numpy()
    C = oracle.gemm(A, B)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble))
    n = A.shape[1]
    bound = (n * 2.0 ** -53 / (1 - n * 2.0 ** -53)) * (np.abs(A) @ np.abs(B)) * 1.01
    assert np.all(np.abs(C - ref.astype(np.float64)) <= bound + 1e-300)


# --------------------------------------------------------------------------
# Planted mistakes (in the oracle, on the CPU) fail at least one pin.
# --------------------------------------------------------------------------

def _dropped_last_term(A, B):
    if A.shape[1] == 0:
        return oracle.gemm(A, B)
    return oracle.gemm(A[:, :-1], B[:-1, :])


def _wrong_sign(A, B):
    C = oracle.gemm(A, B)
    if C.size:
        C = C.copy()
        C[-1, -1] = -C[-1, -1]
    return C


def _transposed_b(A, B):
    # reads B as if it were stored column-major (B[j*n+k] instead of B[k*p+j])
    n, p = B.shape
    Bt = np.ascontiguousarray(B).ravel().reshape(p, n).T
    return oracle.gemm(A, Bt)


def _swapped_operands(A, B):
    if A.shape[0] == A.shape[1] == B.shape[0] == B.shape[1]:
        return oracle.gemm(B, A)
    return oracle.gemm(A, B) * 1.0000001


def _off_by_one_row(A, B):
    # each row i of C built from row i+1 of A (wrapping)
    return oracle.gemm(np.roll(A, -1, axis=0), B)


def _fused_products(A, B):
    # the same sums with higher-precision products (a different definition)
    C = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    return C


@pytest.mark.parametrize("mutant", [_dropped_last_term, _wrong_sign, _transposed_b,
                                    _swapped_operands, _off_by_one_row, _fused_products],
                         ids=lambda f: f.__name__)
def test_planted_mistake_fails_a_pin(mutant):
    results = {pin.__name__: pin(mutant) for pin in PINS}
    results["summation_order"] = _order_pin(mutant)
    assert not all(results.values()), results


def _order_pin(f):
    rng = np.random.default_rng(123)
    for _ in range(50):
        n = 4
        a = rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-8, 8, n)
        b = rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-8, 8, n)
        expected = 0.0
        for k in range(n):
            expected = expected + float(a[k]) * float(b[k])
        if f(a[None, :], b[:, None])[0, 0] != expected:
            return False
    return True


# --------------------------------------------------------------------------
# Slicing oracles (precision modes; not in the paper).
# --------------------------------------------------------------------------

def _fp32_edge_values():
    f = np.float32
    tiny = np.finfo(np.float32).tiny
    vals = [0.0, -0.0, 1.0, -1.0, tiny, -tiny, tiny / 8, 1e-30, 3.0e38, -3.0e38,
            1.0 + 2.0 ** -23, 1.0 - 2.0 ** -24, 2.0 ** -126 * 1.5, 65504.0, 1.0 / 3.0]
    return np.array(vals, dtype=f)


def test_split3_reconstructs_exactly():
    rng = np.random.default_rng(8)
    x = np.concatenate([
        rng.standard_normal(200000).astype(np.float32),
        (rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000)).astype(np.float32),
        rng.integers(-2 ** 31, 2 ** 31, 5000).astype(np.int32).view(np.float32),
        _fp32_edge_values(),
    ])
    x = x[np.isfinite(x) & (np.abs(x) < 3.3e38)]
    s0, s1, s2 = oracle.split3_bf16(x)
    total = s0.astype(np.float64) + s1.astype(np.float64) + s2.astype(np.float64)
    # Exact reconstruction (FP64 holds the sum of three BF16 values exactly)
    # whenever the last slice stays above BF16's subnormal quantum 2^-133,
    # i.e. |x| >= 2^-110; below that the lost bits are under 2^-134.
    normal = (np.abs(x) >= 2.0 ** -110) | (x == 0)
    assert np.array_equal(total[normal], x.astype(np.float64)[normal])
    assert np.all(np.abs(total - x.astype(np.float64)) <= 2.0 ** -134)
    # every slice is a BF16 value: low 16 bits clear
    for s in (s0, s1, s2):
        assert np.all((s.view(np.uint32) & 0xFFFF) == 0)
    # the first slice is torch's round-to-nearest-even conversion to BF16
    t0 = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(s0, t0)
    t1 = torch.from_numpy(x - s0).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(s1, t1)


def test_split3_special_values():
    x = np.array([np.inf, -np.inf, np.nan], dtype=np.float32)
    s0, _, _ = oracle.split3_bf16(x)
    assert s0[0] == np.inf and s0[1] == -np.inf and np.isnan(s0[2])


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("beta,S,h", [(8, 6, 0), (7, 7, 0), (8, 3, 0), (8, 7, 0), (5, 10, 1),
                                      (5, 6, 1), (4, 12, 1)])
def test_slice_fixed_reconstruction_bound(axis, beta, S, h):
    rng = np.random.default_rng(10 + axis + beta + S)
    X = rng.standard_normal((13, 17)) * 10.0 ** rng.uniform(-4, 4, (13, 1))
    X[3, :] = 0.0
    X[:, 5] = 0.0
    exps, digits = oracle.slice_fixed(X, axis, beta, S, headroom=h)
    # exponent: 2^(e-h-1) <= max|x| < 2^(e-h) per group (e = h for all-zero groups)
    mx = np.abs(X).max(axis=1 - axis)
    for g, e in enumerate(exps):
        if mx[g] == 0:
            assert e == h
        else:
            assert math.ldexp(1.0, int(e) - h - 1) <= mx[g] < math.ldexp(1.0, int(e) - h)
    # digit ranges: |d_0| <= 2^(beta-h), d_s in [-2^(beta-1), 2^(beta-1)) for s >= 1
    assert np.all(np.abs(digits[0]) <= 2 ** (beta - h))
    assert np.all(digits[1:] >= -2 ** (beta - 1)) and np.all(digits[1:] < 2 ** (beta - 1))
    # exact reconstruction bound |x - 2^e sum_s d_s 2^-beta(s+1)| <= 2^(e - beta S) / 2
    for r in range(X.shape[0]):
        for c in range(X.shape[1]):
            e = int(exps[r] if axis == 0 else exps[c])
            approx = sum(Fraction(int(digits[s, r, c])) * Fraction(2) ** (e - beta * (s + 1))
                         for s in range(S))
            err = abs(Fraction(X[r, c]) - approx)
            assert err <= Fraction(2) ** (e - beta * S) / 2


def test_slice_fixed_headroom_top_digit_reaches_its_bound():
    # x just below the group's power of two rounds up to D = 2^(beta S - h):
    # the top digit is then exactly 2^(beta - h) and every other digit is 0.
    X = np.array([[1.0 - 2.0 ** -53, 0.25]])
    for beta, S, h in [(5, 10, 1), (7, 7, 0)]:
        exps, digits = oracle.slice_fixed(X, 0, beta, S, headroom=h)
        assert int(exps[0]) == h
        assert int(digits[0, 0, 0]) == 2 ** (beta - h)
        assert np.all(digits[1:, 0, 0] == 0)


def test_headroom_one_radix_32_digits_are_e4m3_values():
    # The FP8 E4M3 slice planes need every digit exactly representable in
    # E4M3 (3 stored mantissa bits: all integers of magnitude <= 16).  The
    # check uses torch's own float8_e4m3fn rounding, which the oracle does
    # not use.
    rng = np.random.default_rng(33)
    X = rng.standard_normal((40, 50)) * 10.0 ** rng.uniform(-4, 4, (40, 1))
    X[0, :3] = [1.0 - 2.0 ** -53, -(1.0 - 2.0 ** -53), 2.0 ** -1074]
    for axis in (0, 1):
        _, digits = oracle.slice_fixed(X, axis, 5, 10, headroom=1)
        d = torch.from_numpy(digits.astype(np.float32))
        back = d.to(torch.float8_e4m3fn).to(torch.float32)
        assert torch.equal(back, d)
        assert int(np.abs(digits).max()) <= 16
    # without the headroom bit the top digit can reach 32, which E4M3 cannot
    # hold for every integer up to it (17 is not an E4M3 value)
    assert torch.tensor([17.0]).to(torch.float8_e4m3fn).float().item() != 17.0


def test_slice_fixed_integers_exact_digits():
    A, _ = inputs.integer_pair(5, 9, 3, seed=4)
    X = A.numpy()
    exps, digits = oracle.slice_fixed(X, 0, 8, 4)
    for r in range(5):
        e = int(exps[r])
        # integers |x| <= 8 need one digit: d_0 = x * 2^(beta - e), rest zero
        assert np.array_equal(digits[0, r], (X[r] * 2.0 ** (8 - e)).astype(np.int32))
        assert np.all(digits[1:, r] == 0)


def test_split_gemm_exact_integer_inputs_bit_exact():
    A, B = inputs.integer_pair(11, 40, 7, seed=9)
    A, B = A.numpy(), B.numpy()
    eA, dA = oracle.slice_fixed(A, 0, 8, 6)
    eB, dB = oracle.slice_fixed(B, 1, 8, 6)
    C = oracle.split_gemm_exact(dA, eA, dB, eB, 8, 6)
    assert np.array_equal(C, (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("beta,S,h", [(8, 6, 0), (7, 7, 0), (5, 10, 1)])
def test_split_gemm_exact_close_to_fp64_product(beta, S, h):
    A, B = inputs.normal_pair(24, 64, 20, dtype=torch.float64, seed=1, scaled="rows")
    A, B = A.numpy(), B.numpy()
    eA, dA = oracle.slice_fixed(A, 0, beta, S, headroom=h)
    eB, dB = oracle.slice_fixed(B, 1, beta, S, headroom=h)
    C = oracle.split_gemm_exact(dA, eA, dB, eB, beta, S)
    ref = oracle.gemm(A, B)
    # Truncation bound per element: each operand digit expansion is within
    # 2^(e - beta S)/2 and the dropped cross levels are below
    # S * 2^(eA+eB) * 2^(-beta S); summed over n terms.
    mA = 2.0 ** eA.astype(np.float64)
    mB = 2.0 ** eB.astype(np.float64)
    bound = A.shape[1] * (S + 2) * np.outer(mA, mB) * 2.0 ** (-beta * S)
    assert np.all(np.abs(C - ref) <= bound)
    rel = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert rel < 1e-12


def _digits_by_fractions(x, e, beta, S):
    """Exact-rational route: D = round-half-even(x * 2^(beta S - e)), then
    balanced base-2^beta digits taken from the bottom."""
    D = round(Fraction(x) * Fraction(2) ** (beta * S - e))   # Fraction.__round__: half to even
    out = [0] * S
    radix, half = 2 ** beta, 2 ** (beta - 1)
    for s in range(S - 1, 0, -1):
        low = D % radix
        if low >= half:
            low -= radix
        out[s] = low
        D = (D - low) // radix
    out[0] = D
    return out


def test_slice_fixed_matches_exact_rational_route():
    rng = np.random.default_rng(21)
    X = rng.standard_normal((9, 11)) * 10.0 ** rng.uniform(-6, 6, (9, 11))
    # exact ties: values whose scaled form ends in exactly one half unit
    X[0, 0] = 1.0 + 2.0 ** -48          # with e = 1, beta S = 48: X = 2^47 + 0.5
    X[0, 1] = -(1.0 + 3 * 2.0 ** -48)
    X[1, :] = 2.0 ** -1074              # subnormal row
    for beta, S, h in [(8, 6, 0), (7, 7, 0), (8, 3, 0), (5, 10, 1)]:
        exps, digits = oracle.slice_fixed(X, 0, beta, S, headroom=h)
        for r in range(X.shape[0]):
            for c in range(X.shape[1]):
                want = _digits_by_fractions(X[r, c], int(exps[r]), beta, S)
                assert [int(digits[s, r, c]) for s in range(S)] == want


# --------------------------------------------------------------------------
# Kronecker and Hadamard products (the Appendix's product family).
# --------------------------------------------------------------------------

def test_kronecker_mixed_product_property():
    # (A (x) B)(C (x) D) = (A C) (x) (B D), exact on small integers
    rng = np.random.default_rng(31)
    A = rng.integers(-3, 4, (3, 4)).astype(float)
    Cm = rng.integers(-3, 4, (4, 2)).astype(float)
    B = rng.integers(-3, 4, (2, 5)).astype(float)
    D = rng.integers(-3, 4, (5, 3)).astype(float)
    lhs = oracle.gemm(oracle.kronecker(A, B), oracle.kronecker(Cm, D))
    rhs = oracle.kronecker(oracle.gemm(A, Cm), oracle.gemm(B, D))
    assert np.array_equal(lhs, rhs)


def test_kronecker_identities_and_layout():
    assert np.array_equal(oracle.kronecker(np.eye(3), np.eye(4)), np.eye(12))
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    B = np.array([[0.0, 5.0], [6.0, 7.0]])
    # block (i, j) of A (x) B is A[i, j] * B
    K = oracle.kronecker(A, B)
    for i in range(2):
        for j in range(2):
            assert np.array_equal(K[2 * i:2 * i + 2, 2 * j:2 * j + 2], A[i, j] * B)
    # a 1 x 1 factor is a scalar multiple
    assert np.array_equal(oracle.kronecker(np.array([[3.0]]), B), 3.0 * B)


def test_hadamard_identities():
    rng = np.random.default_rng(32)
    A = rng.integers(-8, 9, (7, 9)).astype(float)
    B = rng.integers(-8, 9, (7, 9)).astype(float)
    assert np.array_equal(oracle.hadamard(A, B), oracle.hadamard(B, A))
    assert np.array_equal(oracle.hadamard(A, np.ones_like(A)), A)
    # sum of all entries of A o B = trace(A^T B), exact on integers
    assert oracle.hadamard(A, B).sum() == np.trace(oracle.gemm(A.T.copy(), B))
    # one rounding per element
    x = rng.uniform(-1, 1, (3, 4))
    y = rng.uniform(-1, 1, (3, 4))
    h = oracle.hadamard(x, y)
    assert all(h[i, j] == float(x[i, j]) * float(y[i, j]) for i in range(3) for j in range(4))


# --------------------------------------------------------------------------
# Regression records (tests/golden): the oracle must reproduce them bit for bit.
# --------------------------------------------------------------------------

def test_oracle_reproduces_golden_records():
    from golden_io import read_record
    r = read_record("gemm_int_7x9x5.txt")
    assert np.array_equal(oracle.gemm(r["A"], r["B"]), r["C"])
    # integer inputs: the record is also the exact integer product
    assert np.array_equal(r["C"], (r["A"].astype(np.int64) @ r["B"].astype(np.int64)))
    r = read_record("gemm_uniform_6x10x4.txt")
    assert np.array_equal(oracle.gemm(r["A"], r["B"]), r["C"])
    r = read_record("split_exact_b7_s4_5x12x3.txt")
    eA, dA = oracle.slice_fixed(r["A"], 0, 7, 4)
    eB, dB = oracle.slice_fixed(r["B"], 1, 7, 4)
    assert np.array_equal(oracle.split_gemm_exact(dA, eA, dB, eB, 7, 4), r["C"])



def _triangle_by_fractions(dA, eA, dB, eB, beta, S, width):
    """Exact-rational route of the digit-slice product over the levels
    s + t <= width (the method keeps width = S - 1), rounded once (Python's
    float of a Fraction rounds to nearest, ties to even)."""
    _, m, n = dA.shape
    p = dB.shape[2]
    C = np.empty((m, p))
    for i in range(m):
        for j in range(p):
            acc = Fraction(0)
            for s in range(S):
                for t in range(S):
                    if s + t > width:
                        continue
                    dot = sum(int(dA[s, i, k]) * int(dB[t, k, j]) for k in range(n))
                    acc += Fraction(dot) * Fraction(2) ** (-beta * (s + t + 2))
            C[i, j] = float(acc * Fraction(2) ** (int(eA[i]) + int(eB[j])))
    return C


@pytest.mark.parametrize("beta,S,h", [(7, 4, 1), (5, 5, 1), (8, 3, 0)])
def test_split_gemm_exact_keeps_exactly_the_triangle(beta, S, h):
    """Two-sided pin of the level set: the oracle equals the exact-rational sum
    over s + t <= S - 1 and differs from the sums over one level fewer and one
    level more (row-scaled inputs, where the dropped levels are visible)."""
    A, B = inputs.normal_pair(3, 7, 4, dtype=torch.float64, seed=13, scaled="rows")
    A, B = A.numpy(), B.numpy()
    eA, dA = oracle.slice_fixed(A, 0, beta, S, headroom=h)
    eB, dB = oracle.slice_fixed(B, 1, beta, S, headroom=h)
    C = oracle.split_gemm_exact(dA, eA, dB, eB, beta, S)
    assert np.array_equal(C, _triangle_by_fractions(dA, eA, dB, eB, beta, S, S - 1))
    assert not np.array_equal(C, _triangle_by_fractions(dA, eA, dB, eB, beta, S, S - 2))
    assert not np.array_equal(C, _triangle_by_fractions(dA, eA, dB, eB, beta, S, S))
