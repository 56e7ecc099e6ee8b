"""Pins for the oracle of the FP64-accuracy modular-slice mode (CPU only).

That mode is not in the paper: it reaches FP64 accuracy for Eq. (eq:dnf) by
scaling each row of A and each column of B to integers of at most t bits,
forming their exact integer product and rounding it once.  The oracle states
exactly that value (``oracle.crt_gemm``); the GPU computes the same integer
product from residues modulo M small pairwise-coprime moduli.  These tests pin
the oracle's pieces to what the mathematics fixes:

* the moduli: pairwise coprime, at most 2^8, and the greedy descending choice
  (checked by factoring with sympy, independently of the oracle's gcd loop);
* the bit count t: the largest with n * 2^(2t+1) < P, checked with Python's
  big integers;
* the scaling: an exact-rational route (Fraction, Python's half-even round);
* the exact product: brute force in exact rationals, two cases worked by
  hand, integer inputs (where the method is exact end to end) against the
  FP64 GEMM oracle, and the elementwise truncation bound against the FP64
  GEMM oracle on random inputs.

Planted mistakes in the method (wrong scaling axis, one bit too many, floor
instead of round-to-nearest, a dropped exponent) each fail one of the pins.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import sympy
import torch

import oracle
from paper_2306_11148_b300 import inputs


def test_moduli_pairwise_coprime_bounded_descending():
    mods = oracle.crt_moduli(20)
    assert mods[:5] == [256, 255, 253, 251, 247]
    assert all(2 <= q <= 256 for q in mods)
    assert mods == sorted(mods, reverse=True)
    for i, a in enumerate(mods):
        for b in mods[i + 1:]:
            assert not set(sympy.factorint(a)) & set(sympy.factorint(b)), (a, b)
    # greedy: every skipped integer between the chosen ones shares a prime
    # with a larger chosen modulus
    chosen = set(mods)
    for c in range(mods[-1] + 1, 257):
        if c in chosen:
            continue
        primes = set(sympy.factorint(c))
        assert any(primes & set(sympy.factorint(q)) for q in mods if q > c), c
    # every prefix is the same choice
    for M in (1, 7, 14, 16):
        assert oracle.crt_moduli(M) == mods[:M]


def test_bits_bound_with_big_integers():
    rng = np.random.default_rng(7)
    ns = [1, 2, 3, 255, 256, 257, 1024, 2048, 8192, 16384, 32768, 65536] + \
        [int(x) for x in rng.integers(1, 1 << 24, 30)]
    for M in range(1, 17):
        P = math.prod(oracle.crt_moduli(M))
        for n in ns:
            t = oracle.crt_bits(n, M)
            if t < 0:
                assert n * 2 >= P
                continue
            assert n * 2 ** (2 * t + 1) < P, (n, M, t)
            assert t == 62 or n * 2 ** (2 * t + 3) >= P, (n, M, t)


def _scale_rational(X, axis, t):
    """Exponents and integers by exact rationals (independent route)."""
    rows, cols = X.shape
    groups = rows if axis == 0 else cols
    exps = []
    for g in range(groups):
        vals = X[g, :] if axis == 0 else X[:, g]
        mu = max(abs(float(v)) for v in vals)
        exps.append(0 if mu == 0.0 else math.frexp(mu)[1])
    ints = np.empty((rows, cols), dtype=object)
    for r in range(rows):
        for c in range(cols):
            e = exps[r] if axis == 0 else exps[c]
            ints[r, c] = round(Fraction(float(X[r, c])) * Fraction(2) ** (t - e))
    return exps, ints


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("t", [0, 5, 24, 47, 53, 62])
def test_scale_int_matches_exact_rational_route(axis, t):
    rng = np.random.default_rng(100 + 10 * axis + t)
    X = rng.standard_normal((9, 13)) * 10.0 ** rng.uniform(-6, 6, (9, 1))
    X[2, :] = 0.0                           # an all-zero row
    X[:, 3] = 0.0                           # an all-zero column
    X[4, 5] = 5e-324                        # subnormal
    X[5, 6] = -2.0 ** -1074 * 3
    X[6, :] = np.array([1.5, 2.5, -0.5, 3.5, 0.75, 1.25, 4.0, -4.0, 2.0, 1.0, 0.5, 0.25, -3.0])
    X = X.astype(np.float32).astype(np.float64) if t <= 24 else X
    exps, ints = oracle.scale_int(X, axis, t)
    e2, i2 = _scale_rational(X, axis, t)
    assert list(exps) == e2
    assert all(int(a) == b for a, b in zip(ints.ravel(), i2.ravel()))
    assert np.abs(ints).max() <= 2 ** t
    # every nonzero group's largest integer has its top bit at t - 1 or t
    for g in range(len(exps)):
        vals = np.abs(ints[g, :] if axis == 0 else ints[:, g])
        if vals.max() > 0:
            assert vals.max() >= 2 ** t // 2


def test_scale_int_ties_round_to_even():
    X = np.array([[0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 3.5, 1.0 / 1024]])
    # row max 3.5 -> e = 2; t = 2 scales by 1: ties go to the even integer
    _, ints = oracle.scale_int(X, 0, 2)
    assert list(ints[0]) == [0, 2, 2, 0, -2, -2, 4, 0]


def _exact_value(Ai, eA, Bi, eB, t):
    m, n = Ai.shape
    p = Bi.shape[1]
    C = np.empty((m, p))
    for i in range(m):
        for j in range(p):
            acc = sum(int(Ai[i, k]) * int(Bi[k, j]) for k in range(n))
            C[i, j] = float(Fraction(acc) * Fraction(2) ** (int(eA[i]) + int(eB[j]) - 2 * t))
    return C


def test_int_gemm_exact_brute_force():
    rng = np.random.default_rng(11)
    for m, n, p, bits in [(1, 1, 1, 62), (3, 4, 5, 60), (4, 7, 3, 40), (5, 8, 6, 61)]:
        Ai = rng.integers(-(2 ** bits), 2 ** bits, (m, n), dtype=np.int64)
        Bi = rng.integers(-(2 ** bits), 2 ** bits, (n, p), dtype=np.int64)
        eA = rng.integers(-40, 40, m).astype(np.int32)
        eB = rng.integers(-40, 40, p).astype(np.int32)
        t = 30
        got = oracle.int_gemm_exact(Ai, eA, Bi, eB, t)
        assert np.array_equal(got, _exact_value(Ai, eA, Bi, eB, t))
    # ties of the final rounding: 2^53 + 1 rounds to even
    Ai = np.array([[2 ** 53 + 1]], dtype=np.int64)
    Bi = np.array([[1]], dtype=np.int64)
    got = oracle.int_gemm_exact(Ai, np.zeros(1, np.int32), Bi, np.zeros(1, np.int32), 0)
    assert got[0, 0] == float(2 ** 53)


def _crt_gemm_variant(A, B, M, mistake=None):
    """The method with one planted mistake (None: as the oracle states it)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n = A.shape[1]
    t = oracle.crt_bits(max(n, 1), M)
    eA, Ai = oracle.scale_int(A, 0, t)
    eB, Bi = oracle.scale_int(B, 1, t)
    if mistake == "axis":        # B scaled per row instead of per column
        eB_r, Bi = oracle.scale_int(B, 0, t)
        eB = np.full(B.shape[1], int(eB_r.max()), dtype=np.int32)
        Bi = np.rint(np.ldexp(B, t - int(eB_r.max()))).astype(np.int64)
    elif mistake == "extra_bit":  # scale by one bit more than the exponent removes
        Ai = np.rint(np.ldexp(A, (t + 1) - eA[:, None])).astype(np.int64)
    elif mistake == "floor":     # truncate instead of rounding to nearest
        Ai = np.floor(np.ldexp(A, t - eA[:, None])).astype(np.int64)
    elif mistake == "exponent":  # B's exponent dropped from the final scale
        eB = np.zeros_like(eB)
    return oracle.int_gemm_exact(Ai, eA, Bi, eB, t)


def pin_crt_integer_exact(f):
    A, B = inputs.integer_pair(19, 45, 23, seed=4)
    return np.array_equal(f(A.numpy(), B.numpy(), 14), oracle.gemm(A.numpy(), B.numpy()))


def pin_crt_truncation_bound(f):
    """|C - A.B| <= sum_k (|a| db + da |b| + da db) + the final and the
    oracle's rounding, elementwise, on row-scaled N(0, 1) inputs."""
    ok = True
    for kind in (None, "rows", "rowcol"):
        A, B = inputs.normal_pair(24, 300, 20, dtype=torch.float32, seed=9, scaled=kind)
        A = A.double().numpy()
        B = B.double().numpy()
        M = 12
        n = A.shape[1]
        t = oracle.crt_bits(n, M)
        eA, _ = oracle.scale_int(A, 0, t)
        eB, _ = oracle.scale_int(B, 1, t)
        da = np.ldexp(1.0, eA - t - 1)[:, None]          # half a unit of A's grid
        db = np.ldexp(1.0, eB - t - 1)[None, :]
        absA, absB = np.abs(A), np.abs(B)
        trunc = absA.sum(1, keepdims=True) * db + da * absB.sum(0, keepdims=True) + n * da * db
        ref = oracle.gemm(A, B)
        gam = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
        bound = trunc + 2.0 ** -53 * np.abs(ref) * 2 + gam * (absA @ absB)
        C = f(A, B, M)
        ok = ok and bool(np.all(np.abs(C - ref) <= bound))
    return ok


def pin_crt_hand_examples(f):
    """Two cases worked by hand from the definition.
    (a) One modulus (P = 256), n = 1: t = 3 (1 * 2^7 < 256 <= 2^9).
        A = 0.99: e = 0, A' = rint(7.92) = 8; B = 1.0: e = 1, B' = rint(4) = 4;
        C = 32 * 2^(0 + 1 - 6) = 1.0.
    (b) One modulus, n = 2: t = 2 (2 * 2^5 < 256 <= 2 * 2^7).
        A = [0.75, -0.3]: e = 0, A' = rint([3, -1.2]) = [3, -1];
        B = [0.5, 0.25]^T: e = 0, B' = rint([2, 1]) = [2, 1];
        C' = 6 - 1 = 5, C = 5 * 2^-4 = 0.3125."""
    a = f(np.array([[0.99]]), np.array([[1.0]]), 1)
    b = f(np.array([[0.75, -0.3]]), np.array([[0.5], [0.25]]), 1)
    return a.shape == (1, 1) and a[0, 0] == 1.0 and b.shape == (1, 1) and b[0, 0] == 0.3125


def test_crt_hand_examples():
    assert oracle.crt_bits(1, 1) == 3 and oracle.crt_bits(2, 1) == 2
    assert pin_crt_hand_examples(lambda A, B, M: oracle.crt_gemm(A, B, M))


def test_crt_gemm_integer_inputs_bit_exact():
    assert pin_crt_integer_exact(lambda A, B, M: oracle.crt_gemm(A, B, M))


def test_crt_gemm_within_truncation_bound():
    assert pin_crt_truncation_bound(lambda A, B, M: oracle.crt_gemm(A, B, M))


def test_crt_gemm_equals_variant_without_mistake():
    A, B = inputs.normal_pair(7, 50, 6, dtype=torch.float32, seed=2, scaled="rows")
    assert np.array_equal(oracle.crt_gemm(A.numpy(), B.numpy(), 14),
                          _crt_gemm_variant(A.numpy(), B.numpy(), 14))


@pytest.mark.parametrize("mistake", ["axis", "extra_bit", "floor", "exponent"])
def test_planted_mistake_fails_a_crt_pin(mistake):
    f = lambda A, B, M: _crt_gemm_variant(A, B, M, mistake)   # noqa: E731
    assert not (pin_crt_integer_exact(f) and pin_crt_truncation_bound(f)
                and pin_crt_hand_examples(f)), mistake


def test_crt_gemm_fp64_accuracy_on_row_scaled_inputs():
    """At the mode's default of 14 moduli the exact product of the truncated
    operands is within 1e-12 (relative Frobenius) of the FP64 product."""
    for kind in (None, "rows", "rowcol"):
        A, B = inputs.normal_pair(32, 2048, 32, dtype=torch.float32, seed=0, scaled=kind)
        A = A.double().numpy()
        B = B.double().numpy()
        ref = oracle.gemm(A, B)
        C = oracle.crt_gemm(A, B, 14)
        assert np.linalg.norm(C - ref) / np.linalg.norm(ref) <= 1e-12, kind
