"""CPU oracle for the MoA ONF GEMM -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2306_11148_b300``) and never imports
it; the two meet only through the seeded input generators.

The arithmetic lives in ``moa_oracle.c`` (plain C, FP64, no fused
multiply-add).  This module compiles it with gcc on first use and wraps each
function with ctypes over numpy arrays.

Functions and the passages they follow:

* :func:`gemm` -- Eq. (eq:dnf), Sec. 2: ``C[i*p+j] := sum_k A[i*n+k] B[k*p+j]``
  in the i-k-j order of Fig. ip.c.
* :func:`gemm_rows` -- the same for a sample of rows i.
* :func:`gemm_omp` -- rows dealt to threads (the i-loop lift, Sec. 3.1,
  Fig. ip_rows.c); bit-identical to :func:`gemm`.
* :func:`split3_bf16` -- FP32-accuracy slicing (not in the paper).
* :func:`slice_fixed` -- FP64-accuracy integer-digit slicing (not in the paper).
* :func:`split_gemm_exact` -- the exact value the digit-slice product reaches.
* :func:`crt_moduli`, :func:`crt_bits`, :func:`scale_int`,
  :func:`int_gemm_exact` -- FP64 accuracy from modular slices (not in the
  paper): operands scaled per row / column to integers of at most ``t`` bits,
  their exact integer product, rounded once.
* :func:`kronecker`, :func:`hadamard` -- the Appendix's other products of the
  inner/outer-product family.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmoa_oracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``moa_oracle.c`` into ``libmoa_oracle.so`` (next to it)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-std=c11", "-Wall", "-Wextra", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.moa_oracle_gemm_f64.argtypes = [_i64, _i64, _i64, _ptr, _ptr, _ptr]
            lib.moa_oracle_gemm_f64.restype = None
            lib.moa_oracle_gemm_f64_rows.argtypes = [_i64, _i64, _i64, _ptr, _ptr,
                                                     _i64, _ptr, _ptr]
            lib.moa_oracle_gemm_f64_rows.restype = None
            lib.moa_oracle_gemm_f64_omp.argtypes = [_i64, _i64, _i64, _ptr, _ptr, _ptr,
                                                    ctypes.c_int]
            lib.moa_oracle_gemm_f64_omp.restype = ctypes.c_int
            lib.moa_oracle_split3_bf16.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr]
            lib.moa_oracle_split3_bf16.restype = None
            lib.moa_oracle_slice_fixed.argtypes = [_i64, _i64, _ptr, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   _ptr, _ptr]
            lib.moa_oracle_slice_fixed.restype = None
            lib.moa_oracle_split_gemm_exact.argtypes = [_i64, _i64, _i64, _ptr, _ptr,
                                                        _ptr, _ptr, ctypes.c_int,
                                                        ctypes.c_int, _ptr]
            lib.moa_oracle_split_gemm_exact.restype = None
            lib.moa_oracle_crt_moduli.argtypes = [ctypes.c_int, _ptr]
            lib.moa_oracle_crt_moduli.restype = None
            lib.moa_oracle_crt_bits.argtypes = [_i64, ctypes.c_int]
            lib.moa_oracle_crt_bits.restype = ctypes.c_int
            lib.moa_oracle_scale_int.argtypes = [_i64, _i64, _ptr, ctypes.c_int, ctypes.c_int,
                                                 _ptr, _ptr]
            lib.moa_oracle_scale_int.restype = None
            lib.moa_oracle_int_gemm_exact.argtypes = [_i64, _i64, _i64, _ptr, _ptr, _ptr, _ptr,
                                                      ctypes.c_int, _ptr]
            lib.moa_oracle_int_gemm_exact.restype = None
            lib.moa_oracle_kronecker_f64.argtypes = [_i64, _i64, _i64, _i64, _ptr, _ptr, _ptr]
            lib.moa_oracle_kronecker_f64.restype = None
            lib.moa_oracle_hadamard_f64.argtypes = [_i64, _i64, _ptr, _ptr, _ptr]
            lib.moa_oracle_hadamard_f64.restype = None
            _lib = lib
    return _lib


def _f64(x) -> np.ndarray:
    """Exact conversion of FP64/FP32/integer (or BF16-valued) arrays to FP64."""
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def gemm(A, B) -> np.ndarray:
    """C = A . B in FP64 (Eq. eq:dnf), i-k-j order (Fig. ip.c)."""
    A = _f64(A)
    B = _f64(B)
    m, n = A.shape
    n2, p = B.shape
    if n != n2:
        raise ValueError("inner dimensions differ")
    C = np.empty((m, p), dtype=np.float64)
    _load().moa_oracle_gemm_f64(m, n, p, _p(A), _p(B), _p(C))
    return C


def gemm_rows(A, B, rows) -> np.ndarray:
    """Rows ``rows`` of A . B (FP64), as a len(rows) x p array."""
    A = _f64(A)
    B = _f64(B)
    m, n = A.shape
    n2, p = B.shape
    if n != n2:
        raise ValueError("inner dimensions differ")
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= m):
        raise ValueError("row index out of range")
    C = np.empty((rows.size, p), dtype=np.float64)
    _load().moa_oracle_gemm_f64_rows(m, n, p, _p(A), _p(B), rows.size, _p(rows), _p(C))
    return C


def gemm_omp(A, B, threads: int = 0):
    """A . B with rows dealt to OpenMP threads; returns (C, threads_used)."""
    A = _f64(A)
    B = _f64(B)
    m, n = A.shape
    n2, p = B.shape
    if n != n2:
        raise ValueError("inner dimensions differ")
    C = np.empty((m, p), dtype=np.float64)
    used = _load().moa_oracle_gemm_f64_omp(m, n, p, _p(A), _p(B), _p(C), int(threads))
    return C, int(used)


def split3_bf16(x):
    """(s0, s1, s2) with s_t = RN_bf16(x - sum_{u<t} s_u); BF16 values as FP32."""
    x = np.ascontiguousarray(np.asarray(x), dtype=np.float32)
    s = [np.empty_like(x) for _ in range(3)]
    _load().moa_oracle_split3_bf16(x.size, _p(x), _p(s[0]), _p(s[1]), _p(s[2]))
    return tuple(s)


def slice_fixed(X, axis: int, beta: int, S: int, headroom: int = 0):
    """Per-group exponents and S integer digits of radix 2^beta.

    ``axis=0``: one exponent per row; ``axis=1``: one per column.
    ``headroom``: bits left unused above the top digit (the exponent is the
    group's frexp exponent plus ``headroom``, so |d_0| <= 2^(beta - headroom)).
    Returns ``(exps int32[groups], digits int32[S, rows, cols])``.
    """
    X = _f64(X)
    rows, cols = X.shape
    exps = np.empty(rows if axis == 0 else cols, dtype=np.int32)
    digits = np.empty((S, rows, cols), dtype=np.int32)
    if not 0 <= headroom < beta:
        raise ValueError("headroom must lie in [0, beta)")
    _load().moa_oracle_slice_fixed(rows, cols, _p(X), int(axis), int(beta), int(S),
                                   int(headroom), _p(exps), _p(digits))
    return exps, digits


def split_gemm_exact(dA, eA, dB, eB, beta: int, S: int) -> np.ndarray:
    """Exact value of the triangular digit-slice product, rounded once to FP64."""
    dA = np.ascontiguousarray(dA, dtype=np.int32)
    dB = np.ascontiguousarray(dB, dtype=np.int32)
    eA = np.ascontiguousarray(eA, dtype=np.int32)
    eB = np.ascontiguousarray(eB, dtype=np.int32)
    _, m, n = dA.shape
    _, n2, p = dB.shape
    if n != n2:
        raise ValueError("inner dimensions differ")
    C = np.empty((m, p), dtype=np.float64)
    _load().moa_oracle_split_gemm_exact(m, n, p, _p(dA), _p(eA), _p(dB), _p(eB),
                                        int(beta), int(S), _p(C))
    return C


def crt_moduli(M: int) -> list:
    """The first M integers of 256, 255, ... coprime to all taken before."""
    if not 1 <= M <= 20:
        raise ValueError("M must lie in [1, 20]")
    out = np.zeros(M, dtype=np.int32)
    _load().moa_oracle_crt_moduli(int(M), _p(out))
    return [int(x) for x in out]


def crt_bits(n: int, M: int) -> int:
    """Largest t <= 62 with n * 2^(2t+1) < (product of the first M moduli)."""
    if not 1 <= M <= 16 or n < 1:
        raise ValueError("needs 1 <= M <= 16 and n >= 1")
    return int(_load().moa_oracle_crt_bits(int(n), int(M)))


def scale_int(X, axis: int, t: int):
    """Per-row (axis 0) or per-column (axis 1) exponents e and the integers
    rint(x * 2^(t - e)); returns (exps int32[groups], ints int64[rows, cols])."""
    X = _f64(X)
    rows, cols = X.shape
    if not 0 <= t <= 62:
        raise ValueError("t must lie in [0, 62]")
    exps = np.empty(rows if axis == 0 else cols, dtype=np.int32)
    ints = np.empty((rows, cols), dtype=np.int64)
    _load().moa_oracle_scale_int(rows, cols, _p(X), int(axis), int(t), _p(exps), _p(ints))
    return exps, ints


def int_gemm_exact(Ai, eA, Bi, eB, t: int) -> np.ndarray:
    """(Ai . Bi)[i,j] * 2^(eA_i + eB_j - 2t), the product exact, rounded once."""
    Ai = np.ascontiguousarray(Ai, dtype=np.int64)
    Bi = np.ascontiguousarray(Bi, dtype=np.int64)
    eA = np.ascontiguousarray(eA, dtype=np.int32)
    eB = np.ascontiguousarray(eB, dtype=np.int32)
    m, n = Ai.shape
    n2, p = Bi.shape
    if n != n2:
        raise ValueError("inner dimensions differ")
    C = np.empty((m, p), dtype=np.float64)
    _load().moa_oracle_int_gemm_exact(m, n, p, _p(Ai), _p(eA), _p(Bi), _p(eB), int(t), _p(C))
    return C


def crt_gemm(A, B, M: int) -> np.ndarray:
    """The value the modular-slice method reaches for A . B with M moduli:
    t = crt_bits(n, M); A scaled per row, B per column; exact product."""
    A = _f64(A)
    B = _f64(B)
    n = A.shape[1]
    t = crt_bits(max(n, 1), M)
    eA, Ai = scale_int(A, 0, t)
    eB, Bi = scale_int(B, 1, t)
    return int_gemm_exact(Ai, eA, Bi, eB, t)


def kronecker(A, B) -> np.ndarray:
    """C[(i*p)+k, (j*q)+l] = A[i,j] * B[k,l] in FP64."""
    A = _f64(A)
    B = _f64(B)
    m, n = A.shape
    p, q = B.shape
    C = np.empty((m * p, n * q), dtype=np.float64)
    _load().moa_oracle_kronecker_f64(m, n, p, q, _p(A), _p(B), _p(C))
    return C


def hadamard(A, B) -> np.ndarray:
    """C[i,j] = A[i,j] * B[i,j] in FP64."""
    A = _f64(A)
    B = _f64(B)
    if A.shape != B.shape:
        raise ValueError("shapes differ")
    C = np.empty(A.shape, dtype=np.float64)
    _load().moa_oracle_hadamard_f64(A.shape[0], A.shape[1], _p(A), _p(B), _p(C))
    return C
