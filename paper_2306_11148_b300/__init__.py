"""B300-native MoA ONF GEMM: C[(i*p)+j] := sum_k A[(i*n)+k] * B[(k*p)+j] (Eq. eq:dnf).

The compute path is ``libmoa.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/moa.h``); :mod:`paper_2306_11148_b300.moa` is the thin
ctypes binding over it.  Importing this package loads nothing; the library is
opened on first use and a missing or unloadable library is an error (there is
no CPU fallback).
"""

__all__ = ["moa", "inputs"]
