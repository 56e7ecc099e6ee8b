"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module only draws random numbers; it holds none of the GEMM's or the
slicing's arithmetic, and imports neither the CUDA library nor the oracle.
Every generator is a CPU ``torch.Generator`` seeded explicitly, so the same
call gives the same bits on any machine.

Workloads (all row-major, the layout of Eq. (eq:dnf)):

* ``square_uniform(N, dtype)``  -- i.i.d. uniform[-1, 1), A drawn before B
  (the square FP64/FP32 sizes of the scaling sweep).
* ``integer_pair(m, n, p)``     -- i.i.d. integers in {-8..8}: every partial
  sum stays below 2^24 for n <= 16384, so every precision path must be
  bit-exact on them.
* ``normal_pair(m, n, p, scaled=...)`` -- i.i.d. N(0, 1) FP32, optionally with
  each row of A and each row (or column) of B multiplied by 10^U(-4, 4).
* ``grouped_shapes(count)``     -- m, n, p log-uniform in [32, 2048], rounded to
  a multiple of 16.
* ``serve_arrivals(rate, seconds)`` -- Poisson arrival times and log-uniform
  request shapes with a precision tag.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def uniform_pair(m: int, n: int, p: int, dtype=torch.float64, seed: int = 0):
    """A (m x n), B (n x p) i.i.d. uniform[-1, 1) in ``dtype`` (A drawn first).

    BF16 operands are drawn in FP32 and rounded to BF16 by torch.
    """
    g = _gen(seed)
    draw = torch.float64 if dtype == torch.float64 else torch.float32
    A = torch.rand((m, n), generator=g, dtype=draw) * 2 - 1
    B = torch.rand((n, p), generator=g, dtype=draw) * 2 - 1
    return A.to(dtype).contiguous(), B.to(dtype).contiguous()


def square_uniform(N: int, dtype=torch.float64, seed: int = 0):
    return uniform_pair(N, N, N, dtype, seed)


def integer_pair(m: int, n: int, p: int, dtype=torch.float64, seed: int = 0):
    """A, B with i.i.d. integer entries in {-8, ..., 8}, stored as ``dtype``."""
    g = _gen(seed)
    A = torch.randint(-8, 9, (m, n), generator=g, dtype=torch.int64)
    B = torch.randint(-8, 9, (n, p), generator=g, dtype=torch.int64)
    return A.to(dtype).contiguous(), B.to(dtype).contiguous()


def normal_pair(m: int, n: int, p: int, dtype=torch.float32, seed: int = 0,
                scaled: str | None = None):
    """A, B i.i.d. N(0, 1).

    ``scaled``: ``None``; ``"rows"`` (each row of A and each row of B times its
    own 10^u, u ~ U(-4, 4)); ``"rowcol"`` (each row of A and each column of B).
    """
    g = _gen(seed)
    A = torch.randn((m, n), generator=g, dtype=torch.float64)
    B = torch.randn((n, p), generator=g, dtype=torch.float64)
    if scaled is not None:
        ua = torch.rand((m, 1), generator=g, dtype=torch.float64) * 8 - 4
        A = A * torch.pow(10.0, ua)
        if scaled == "rows":
            ub = torch.rand((n, 1), generator=g, dtype=torch.float64) * 8 - 4
        elif scaled == "rowcol":
            ub = torch.rand((1, p), generator=g, dtype=torch.float64) * 8 - 4
        else:
            raise ValueError(f"unknown scaling {scaled!r}")
        B = B * torch.pow(10.0, ub)
    return A.to(dtype).contiguous(), B.to(dtype).contiguous()


def grouped_shapes(count: int = 512, lo: int = 32, hi: int = 2048, mult: int = 16,
                   seed: int = 0):
    """``count`` (m, n, p) triples, each log-uniform in [lo, hi], rounded to ``mult``."""
    g = _gen(seed)
    u = torch.rand((count, 3), generator=g, dtype=torch.float64)
    v = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    r = torch.clamp(torch.round(v / mult) * mult, min=lo).to(torch.int64)
    return [tuple(int(x) for x in row) for row in r.tolist()]


def serve_arrivals(rate: float = 2000.0, seconds: float = 60.0, seed: int = 0,
                   mp_range=(64, 4096), n_range=(64, 8192), mult: int = 16):
    """Poisson arrivals: list of (t_arrival_s, m, n, p, tag) with tag in
    {"f32", "f64"} (FP32-accuracy or FP64-accuracy request), each w.p. 1/2.
    Shapes are log-uniform and rounded to ``mult``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    lmp = (math.log(mp_range[0]), math.log(mp_range[1]))
    ln_ = (math.log(n_range[0]), math.log(n_range[1]))
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        m = int(max(mult, round(math.exp(rng.uniform(*lmp)) / mult) * mult))
        p = int(max(mult, round(math.exp(rng.uniform(*lmp)) / mult) * mult))
        n = int(max(mult, round(math.exp(rng.uniform(*ln_)) / mult) * mult))
        tag = "f32" if rng.random() < 0.5 else "f64"
        out.append((t, m, n, p, tag))
    return out


def sample_rows(m: int, count: int = 64, seed: int = 0) -> np.ndarray:
    """A fixed, seed-derived sorted sample of ``count`` distinct row indices."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    count = min(count, m)
    return np.sort(rng.choice(m, size=count, replace=False)).astype(np.int64)
