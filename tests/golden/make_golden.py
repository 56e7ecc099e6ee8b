"""Writes the oracle regression records of tests/golden from the oracle alone.
Calls only oracle/ and the seeded input generators."""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2306_11148_b300 import inputs  # noqa: E402


def _mat(name, X):
    rows = [" ".join(float(v).hex() for v in r) for r in np.atleast_2d(X)]
    return [f"{name} {X.shape[0]} {X.shape[1]}"] + rows


def write(path, header, blocks):
    lines = [f"# {header}"]
    for name, X in blocks:
        lines += _mat(name, X)
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    A, B = inputs.integer_pair(7, 9, 5, dtype=torch.float64, seed=11)
    A, B = A.numpy(), B.numpy()
    write(os.path.join(HERE, "gemm_int_7x9x5.txt"),
          "oracle.gemm on integer inputs in {-8..8}, seed 11 (values as hex floats)",
          [("A", A), ("B", B), ("C", oracle.gemm(A, B))])
    A, B = inputs.uniform_pair(6, 10, 4, dtype=torch.float64, seed=12)
    A, B = A.numpy(), B.numpy()
    write(os.path.join(HERE, "gemm_uniform_6x10x4.txt"),
          "oracle.gemm on uniform[-1,1) FP64 inputs, seed 12 (values as hex floats)",
          [("A", A), ("B", B), ("C", oracle.gemm(A, B))])
    A, B = inputs.normal_pair(5, 12, 3, dtype=torch.float64, seed=13, scaled="rows")
    A, B = A.numpy(), B.numpy()
    eA, dA = oracle.slice_fixed(A, 0, 7, 4)
    eB, dB = oracle.slice_fixed(B, 1, 7, 4)
    C = oracle.split_gemm_exact(dA, eA, dB, eB, 7, 4)
    write(os.path.join(HERE, "split_exact_b7_s4_5x12x3.txt"),
          "oracle.split_gemm_exact of oracle.slice_fixed digits (radix 2^7, S = 4), "
          "normal inputs with rows scaled by 10^U(-4,4), seed 13 (hex floats)",
          [("A", A), ("B", B), ("C", C)])


if __name__ == "__main__":
    main()
