"""Reader for the text records of tests/golden (matrices of hex floats)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_record(name):
    """{matrix name: np.ndarray float64} of one record file."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        key, r, c = lines[i].split()
        r, c = int(r), int(c)
        rows = [[float.fromhex(v) for v in lines[i + 1 + k].split()] for k in range(r)]
        out[key] = np.array(rows, dtype=np.float64).reshape(r, c)
        i += 1 + r
    return out
