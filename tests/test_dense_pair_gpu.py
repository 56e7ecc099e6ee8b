"""Dense BF16 / TF32 GEMMs on 256 x 256 tiles of CTA pairs (moa_set_block_m(256)).

Each pair of SMs computes one 256 x 256 tile with cta_group::2 MMAs, each SM
holding its 128 rows of the tile in a double-buffered TMEM accumulator.  On
integer inputs (every product and partial sum exact in FP32) the result must
equal the FP64 oracle exactly; on random inputs it must equal the one-CTA
kernels bit for bit (every output sums the same products in the same K order),
at ragged shapes and with several tiles per cluster.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu

MODES = [moa.MOA_BF16, moa.MOA_F32_TF32]
NAMES = {v: k for k, v in moa.MODES.items()}
SHAPES = [(1, 8, 8), (64, 64, 64), (257, 1024, 264), (300, 1000, 520), (1024, 512, 2048),
          (4096, 256, 4096), (130, 3000, 600)]


def _run(A, B, dt, block_m):
    L = moa.lib()
    moa.check(L.moa_set_block_m(block_m))
    try:
        C, st = moa.gemm(A.cuda(), B.cuda(), dt, stats=True)
        moa.sync_status()
    finally:
        moa.check(L.moa_set_block_m(0))
    return C.cpu(), st


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_pair_tiles_exact_on_integers(dt, shape):
    m, n, p = shape
    A, B = inputs.integer_pair(m, n, p, dtype=moa.in_dtype(dt), seed=m + n + p)
    C, st = _run(A, B, dt, 256)
    assert st.block_m == 256 and st.block_n == 256 and st.grid % 2 == 0
    assert np.array_equal(C.double().numpy(), oracle.gemm(A.double().numpy(), B.double().numpy()))


@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
@pytest.mark.parametrize("shape", SHAPES[2:], ids=lambda s: "x".join(map(str, s)))
def test_pair_tiles_equal_one_cta_tiles(dt, shape):
    m, n, p = shape
    A, B = inputs.uniform_pair(m, n, p, dtype=moa.in_dtype(dt), seed=7 * m + p)
    pair, st = _run(A, B, dt, 256)
    one, st1 = _run(A, B, dt, 128)
    assert st.block_m == 256 and st1.block_m == 128
    assert torch.equal(pair, one)
