"""moa_gemm_host: the GEMM with A, B and C in host memory.

The library copies A and B to the device, runs the same kernels moa_gemm_ex
runs and copies C back, so the result must equal moa_gemm_ex's on device
copies bit for bit, in every mode, from page-locked and from pageable host
memory, and for independent calls overlapping on several streams.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

pytestmark = pytest.mark.gpu

MODES = [moa.MOA_F64_CRT_F32IN, moa.MOA_F64_CRT_F64IN, moa.MOA_F64_SPLIT_F32IN,
         moa.MOA_F32_SPLIT, moa.MOA_BF16, moa.MOA_F32_TF32, moa.MOA_F64]
NAMES = {v: k for k, v in moa.MODES.items()}


def _host_pair(m, n, p, dt, seed, pinned):
    A, B = inputs.normal_pair(m, n, p, dtype=moa.in_dtype(dt), seed=seed)
    if pinned:
        A, B = A.pin_memory(), B.pin_memory()
    return A, B


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("dt", MODES, ids=lambda d: NAMES[d])
def test_host_entry_equals_device_entry(dt, pinned):
    m, n, p = 257, 1030, 190
    A, B = _host_pair(m, n, p, dt, seed=dt + 40, pinned=pinned)
    C, st = moa.gemm_host(A, B, dt, stats=True)
    moa.sync_status()
    want = moa.gemm(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    assert C.device.type == "cpu" and C.is_pinned() == pinned
    assert torch.equal(C, want.cpu())
    assert st.kernels >= 1


def test_host_entry_modular_slices_match_the_oracle():
    m, n, p = 300, 2100, 520
    A, B = _host_pair(m, n, p, moa.MOA_F64_CRT_F32IN, seed=7, pinned=True)
    C = moa.gemm_host(A, B, moa.MOA_F64_CRT_F32IN)
    moa.sync_status()
    assert np.array_equal(C.numpy(), oracle.crt_gemm(A.double().numpy(), B.double().numpy(), 14))


@pytest.mark.parametrize("shape", [(5000, 700, 300), (2049, 1030, 514), (4100, 3000, 64)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dt", [moa.MOA_F64_CRT_F32IN, moa.MOA_F64_CRT_F64IN],
                         ids=lambda d: NAMES[d])
def test_host_entry_bands_equal_device_entry(dt, shape):
    """Modular slices with host buffers run A in bands of about 2048 rows
    (uploads, band GEMMs and downloads overlapping on their own streams):
    3, 2 and 2 bands here, the last one ragged; the result equals the
    device-side call bit for bit, and sampled rows equal the exact integer
    product."""
    m, n, p = shape
    A, B = _host_pair(m, n, p, dt, seed=m + p, pinned=True)
    C, st = moa.gemm_host(A, B, dt, stats=True)
    moa.sync_status()
    assert st.kernels > 4
    want = moa.gemm(A.cuda(), B.cuda(), dt)
    moa.sync_status()
    assert torch.equal(C, want.cpu())
    rows = inputs.sample_rows(m, 4, seed=3)
    exact = oracle.crt_gemm(A.double().numpy()[rows], B.double().numpy(), 14)
    assert np.array_equal(C.numpy()[rows], exact)


def test_host_entry_k_zero_gives_zeros():
    A = torch.zeros((5, 0), dtype=torch.float32)
    B = torch.zeros((0, 7), dtype=torch.float32)
    C = torch.full((5, 7), float("nan"), dtype=torch.float64)
    moa.gemm_host(A, B, moa.MOA_F64_CRT_F32IN, C=C)
    moa.sync_status()
    assert torch.equal(C, torch.zeros((5, 7), dtype=torch.float64))


def test_independent_calls_on_three_streams():
    """Six calls round-robin over three streams, each stream with its own
    workspace and output: every result equals its lone device-side GEMM."""
    dt = moa.MOA_F64_CRT_F32IN
    streams = [torch.cuda.Stream() for _ in range(3)]
    spaces = [moa.Workspace(torch.device("cuda")) for _ in range(3)]
    probs = [_host_pair(600 + 64 * i, 900, 500 - 32 * i, dt, seed=60 + i, pinned=True)
             for i in range(6)]
    # each workspace sized once for its largest call: a call reuses its
    # stream's workspace only after that stream's earlier work (stream order)
    for k in range(3):
        spaces[k].get(max(moa.moa_gemm_host_workspace_size(A.shape[0], A.shape[1], B.shape[1],
                                                           dt, 0)
                          for A, B in probs[k::3]))
    outs = []
    for i, (A, B) in enumerate(probs):
        outs.append(moa.gemm_host(A, B, dt, stream=streams[i % 3], workspace=spaces[i % 3]))
    torch.cuda.synchronize()
    for s in streams:
        moa.sync_status(s)
    for (A, B), C in zip(probs, outs):
        assert torch.equal(C, moa.gemm(A.cuda(), B.cuda(), dt).cpu())
