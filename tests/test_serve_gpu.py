"""The continuous-batching server (moa_serve_*).

* Each result is the same alone and in the mix: every request of a mixed
  batch (FP32-accuracy and FP64-accuracy split requests, BF16 and
  modular-slice requests; the small split-precision and BF16 ones share
  grouped launches) equals, bit for bit, the same GEMM computed
  alone through moa_gemm_ex, and a sample also matches the FP64 oracle within
  the mode's tolerance.
* Admission: a request whose workspace exceeds the arena is refused
  (MOA_ERR_BUDGET); a full queue refuses (MOA_ERR_BUSY); a request queued past
  its deadline completes as MOA_ERR_REJECTED; every queued ticket completes
  exactly once and the arena is empty after the drain.
* Continuous batching: requests are admitted in several batches while
  others run, and their device work overlaps.
Host-side failures only; no test faults or stalls the GPU.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2306_11148_b300 import inputs, moa

TOL = {moa.MOA_F32_SPLIT: 1e-5, moa.MOA_F64_SPLIT_F32IN: 1e-12, moa.MOA_BF16: 1e-5,
       moa.MOA_F64_SPLIT_F32IN_E4M3: 1e-12, moa.MOA_F64_CRT_F32IN: 1e-12}


def _req(m, n, p, dt, seed):
    tdt = torch.bfloat16 if dt == moa.MOA_BF16 else torch.float32
    A, B = inputs.normal_pair(m, n, p, dtype=tdt, seed=seed)
    C = torch.full((m, p), float("nan"), dtype=moa.out_dtype(dt), device="cuda")
    return A.cuda(), B.cuda(), C, dt


def _drain(srv, want, timeout=60.0):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout:
        for c in srv.poll():
            assert c[0] not in got, "ticket completed twice"
            got[c[0]] = c
        time.sleep(0.002)
    return got


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(40):
        m, p = (int(x) for x in rng.integers(1, 40, 2) * 16)
        n = int(rng.integers(1, 80)) * 16
        dt = [moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN, moa.MOA_BF16,
              moa.MOA_F64_SPLIT_F32IN_E4M3, moa.MOA_F64_CRT_F32IN][i % 5]
        reqs.append(_req(m, n, p, dt, seed=i))
    alone = [moa.gemm(A, B, dt) for A, B, C, dt in reqs]
    torch.cuda.synchronize()
    srv = moa.Server(arena_bytes=1 << 30, max_inflight=12, n_streams=4)
    try:
        tickets = {}
        for i, (A, B, C, dt) in enumerate(reqs):
            rc, t = srv.submit(A, B, C, dt)
            assert rc == moa.MOA_OK
            tickets[t] = i
        got = _drain(srv, len(reqs))
        assert set(got) == set(tickets)
        assert all(c[1] == moa.MOA_OK for c in got.values())
        st = srv.stats()
    finally:
        srv.close()
    torch.cuda.synchronize()
    for t, i in tickets.items():
        A, B, C, dt = reqs[i]
        assert torch.equal(C, alone[i]), f"request {i} differs from its alone result"
    for i in range(0, len(reqs), 5):
        A, B, C, dt = reqs[i]
        ref = oracle.gemm(A.double().cpu().numpy(), B.double().cpu().numpy())
        got_c = C.double().cpu().numpy()
        assert np.linalg.norm(got_c - ref) / np.linalg.norm(ref) <= TOL[dt]
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["arena_used"] == 0 and 0 < st["arena_peak"] <= 1 << 30
    assert st["batches"] >= 1 and st["p99_ms"] >= st["p50_ms"] > 0


@pytest.mark.gpu
def test_continuous_batching_overlaps_requests():
    # the big request runs for several milliseconds (21 BF16 slice products
    # of 4096 x 8192 x 4096); the small ones arrive once it has been admitted
    big = _req(4096, 8192, 4096, moa.MOA_F64_SPLIT_F32IN, seed=50)
    small = [_req(256, 512, 256, moa.MOA_F32_SPLIT, seed=60 + i) for i in range(8)]
    srv = moa.Server(arena_bytes=8 << 30, max_inflight=16, n_streams=4)
    try:
        rc, tb = srv.submit(*big)
        assert rc == moa.MOA_OK
        t0 = time.time()
        while srv.stats()["admitted"] < 1 and time.time() - t0 < 10:
            time.sleep(0.0002)
        ts = [srv.submit(*r)[1] for r in small]
        got = _drain(srv, 1 + len(small))
        st = srv.stats()
    finally:
        srv.close()
    assert st["batches"] >= 2            # admitted in more than one pass
    assert st["inflight_peak"] >= 2
    b = got[tb]
    # some small request started before the big one finished
    assert any(got[t][3] < b[4] for t in ts)


@pytest.mark.gpu
def test_budget_busy_and_deadline_paths():
    # arena too small for a split request's slices
    srv = moa.Server(arena_bytes=1 << 20, max_inflight=2, n_streams=1)
    try:
        A, B, C, dt = _req(512, 512, 512, moa.MOA_F32_SPLIT, seed=1)
        rc, _ = srv.submit(A, B, C, dt)
        assert rc == moa.MOA_ERR_BUDGET
        rc, _ = srv.submit(A, B, C, 77)
        assert rc == moa.MOA_ERR_DTYPE
    finally:
        srv.close()
    # one slot, short deadline, tiny queue: later requests are refused or rejected
    # the big request keeps the only slot busy for ~30 ms (21 BF16 slice
    # products of 8192^3), so the small ones queue well past their 2 ms deadline
    big = _req(8192, 8192, 8192, moa.MOA_F64_SPLIT_F32IN, seed=2)
    small = _req(64, 64, 64, moa.MOA_F32_SPLIT, seed=3)
    srv = moa.Server(arena_bytes=8 << 30, max_inflight=1, n_streams=1, queue_capacity=4,
                     queue_deadline_s=0.002)
    try:
        rc, tb = srv.submit(*big)
        assert rc == moa.MOA_OK
        time.sleep(0.001)
        codes = [srv.submit(*small) for _ in range(12)]
        queued = [t for rc, t in codes if rc == moa.MOA_OK]
        assert any(rc == moa.MOA_ERR_BUSY for rc, _ in codes)
        got = _drain(srv, 1 + len(queued))
        st = srv.stats()
    finally:
        srv.close()
    assert set(got) == {tb, *queued}                     # each ticket exactly once
    assert got[tb][1] == moa.MOA_OK
    assert any(got[t][1] == moa.MOA_ERR_REJECTED for t in queued)
    assert st["rejected"] >= 1 and st["arena_used"] == 0


def test_bad_configs_rejected_on_the_host():
    from paper_2306_11148_b300 import build as moa_build
    import ctypes
    moa_build.build()
    L = moa.lib()
    h = ctypes.c_void_p()
    assert L.moa_serve_create(None, ctypes.byref(h)) == moa.MOA_ERR_ARG
    cfg = moa.moa_serve_config(0, 1024, 4, 1, 0, 0.0)          # arena NULL with bytes
    assert L.moa_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == moa.MOA_ERR_ARG
    cfg = moa.moa_serve_config(256 + 8, 1024, 4, 1, 0, 0.0)    # misaligned arena
    assert L.moa_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == moa.MOA_ERR_ALIGN
    cfg = moa.moa_serve_config(256, 1024, 0, 1, 0, 0.0)        # no slots
    assert L.moa_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == moa.MOA_ERR_ARG
    cfg = moa.moa_serve_config(256, 1024, 4, 65, 0, 0.0)       # too many streams
    assert L.moa_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == moa.MOA_ERR_ARG
    assert L.moa_serve_destroy(None) == moa.MOA_ERR_ARG


@pytest.mark.gpu
def test_per_request_device_status():
    """A split-mode request with a NaN input completes as MOA_ERR_NONFINITE;
    its neighbours complete normally and the per-device status word stays
    clean (each request records into its own status slot)."""
    good = [_req(128, 256, 128, moa.MOA_F32_SPLIT, seed=70 + i) for i in range(3)]
    bad = _req(128, 256, 128, moa.MOA_F64_SPLIT_F32IN, seed=80)
    bad[0][5, 7] = float("nan")
    moa.check(moa.moa_sync_status(moa._stream_handle(None)))
    srv = moa.Server(arena_bytes=1 << 28, max_inflight=4, n_streams=2)
    try:
        tg = [srv.submit(*r)[1] for r in good[:2]]
        tb = srv.submit(*bad)[1]
        tg.append(srv.submit(*good[2])[1])
        got = _drain(srv, 4)
        st = srv.stats()
    finally:
        srv.close()
    assert got[tb][1] == moa.MOA_ERR_NONFINITE
    assert all(got[t][1] == moa.MOA_OK for t in tg)
    assert st["failed"] == 1 and st["completed"] == 3
    assert moa.moa_sync_status(moa._stream_handle(None)) == moa.MOA_OK


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [moa.MOA_F64_CRT_F32IN, moa.MOA_F32_SPLIT],
                         ids=["modular_slices", "f32_split"])
def test_grouped_split_requests_keep_their_own_status(dt):
    """Small modular-slice and FP32-accuracy split requests share grouped
    launches in the server; one with a NaN input completes as
    MOA_ERR_NONFINITE while the others, grouped with it or not, complete
    normally and equal their alone results bit for bit."""
    reqs = [_req(96 + 16 * i, 320, 80 + 16 * i, dt, seed=90 + i) for i in range(6)]
    assert all(moa.grouped_path(*r) in (moa.MOA_GROUPED_CRT, moa.MOA_GROUPED_F32_SPLIT)
               for r in reqs)
    bad = 2
    reqs[bad][0][3, 11] = float("nan")
    alone = {i: moa.gemm(A, B, dt) for i, (A, B, C, dt) in enumerate(reqs) if i != bad}
    torch.cuda.synchronize()
    moa.check(moa.moa_sync_status(moa._stream_handle(None)))
    srv = moa.Server(arena_bytes=1 << 28, max_inflight=8, n_streams=2)
    try:
        tickets = {srv.submit(*r)[1]: i for i, r in enumerate(reqs)}
        got = _drain(srv, len(reqs))
        st = srv.stats()
    finally:
        srv.close()
    torch.cuda.synchronize()
    assert set(got) == set(tickets)
    for t, i in tickets.items():
        if i == bad:
            assert got[t][1] == moa.MOA_ERR_NONFINITE
        else:
            assert got[t][1] == moa.MOA_OK, f"request {i}"
            assert torch.equal(reqs[i][2], alone[i]), f"request {i} differs from its alone result"
    assert st["failed"] == 1 and st["completed"] == len(reqs) - 1
    assert moa.moa_sync_status(moa._stream_handle(None)) == moa.MOA_OK
