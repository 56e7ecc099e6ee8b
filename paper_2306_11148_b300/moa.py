"""Thin ctypes binding over libmoa.so (the C ABI declared in include/moa.h).

Every function here only marshals arguments: device memory comes from
PyTorch tensors, streams from ``torch.cuda.Stream``, and every step of the
GEMM runs in the library's CUDA kernels.  If libmoa.so is missing or cannot
be loaded, :func:`lib` raises -- there is no CPU fallback.

Low-level names mirror the C ABI (``moa_gemm``, ``moa_gemm_ex``,
``moa_gemm_workspace_size``, ``moa_gemm_grouped``, ``moa_sync_status`` ...);
:func:`gemm` and :func:`gemm_grouped` are convenience wrappers over them.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmoa.so")

# moa_status
MOA_OK = 0
MOA_ERR_ARG = -1
MOA_ERR_DTYPE = -2
MOA_ERR_ALIGN = -3
MOA_ERR_WORKSPACE = -4
MOA_ERR_NONFINITE = -5
MOA_ERR_CUDA = -6
MOA_ERR_TIMEOUT = -7
MOA_ERR_BUDGET = -8
MOA_ERR_REJECTED = -9
MOA_ERR_BUSY = -10
MOA_ERR_UNSUPPORTED = -11

# moa_dtype
MOA_F64 = 0
MOA_F32_TF32 = 1
MOA_F32_SIMT = 2
MOA_BF16 = 3
MOA_F32_SPLIT = 4
MOA_F64_SPLIT_F32IN = 5
MOA_F64_SPLIT_F64IN = 6
MOA_F64_SPLIT_F32IN_E4M3 = 7
MOA_F64_SPLIT_F64IN_E4M3 = 8
MOA_F64_CRT_F32IN = 9
MOA_F64_CRT_F64IN = 10

MODES = {
    "f64": MOA_F64, "tf32": MOA_F32_TF32, "f32_simt": MOA_F32_SIMT, "bf16": MOA_BF16,
    "f32_split": MOA_F32_SPLIT, "f64_split_f32in": MOA_F64_SPLIT_F32IN,
    "f64_split_f64in": MOA_F64_SPLIT_F64IN,
    "f64_split_f32in_e4m3": MOA_F64_SPLIT_F32IN_E4M3,
    "f64_split_f64in_e4m3": MOA_F64_SPLIT_F64IN_E4M3,
    "f64_crt_f32in": MOA_F64_CRT_F32IN, "f64_crt_f64in": MOA_F64_CRT_F64IN,
}
# FP64-accuracy modes (FP64 output) and their digit format: (radix bits, headroom bits)
F64_ACCURATE = (MOA_F64, MOA_F64_SPLIT_F32IN, MOA_F64_SPLIT_F64IN, MOA_F64_SPLIT_F32IN_E4M3,
                MOA_F64_SPLIT_F64IN_E4M3, MOA_F64_CRT_F32IN, MOA_F64_CRT_F64IN)
# modular-slice modes (slices = number of moduli)
CRT = (MOA_F64_CRT_F32IN, MOA_F64_CRT_F64IN)
DIGITS = {MOA_F64_SPLIT_F32IN: (7, 1), MOA_F64_SPLIT_F64IN: (7, 1),
          MOA_F64_SPLIT_F32IN_E4M3: (5, 1), MOA_F64_SPLIT_F64IN_E4M3: (5, 1)}
DEFAULT_SLICES = {MOA_F32_SPLIT: 3, MOA_F64_SPLIT_F32IN: 7, MOA_F64_SPLIT_F64IN: 7,
                  MOA_F64_SPLIT_F32IN_E4M3: 10, MOA_F64_SPLIT_F64IN_E4M3: 10}


# moa_product_kind
MOA_GROUPED_ALONE, MOA_GROUPED_BF16, MOA_GROUPED_CRT, MOA_GROUPED_F32_SPLIT = 0, 1, 2, 3
MOA_PRODUCT_HADAMARD = 0
MOA_PRODUCT_KRONECKER = 1
MOA_PRODUCT_MATMUL = 2


class moa_stats(ctypes.Structure):
    _fields_ = [("block_m", ctypes.c_int32), ("block_n", ctypes.c_int32),
                ("block_k", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("products", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("tiles", ctypes.c_int64), ("kernels", ctypes.c_int32),
                ("padded", ctypes.c_int32)]


class moa_gemm_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("p", ctypes.c_int64),
                ("dt", ctypes.c_int), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p)]


class moa_serve_config(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("max_inflight", ctypes.c_int), ("n_streams", ctypes.c_int),
                ("queue_capacity", ctypes.c_int), ("queue_deadline_s", ctypes.c_double)]


class moa_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int), ("dt", ctypes.c_int),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("p", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class moa_serve_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("inflight", ctypes.c_uint64),
                ("inflight_peak", ctypes.c_int), ("arena_peak", ctypes.c_size_t),
                ("arena_used", ctypes.c_size_t), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MoaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"moa status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t

# Symbols the library exports (the declarations of include/moa.h).
EXPORTS = {
    "moa_gemm": (ctypes.c_int, [_i64, _i64, _i64, ctypes.c_int, _vp, _vp, _vp]),
    "moa_gemm_workspace_size": (_sz, [_i64, _i64, _i64, ctypes.c_int, ctypes.c_int]),
    "moa_gemm_host_workspace_size": (_sz, [_i64, _i64, _i64, ctypes.c_int, ctypes.c_int]),
    "moa_gemm_host": (ctypes.c_int, [_i64, _i64, _i64, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int,
                                     _vp, _sz, _vp, ctypes.POINTER(moa_stats)]),
    "moa_gemm_ex": (ctypes.c_int, [_i64, _i64, _i64, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int,
                                   _vp, _sz, _vp, ctypes.POINTER(moa_stats)]),
    "moa_gemm_grouped_workspace_size": (_sz, [ctypes.c_int, ctypes.POINTER(moa_gemm_desc)]),
    "moa_gemm_grouped": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(moa_gemm_desc), _vp, _sz,
                                        _vp]),
    "moa_gemm_f32split_noalloc": (ctypes.c_int, [_i64, _i64, _i64, _vp, _vp, _vp, _vp]),
    "moa_serve_create": (ctypes.c_int, [ctypes.POINTER(moa_serve_config),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "moa_serve_submit": (ctypes.c_int, [_vp, ctypes.POINTER(moa_gemm_desc),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "moa_serve_poll": (ctypes.c_int, [_vp, ctypes.POINTER(moa_completion), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "moa_serve_stats": (ctypes.c_int, [_vp, ctypes.POINTER(moa_serve_counters)]),
    "moa_serve_destroy": (ctypes.c_int, [_vp]),
    "moa_sync_status": (ctypes.c_int, [_vp]),
    "moa_last_error": (ctypes.c_char_p, []),
    "moa_set_wait_limit_ns": (ctypes.c_uint64, [ctypes.c_uint64]),
    "moa_version": (ctypes.c_char_p, []),
    "moa_profile_events": (ctypes.c_int, [_vp, _vp]),
    "moa_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_uint64, _vp]),
    "moa_set_block_n": (ctypes.c_int, [ctypes.c_int]),
    "moa_set_block_m": (ctypes.c_int, [ctypes.c_int]),
    "moa_grouped_path": (ctypes.c_int, [ctypes.POINTER(moa_gemm_desc)]),
    "moa_measure_fp64_rate": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)]),
    "moa_kronecker": (ctypes.c_int, [_i64, _i64, _i64, _i64, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "moa_hadamard": (ctypes.c_int, [_i64, _i64, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "moa_product": (ctypes.c_int, [ctypes.c_int, _i64, _i64, _i64, _i64, ctypes.c_int, _vp, _vp,
                                   _vp, _vp]),
    "moa_gemm_batched_workspace_size": (_sz, [ctypes.c_int, _i64, _i64, _i64, ctypes.c_int, _i64,
                                              _i64, _i64]),
    "moa_gemm_batched": (ctypes.c_int, [ctypes.c_int, _i64, _i64, _i64, ctypes.c_int, _vp, _i64,
                                        _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "moa_tune_dense": (ctypes.c_int, [_i64, _i64, _i64, ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _vp,
                                      ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_float)]),
    "moa_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "moa_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "moa_tune_clear": (ctypes.c_int, []),
    "moa_grouped_block_n": (ctypes.c_int, [_i64, _i64, _i64]),
    "moa_shutdown": (None, []),
}


def lib():
    """Loads libmoa.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmoa.so not built ({LIB_PATH}); run "
                                   "`python -m paper_2306_11148_b300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in EXPORTS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().moa_last_error().decode()


def check(status: int):
    if status != MOA_OK:
        raise MoaError(status, last_error())
    return status


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ---------------------------------------------------------------- raw ABI
def moa_gemm(m, n, p, dt, A, B, C) -> int:
    return lib().moa_gemm(m, n, p, dt, A, B, C)


def moa_gemm_workspace_size(m, n, p, dt, slices=0) -> int:
    return int(lib().moa_gemm_workspace_size(m, n, p, dt, slices))


def moa_gemm_ex(m, n, p, dt, A, B, C, slices, ws, ws_bytes, stream, stats=None) -> int:
    return lib().moa_gemm_ex(m, n, p, dt, A, B, C, slices, ws, ws_bytes, stream,
                             ctypes.byref(stats) if stats is not None else None)


def moa_gemm_host_workspace_size(m, n, p, dt, slices=0) -> int:
    return int(lib().moa_gemm_host_workspace_size(m, n, p, dt, slices))


def moa_gemm_host(m, n, p, dt, hA, hB, hC, slices, ws, ws_bytes, stream, stats=None) -> int:
    return lib().moa_gemm_host(m, n, p, dt, hA, hB, hC, slices, ws, ws_bytes, stream,
                               ctypes.byref(stats) if stats is not None else None)


def moa_sync_status(stream=0) -> int:
    return lib().moa_sync_status(stream)


def moa_set_wait_limit_ns(ns: int) -> int:
    return int(lib().moa_set_wait_limit_ns(ns))


def moa_version() -> str:
    return lib().moa_version().decode()


# ---------------------------------------------------------------- torch helpers
def out_dtype(dt: int):
    import torch
    return torch.float64 if dt in F64_ACCURATE else torch.float32


def in_dtype(dt: int):
    import torch
    if dt in (MOA_F64, MOA_F64_SPLIT_F64IN, MOA_F64_SPLIT_F64IN_E4M3, MOA_F64_CRT_F64IN):
        return torch.float64
    if dt == MOA_BF16:
        return torch.bfloat16
    return torch.float32


def check_tensors(A, B, C, dt):
    """Refuses operands whose dtype, device, layout or shape do not match the
    mode: the C ABI receives raw pointers and reads exactly what the mode
    implies (e.g. 8 bytes per element for FP64 inputs)."""
    import torch
    ind, outd = in_dtype(dt), out_dtype(dt)
    if A.dtype != ind or B.dtype != ind:
        raise TypeError(f"mode {dt} needs {ind} A and B, got {A.dtype} and {B.dtype}")
    if C is not None and C.dtype != outd:
        raise TypeError(f"mode {dt} writes {outd} C, got {C.dtype}")
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t is None:
            continue
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dim() != 2 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous row-major matrix")
    if A.shape[1] != B.shape[0]:
        raise ValueError("A must be m x n and B n x p")
    if C is not None and tuple(C.shape) != (A.shape[0], B.shape[1]):
        raise ValueError("C must be m x p")


class Workspace:
    """A growable device workspace owned by PyTorch (256-byte aligned)."""

    def __init__(self, device=None):
        self.buf = None
        self.device = device

    def get(self, nbytes: int):
        import torch
        if nbytes == 0:
            return 0, 0
        if self.buf is None or self.buf.numel() < nbytes + 256:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8,
                                   device=self.device or torch.device("cuda"))
        base = self.buf.data_ptr()
        aligned = (base + 255) // 256 * 256
        return aligned, nbytes


_default_ws = {}


def gemm(A, B, dt: int, C=None, slices: int = 0, stream=None, workspace: Workspace | None = None,
         stats: bool = False):
    """C := A . B through moa_gemm_ex on torch CUDA tensors (row-major, contiguous)."""
    import torch
    check_tensors(A, B, C, dt)
    m, n = A.shape
    p = B.shape[1]
    if C is None:
        C = torch.empty((m, p), dtype=out_dtype(dt), device=A.device)
    if workspace is None:
        workspace = _default_ws.setdefault(A.device, Workspace(A.device))
    need = moa_gemm_workspace_size(m, n, p, dt, slices)
    ws, wsb = workspace.get(need)
    st = moa_stats() if stats else None
    check(moa_gemm_ex(m, n, p, dt, _ptr(A), _ptr(B), _ptr(C), slices, ws, wsb,
                      _stream_handle(stream), st))
    return (C, st) if stats else C


def gemm_host(A, B, dt: int, C=None, slices: int = 0, stream=None,
              workspace: Workspace | None = None, stats: bool = False):
    """C := A . B through moa_gemm_host on torch CPU tensors (row-major,
    contiguous; page-locked ones let the copies overlap other streams' work).
    The library copies A and B to the device, runs the GEMM and copies C back;
    C holds the result once ``stream`` is synchronised."""
    import torch
    ind, outd = in_dtype(dt), out_dtype(dt)
    if A.dtype != ind or B.dtype != ind:
        raise TypeError(f"mode {dt} needs {ind} A and B, got {A.dtype} and {B.dtype}")
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t is None:
            continue
        if t.device.type != "cpu":
            raise ValueError(f"{name} must be a CPU tensor")
        if t.dim() != 2 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous row-major matrix")
    if A.shape[1] != B.shape[0]:
        raise ValueError("A must be m x n and B n x p")
    m, n = A.shape
    p = B.shape[1]
    if C is None:
        C = torch.empty((m, p), dtype=outd, pin_memory=A.is_pinned())
    elif C.dtype != outd or tuple(C.shape) != (m, p):
        raise ValueError(f"C must be an m x p {outd} tensor")
    dev = torch.device("cuda", torch.cuda.current_device())
    if workspace is None:
        workspace = _default_ws.setdefault(("host", dev), Workspace(dev))
    ws, wsb = workspace.get(moa_gemm_host_workspace_size(m, n, p, dt, slices))
    st = moa_stats() if stats else None
    check(moa_gemm_host(m, n, p, dt, A.data_ptr() if A.numel() else None,
                        B.data_ptr() if B.numel() else None, C.data_ptr() if C.numel() else None,
                        slices, ws, wsb, _stream_handle(stream), st))
    return (C, st) if stats else C


def sync_status(stream=None):
    check(moa_sync_status(_stream_handle(stream)))


def make_descs(problems):
    """ctypes array of moa_gemm_desc from [(A, B, C, dt), ...] torch tensors."""
    arr = (moa_gemm_desc * len(problems))()
    for i, (A, B, C, dt) in enumerate(problems):
        check_tensors(A, B, C, dt)
        arr[i].m, arr[i].n = A.shape
        arr[i].p = B.shape[1]
        arr[i].dt = dt
        arr[i].A = _ptr(A)
        arr[i].B = _ptr(B)
        arr[i].C = _ptr(C)
    return arr


def grouped_path(A, B, C, dt) -> int:
    """The path (MOA_GROUPED_*) the problem C := A . B takes in a grouped call."""
    d = make_descs([(A, B, C, dt)])
    return int(lib().moa_grouped_path(d))


def gemm_grouped(problems, stream=None, workspace: Workspace | None = None, descs=None):
    """Every C := A . B of ``problems`` ([(A, B, C, dt), ...]) in one
    moa_gemm_grouped call.  ``descs`` may pass a prebuilt make_descs() array."""
    if not problems:
        return
    if descs is None:
        descs = make_descs(problems)
    dev = problems[0][0].device
    if workspace is None:
        workspace = _default_ws.setdefault(dev, Workspace(dev))
    need = int(lib().moa_gemm_grouped_workspace_size(len(problems), descs))
    ws, wsb = workspace.get(need)
    check(lib().moa_gemm_grouped(len(problems), descs, ws, wsb, _stream_handle(stream)))


class Server:
    """The continuous-batching server (moa_serve_*) over a torch-owned arena."""

    def __init__(self, arena_bytes: int, max_inflight: int = 32, n_streams: int = 4,
                 queue_capacity: int = 0, queue_deadline_s: float = 0.0, device=None):
        import torch
        self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8,
                                 device=device or torch.device("cuda")) if arena_bytes else None
        base = 0 if self.arena is None else (self.arena.data_ptr() + 255) // 256 * 256
        self.cfg = moa_serve_config(base, arena_bytes, max_inflight, n_streams, queue_capacity,
                                    queue_deadline_s)
        self.h = ctypes.c_void_p()
        check(lib().moa_serve_create(ctypes.byref(self.cfg), ctypes.byref(self.h)))
        self._buf = (moa_completion * 4096)()

    def submit(self, A, B, C, dt):
        """Returns (status, ticket); status != MOA_OK means not queued."""
        d = make_descs([(A, B, C, dt)])
        t = ctypes.c_uint64()
        rc = lib().moa_serve_submit(self.h, d, ctypes.byref(t))
        return rc, t.value

    def poll(self):
        """Completions as (ticket, status, t_submit, t_start, t_done) tuples."""
        n = ctypes.c_int()
        out = []
        while True:
            check(lib().moa_serve_poll(self.h, self._buf, len(self._buf), ctypes.byref(n)))
            # copy out now: the buffer is overwritten by the next poll
            for i in range(n.value):
                c = self._buf[i]
                out.append((c.ticket, c.status, c.t_submit, c.t_start, c.t_done))
            if n.value < len(self._buf):
                return out

    def stats(self):
        st = moa_serve_counters()
        check(lib().moa_serve_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            check(lib().moa_serve_destroy(self.h))
            self.h = ctypes.c_void_p()


def gemm_batched(A, B, dt: int, C=None, stream=None, workspace: Workspace | None = None):
    """C[b] := A[b] . B[b] for 3-D torch tensors (batch x m x n, batch x n x p);
    a 2-D A or B is broadcast to every entry (stride 0)."""
    import torch
    a3 = A if A.dim() == 3 else A.unsqueeze(0)
    b3 = B if B.dim() == 3 else B.unsqueeze(0)
    batch = max(a3.shape[0], b3.shape[0])
    m, n = a3.shape[1:]
    p = b3.shape[2]
    if b3.shape[1] != n:
        raise ValueError("inner dimensions differ")
    for t, name in ((a3, "A"), (b3, "B")):
        if t.shape[0] not in (1, batch):
            raise ValueError(f"{name} batch must be 1 or {batch}")
        if t.dtype != in_dtype(dt) or not t.is_contiguous() or t.device.type != "cuda":
            raise TypeError(f"{name} must be a contiguous CUDA {in_dtype(dt)} tensor")
    sa = 0 if a3.shape[0] == 1 else m * n
    sb = 0 if b3.shape[0] == 1 else n * p
    if C is None:
        C = torch.empty((batch, m, p), dtype=out_dtype(dt), device=A.device)
    if C.shape != (batch, m, p) or C.dtype != out_dtype(dt) or not C.is_contiguous():
        raise ValueError("C must be a contiguous batch x m x p tensor of the mode's output dtype")
    if workspace is None:
        workspace = _default_ws.setdefault(A.device, Workspace(A.device))
    need = int(lib().moa_gemm_batched_workspace_size(batch, m, n, p, dt, sa, sb, m * p))
    ws, wsb = workspace.get(need)
    check(lib().moa_gemm_batched(batch, m, n, p, dt, _ptr(a3), sa, _ptr(b3), sb, _ptr(C), m * p,
                                 ws, wsb, _stream_handle(stream)))
    return C


def kronecker(A, B, dt: int, stream=None):
    """C := A (x) B ((m*p) x (n*q)) through moa_kronecker."""
    import torch
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != in_dtype(dt) or t.dim() != 2 or not t.is_contiguous() or t.device.type != "cuda":
            raise TypeError(f"{name} must be a contiguous 2-D CUDA {in_dtype(dt)} tensor")
    m, n = A.shape
    p, q = B.shape
    C = torch.empty((m * p, n * q), dtype=out_dtype(dt), device=A.device)
    check(lib().moa_kronecker(m, n, p, q, dt, _ptr(A), _ptr(B), _ptr(C), _stream_handle(stream)))
    return C


def product(kind: int, A, B, dt: int, stream=None):
    """C := the product `kind` (MOA_PRODUCT_HADAMARD / _KRONECKER / _MATMUL) of
    A and B through moa_product, the single outer-product kernel."""
    import torch
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != in_dtype(dt) or t.dim() != 2 or not t.is_contiguous() or t.device.type != "cuda":
            raise TypeError(f"{name} must be a contiguous 2-D CUDA {in_dtype(dt)} tensor")
    m, n = A.shape
    p, q = B.shape
    shape = {MOA_PRODUCT_HADAMARD: (m, n), MOA_PRODUCT_KRONECKER: (m * p, n * q),
             MOA_PRODUCT_MATMUL: (m, q)}[kind]
    C = torch.empty(shape, dtype=out_dtype(dt), device=A.device)
    check(lib().moa_product(kind, m, n, p, q, dt, _ptr(A), _ptr(B), _ptr(C),
                            _stream_handle(stream)))
    return C


def hadamard(A, B, dt: int, stream=None):
    """C := A o B through moa_hadamard."""
    import torch
    if A.shape != B.shape:
        raise ValueError("Hadamard operands must have the same shape")
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != in_dtype(dt) or t.dim() != 2 or not t.is_contiguous() or t.device.type != "cuda":
            raise TypeError(f"{name} must be a contiguous 2-D CUDA {in_dtype(dt)} tensor")
    C = torch.empty(A.shape, dtype=out_dtype(dt), device=A.device)
    check(lib().moa_hadamard(A.shape[0], A.shape[1], dt, _ptr(A), _ptr(B), _ptr(C),
                             _stream_handle(stream)))
    return C
