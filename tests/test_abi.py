"""The C-ABI boundary on the CPU: the library loads, exports every function
that include/moa.h declares, and rejects bad arguments on the host before
launching anything (no GPU is needed for any of these calls)."""
import ctypes
import os
import re

import pytest

from paper_2306_11148_b300 import build as moa_build
from paper_2306_11148_b300 import moa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    moa_build.build()
    return moa.lib()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"\b(moa_[a-z0-9_]+)\s*\(", text):
            names.add(mt.group(1))
    return names


def test_every_declared_symbol_is_exported(L):
    declared = _declared_functions()
    assert "moa_gemm" in declared and "moa_gemm_grouped" in declared
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_binding_covers_declared_symbols(L):
    assert _declared_functions() <= set(moa.EXPORTS)


def test_version(L):
    assert "sm_103a" in moa.moa_version()


@pytest.mark.parametrize("m,n,p", [(-1, 4, 4), (4, -1, 4), (4, 4, -1)])
def test_negative_dimensions_rejected(L, m, n, p):
    rc = moa.moa_gemm_ex(m, n, p, moa.MOA_F32_TF32, 16, 16, 16, 0, None, 0, None)
    assert rc == moa.MOA_ERR_ARG
    assert "negative" in moa.last_error()


def test_unknown_dtype_rejected(L):
    assert moa.moa_gemm_ex(4, 4, 4, 99, 16, 16, 16, 0, None, 0, None) == moa.MOA_ERR_DTYPE


def test_null_pointers_rejected(L):
    assert moa.moa_gemm_ex(4, 4, 4, moa.MOA_F64, None, 16, 16, 0, None, 0, None) == moa.MOA_ERR_ARG
    assert moa.moa_gemm_ex(4, 4, 4, moa.MOA_F64, 16, 16, None, 0, None, 0, None) == moa.MOA_ERR_ARG


def test_misaligned_pointers_rejected(L):
    assert moa.moa_gemm_ex(4, 4, 4, moa.MOA_F64, 8 + 4, 16, 16, 0, None, 0, None) == moa.MOA_ERR_ALIGN
    # tensor-core modes need 16-byte aligned operands
    assert moa.moa_gemm_ex(4, 4, 4, moa.MOA_F32_TF32, 16 + 4, 16, 16, 0, None, 0, None) == \
        moa.MOA_ERR_ALIGN


def test_missing_workspace_rejected(L):
    # n = 5 needs padded copies for TMA (20-byte rows)
    need = moa.moa_gemm_workspace_size(8, 5, 8, moa.MOA_F32_TF32, 0)
    assert need > 0
    rc = moa.moa_gemm_ex(8, 5, 8, moa.MOA_F32_TF32, 256, 512, 1024, 0, None, 0, None)
    assert rc == moa.MOA_ERR_WORKSPACE
    for dt in (moa.MOA_F32_SPLIT, moa.MOA_F64_SPLIT_F32IN, moa.MOA_F64_SPLIT_F64IN,
               moa.MOA_F64_SPLIT_F32IN_E4M3, moa.MOA_F64_SPLIT_F64IN_E4M3):
        assert moa.moa_gemm_workspace_size(64, 64, 64, dt, 0) > 0
        rc = moa.moa_gemm_ex(64, 64, 64, dt, 256, 512, 1024, 0, None, 0, None)
        assert rc == moa.MOA_ERR_WORKSPACE


def test_workspace_sizes(L):
    # aligned dense shapes need none; split modes hold S slice planes
    assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_BF16, 0) == 0
    # TF32 stages B transposed (K-major) in the workspace
    assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F32_TF32, 0) == 256 * 256 * 4
    assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64, 0) == 0
    s3 = moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F32_SPLIT, 0)
    assert s3 >= 3 * 2 * (256 * 256 * 2)
    s7 = moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F32IN, 0)
    s8 = moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F32IN, 8)
    assert s8 > s7 >= 7 * 2 * (256 * 256 * 2)
    # unsupported slice counts report 0 and are rejected by the call
    assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F32IN, 9) == 0
    assert moa.moa_gemm_ex(64, 64, 64, moa.MOA_F64_SPLIT_F32IN, 256, 512, 1024, 9, 4096, 1 << 20,
                           None) == moa.MOA_ERR_DTYPE
    # E4M3 digit planes: one byte per element, B stored transposed; 4..12 slices
    e10 = moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F32IN_E4M3, 0)
    assert e10 == moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F32IN_E4M3, 10)
    assert e10 >= 10 * 2 * (256 * 256)
    assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F64IN_E4M3, 12) > e10
    for bad in (3, 13):
        assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_SPLIT_F32IN_E4M3, bad) == 0
    # a 5-column B is padded to 16-byte rows of its transpose: p rows of round_up(n, 16)
    w = moa.moa_gemm_workspace_size(16, 5, 3, moa.MOA_F64_SPLIT_F32IN_E4M3, 4)
    assert w >= 4 * (16 * 16 + 3 * 16)
    assert moa.moa_gemm_ex(4, 4, 4, 11, 16, 16, 16, 0, None, 0, None) == moa.MOA_ERR_DTYPE
    # modular slices: M x (A and B residue planes) + the product's residue planes;
    # 8..16 moduli, default 14 up to n = 36639 and 15 beyond
    c14 = moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_CRT_F32IN, 0)
    assert c14 == moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_CRT_F32IN, 14)
    assert c14 >= 14 * 2 * (2 * 256 * 256) + 14 * 256 * 256
    assert moa.moa_gemm_workspace_size(16, 36640, 16, moa.MOA_F64_CRT_F32IN, 0) == \
        moa.moa_gemm_workspace_size(16, 36640, 16, moa.MOA_F64_CRT_F32IN, 15)
    for bad in (7, 17):
        assert moa.moa_gemm_workspace_size(256, 256, 256, moa.MOA_F64_CRT_F64IN, bad) == 0


def test_host_entry_workspace_and_argument_errors(L):
    """moa_gemm_host: the workspace holds device copies of A, B, C (each
    rounded to 256 bytes) plus the mode's own; bad arguments are refused on
    the host before any copy or launch."""
    for dt in (moa.MOA_BF16, moa.MOA_F32_TF32, moa.MOA_F32_SPLIT, moa.MOA_F64_CRT_F32IN,
               moa.MOA_F64_CRT_F64IN, moa.MOA_F64):
        m, n, p = 100, 70, 30
        ib = 2 if dt == moa.MOA_BF16 else (8 if dt in (moa.MOA_F64, moa.MOA_F64_CRT_F64IN) else 4)
        ob = 8 if dt in moa.F64_ACCURATE else 4
        al = lambda x: (x + 255) // 256 * 256  # noqa: E731
        want = al(m * n * ib) + al(n * p * ib) + al(m * p * ob) + \
            moa.moa_gemm_workspace_size(m, n, p, dt, 0)
        assert moa.moa_gemm_host_workspace_size(m, n, p, dt, 0) == want
    assert moa.moa_gemm_host_workspace_size(4, 4, 4, 11, 0) == 0
    assert moa.moa_gemm_host_workspace_size(-1, 4, 4, moa.MOA_BF16, 0) == 0
    a = (ctypes.c_float * 64)()
    c = (ctypes.c_double * 64)()
    pa, pc = ctypes.addressof(a), ctypes.addressof(c)
    need = moa.moa_gemm_host_workspace_size(8, 8, 8, moa.MOA_F64_CRT_F32IN, 0)
    f = moa.moa_gemm_host
    assert f(8, 8, 8, 11, pa, pa, pc, 0, 256, need, None) == moa.MOA_ERR_DTYPE
    assert f(-8, 8, 8, moa.MOA_F64_CRT_F32IN, pa, pa, pc, 0, 256, need, None) == moa.MOA_ERR_ARG
    assert f(8, 8, 8, moa.MOA_F64_CRT_F32IN, None, pa, pc, 0, 256, need, None) == moa.MOA_ERR_ARG
    assert f(8, 8, 8, moa.MOA_F64_CRT_F32IN, pa, pa, None, 0, 256, need, None) == moa.MOA_ERR_ARG
    assert f(8, 8, 8, moa.MOA_F64_CRT_F32IN, pa, pa, pc, 0, 256, need - 1,
             None) == moa.MOA_ERR_WORKSPACE
    assert f(8, 8, 8, moa.MOA_F64_CRT_F32IN, pa, pa, pc, 0, None, need,
             None) == moa.MOA_ERR_WORKSPACE
    assert f(8, 8, 8, moa.MOA_F64_CRT_F32IN, pa, pa, pc, 0, 128, need,
             None) == moa.MOA_ERR_ALIGN
    assert f(0, 8, 8, moa.MOA_F64_CRT_F32IN, None, None, None, 0, None, 0, None) == moa.MOA_OK


def test_grouped_path_host_query(L):
    """moa_grouped_path on the host: aligned BF16 problems take the persistent
    launch, modular-slice ones the grouped modular-slice launches, small
    FP32-accuracy split ones the grouped split launches, other modes (and
    unaligned operands) their own launches."""
    def path(m, n, p, dt, a=4096, b=8192, c=16384):
        d = moa.moa_gemm_desc()
        d.m, d.n, d.p, d.dt, d.A, d.B, d.C = m, n, p, dt, a, b, c
        return L.moa_grouped_path(ctypes.byref(d))
    assert path(128, 256, 192, moa.MOA_BF16) == moa.MOA_GROUPED_BF16
    assert path(128, 256, 192, moa.MOA_F64_CRT_F32IN) == moa.MOA_GROUPED_CRT
    assert path(128, 256, 192, moa.MOA_F32_SPLIT) == moa.MOA_GROUPED_F32_SPLIT
    assert path(128, 256, 192, moa.MOA_F64) == moa.MOA_GROUPED_ALONE
    assert path(128, 256, 192, moa.MOA_F64_SPLIT_F32IN) == moa.MOA_GROUPED_ALONE
    assert path(128, 256, 192, moa.MOA_F32_SPLIT, a=4100) == moa.MOA_GROUPED_ALONE
    assert path(0, 256, 192, moa.MOA_BF16) == moa.MOA_GROUPED_ALONE
    assert L.moa_grouped_path(None) == moa.MOA_ERR_ARG


def test_fp64_rate_argument_errors(L):
    out = ctypes.c_double(0.0)
    assert L.moa_measure_fp64_rate(2, None, ctypes.byref(out)) == moa.MOA_ERR_ARG
    assert L.moa_measure_fp64_rate(0, None, None) == moa.MOA_ERR_ARG


def test_empty_problems_are_noops(L):
    # m == 0 or p == 0: nothing to do, nothing launched (works without a GPU)
    assert moa.moa_gemm_ex(0, 5, 5, moa.MOA_F64, None, None, None, 0, None, 0, None) == moa.MOA_OK
    assert moa.moa_gemm_ex(5, 5, 0, moa.MOA_F64, None, None, None, 0, None, 0, None) == moa.MOA_OK


def test_grouped_argument_errors(L):
    assert L.moa_gemm_grouped(-1, None, None, 0, None) == moa.MOA_ERR_ARG
    assert L.moa_gemm_grouped(0, None, None, 0, None) == moa.MOA_OK
    assert L.moa_gemm_grouped(2, None, None, 0, None) == moa.MOA_ERR_ARG


def test_binding_refuses_mismatched_tensors(L):
    import torch
    A = torch.zeros((4, 8), dtype=torch.float32)
    B = torch.zeros((8, 3), dtype=torch.float32)
    with pytest.raises(TypeError):       # FP64-input mode reads 8 bytes per element
        moa.check_tensors(A, B, None, moa.MOA_F64_SPLIT_F64IN)
    with pytest.raises(TypeError):
        moa.check_tensors(A, B, None, moa.MOA_F64_SPLIT_F64IN_E4M3)
    with pytest.raises(TypeError):
        moa.check_tensors(A, B, torch.zeros((4, 3), dtype=torch.float32), moa.MOA_F64_SPLIT_F32IN)
    with pytest.raises(ValueError):      # CPU tensors are not device memory
        moa.check_tensors(A, B, None, moa.MOA_F32_TF32)
    with pytest.raises(ValueError):
        moa.check_tensors(A, B[:5], None, moa.MOA_F32_TF32)


def test_log_level_reports_host_errors(L):
    """MOA_LOG=1 prints every error message to stderr (argument errors are
    found on the host, so this needs no GPU); unset, nothing is printed."""
    import subprocess
    import sys
    code = ("import ctypes; from paper_2306_11148_b300 import moa; "
            "rc = moa.moa_gemm_ex(8, 8, 8, 77, 256, 512, 1024, 0, None, 0, None, None); "
            "print(rc)")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for level, expect in (("1", True), ("0", False)):
        env = dict(os.environ, MOA_LOG=level)
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                           text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        assert r.stdout.strip() == str(moa.MOA_ERR_DTYPE)
        assert ("[moa] error -2:" in r.stderr) == expect, r.stderr
