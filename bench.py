#!/usr/bin/env python
"""Benchmark of the B300-native MoA ONF GEMM (Eq. eq:dnf).

Default workload: the FP64-accurate ONF GEMM at m = n = p = 8192 on FP32
inputs drawn i.i.d. N(0, 1) (seed 0): the modular-slice mode
(MOA_F64_CRT_F32IN: rows of A and columns of B scaled to integers, their
residues modulo 14 small moduli as BF16 planes, one exact tensor-core GEMM
per modulus, the exact integer product recovered by the Chinese remainder
theorem and rounded once to FP64), one GEMM (all passes included) per step.  The line carries the oracle's error
on 64 sampled rows for the plain and the two row-scaled input kinds, the
roofline of the slice-product kernel, the CPU oracle's rate, the end-to-end
rate from pinned host memory, joules per GEMM, and the other precision modes
and a short serving run under "modes".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl moa|reference]
                  [--workload crt_f64|split_f64|square|split_f32|bf16|f64|...] [--n N]

Under torchrun (N > 1) every rank runs its own replica of the workload (the
GEMM is not sharded: replicas only); timing is the max over ranks and the
value is the total over ranks.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}
# Dense tensor rates relative to BF16 (nominal datasheet figures).
NOMINAL_RATIO = {"bf16": 1.0, "tf32": 1.1 / 2.25, "fp8": 2.0}
L2_MB = 126.0   # B300 L2 capacity
# DRAM traffic (read + write bytes) per launch of the dominant kernel from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (mode,
# N), with the SHA-256 (first 16 hex digits) of the kernel's source file at
# capture time: a figure whose source has changed since is reported as null.
TRAFFIC = {
    ("tf32", 8192): {"bytes": 1.652613e9 + 0.236939e9, "src": "gemm_tc.cu",
                     "sha": None},
    ("f64_crt_f32in", 8192): {"bytes": 14224164864 + 984522496, "src": "crt.cu",
                              "sha": "33b7df3c3e06828b"},
}


def src_sha(name):
    import hashlib
    path = os.path.join(ROOT, "paper_2306_11148_b300", "csrc", name)
    try:
        with open(path, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def traffic_of(mode, N):
    """(bytes per launch or None, note) for the dominant kernel of `mode`."""
    t = TRAFFIC.get((mode, N))
    if t is None:
        return None, "no ncu capture of this kernel at this size"
    if t["sha"] is None or src_sha(t["src"]) != t["sha"]:
        return None, f"kernel source {t['src']} changed since the ncu capture"
    return t["bytes"], f"ncu capture of {t['src']} (sha {t['sha']})"


def load_peaks():
    try:
        with open(MEASURED) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    except Exception:
        d = dict(FALLBACK)
        d["source"] = "fallback"
        return d


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="moa_clocks_", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_identity(dev):
    """(PCI bus id as NVML prints it, NVML-style UUID) of a torch device."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    pci = uuid = None
    try:
        pci = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except Exception:
        pass
    try:
        uuid = "GPU-" + str(props.uuid)
    except Exception:
        pass
    return pci, uuid


class _NvmlCtypes:
    """Minimal ctypes view of libnvidia-ml (used when the pynvml module is absent)."""

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.L = ctypes.CDLL("libnvidia-ml.so.1")
        if self.L.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")

    def by_pci(self, pci):
        h = self.c.c_void_p()
        rc = self.L.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), self.c.byref(h))
        if rc != 0:
            raise RuntimeError(f"nvmlDeviceGetHandleByPciBusId_v2 rc={rc}")
        return h

    def by_index(self, i):
        h = self.c.c_void_p()
        rc = self.L.nvmlDeviceGetHandleByIndex_v2(i, self.c.byref(h))
        if rc != 0:
            raise RuntimeError(f"nvmlDeviceGetHandleByIndex_v2 rc={rc}")
        return h

    def count(self):
        n = self.c.c_uint()
        self.L.nvmlDeviceGetCount_v2(self.c.byref(n))
        return n.value

    def energy_mj(self, h):
        v = self.c.c_ulonglong()
        rc = self.L.nvmlDeviceGetTotalEnergyConsumption(h, self.c.byref(v))
        if rc != 0:
            raise RuntimeError(f"nvmlDeviceGetTotalEnergyConsumption rc={rc}")
        return v.value


class Energy:
    """NVML total-energy counter (mJ) of the device, found by PCI bus id, then
    by UUID, then as the only visible device (pynvml, else libnvidia-ml via
    ctypes)."""

    def __init__(self, pci, uuid=None):
        self.h = None
        self.why = None
        self.read = None
        errs = []
        try:
            import pynvml
            pynvml.nvmlInit()
            tries = []
            if pci:
                tries += [lambda: pynvml.nvmlDeviceGetHandleByPciBusId(pci)]
            if uuid:
                tries += [lambda: pynvml.nvmlDeviceGetHandleByUUID(uuid)]
            tries += [lambda: pynvml.nvmlDeviceGetHandleByIndex(0)
                      if pynvml.nvmlDeviceGetCount() == 1 else None]
            for t in tries:
                try:
                    h = t()
                    if h is not None:
                        pynvml.nvmlDeviceGetTotalEnergyConsumption(h)
                        self.h = h
                        self.read = lambda: pynvml.nvmlDeviceGetTotalEnergyConsumption(self.h)
                        return
                except Exception as e:
                    errs.append(str(e))
        except Exception as e:
            errs.append(f"pynvml: {e}")
        try:
            nv = _NvmlCtypes()
            tries = ([lambda: nv.by_pci(pci)] if pci else []) + \
                [lambda: nv.by_index(0) if nv.count() == 1 else None]
            for t in tries:
                try:
                    h = t()
                    if h is not None:
                        nv.energy_mj(h)
                        self.h = h
                        self.read = lambda: nv.energy_mj(self.h)
                        return
                except Exception as e:
                    errs.append(str(e))
        except Exception as e:
            errs.append(f"libnvidia-ml: {e}")
        self.why = "; ".join(errs) or "no handle"

    def read_j(self):
        if self.h is None:
            return None
        try:
            return self.read() / 1000.0
        except Exception:
            return None

    def temp_c(self):
        """GPU temperature (C) through NVML, or None."""
        if self.h is None:
            return None
        try:
            import pynvml
            return float(pynvml.nvmlDeviceGetTemperature(self.h, pynvml.NVML_TEMPERATURE_GPU))
        except Exception:
            pass
        try:
            import ctypes
            L = ctypes.CDLL("libnvidia-ml.so.1")
            t = ctypes.c_uint()
            if L.nvmlDeviceGetTemperature(self.h, 0, ctypes.byref(t)) == 0:
                return float(t.value)
        except Exception:
            pass
        return None


# ------------------------------------------------------------------ distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """Max of a per-rank time over all ranks (the only collective of the
    benchmark; the GEMM itself is not sharded)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(flops_per_step, steps, seconds, ws):
    """Whole-job value for N replicas: total flops of all ranks over the
    slowest rank's time (TFLOP/s)."""
    t_max = max_over_ranks(seconds, ws)
    return flops_per_step * steps * ws / t_max / 1e12, t_max


# ------------------------------------------------------------------ workloads
MODE_OF = {"split_f64": "f64_split_f32in", "square": "tf32", "bf16": "bf16",
           "split_f32": "f32_split",
           "split_f64_e4m3": "f64_split_f32in_e4m3", "crt_f64": "f64_crt_f32in",
           "crt_f64in": "f64_crt_f64in",
           "f64": "f64", "simt": "f32_simt",
           "grouped": "grouped", "serve": "serve", "energy_n": "energy_n",
           "tiles": "tiles", "peaks": "peaks", "products": "products", "crt_tiles": "crt_tiles"}


SPLIT_F32IN = ("f32_split", "f64_split_f32in", "f64_split_f32in_e4m3", "f64_crt_f32in")


def make_inputs(mode, N, scaled=None):
    """Seed-0 operands of the square workload: FP32 N(0, 1) for the split
    modes (optionally row-scaled, `scaled` = "rows" | "rowcol"), uniform[-1, 1)
    in the mode's input type otherwise."""
    import torch
    from paper_2306_11148_b300 import inputs, moa
    dt = moa.MODES[mode]
    if mode in SPLIT_F32IN:
        A, B = inputs.normal_pair(N, N, N, dtype=torch.float32, seed=0, scaled=scaled)
    else:
        A, B = inputs.square_uniform(N, moa.in_dtype(dt), seed=0)
    return dt, A, B


def time_device(fn, steps, warmup, stream, ws, warm_fn=None):
    import torch
    for _ in range(warmup):
        (warm_fn or fn)()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    return ev0.elapsed_time(ev1) / 1000.0


def bench_mode(mode, N, steps, warmup, ws, stream, want_energy=False, energy=None,
               want_e2e=False, check_rows=True, keep_rows=None):
    """Times `steps` GEMMs of the square workload of `mode`.  keep_rows: row
    indices of C returned (on the host) as out["rows_C"]."""
    import torch
    from paper_2306_11148_b300 import moa
    dt, A, B = make_inputs(mode, N)
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.empty((N, N), dtype=moa.out_dtype(dt), device="cuda")
    wspace = moa.Workspace(torch.device("cuda"))
    need = moa.moa_gemm_workspace_size(N, N, N, dt, 0)
    wptr, wbytes = wspace.get(need)
    sh = int(stream.cuda_stream)
    st = moa.moa_stats()

    def step():
        rc = moa.moa_gemm_ex(N, N, N, dt, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), 0, wptr,
                             wbytes, sh, st)
        if rc != 0:
            raise moa.MoaError(rc, moa.last_error())

    # Per-step CUDA events around the main GEMM kernel only (recorded by the
    # library on this stream immediately before and after that launch).
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)
    idx = [0]

    def step_timed():
        a, b = kev[idx[0]]
        moa.lib().moa_profile_events(a.cuda_event, b.cuda_event)
        step()
        idx[0] += 1

    with torch.cuda.stream(stream):
        t = time_device(step_timed, steps, warmup, stream, ws, warm_fn=step)
    moa.lib().moa_profile_events(None, None)
    kernel_s = sum(a.elapsed_time(b) for a, b in kev) / 1000.0
    moa.check(moa.moa_sync_status(sh))
    out = {"mode": mode, "N": N, "seconds": t, "kernel_seconds": kernel_s, "steps": steps,
           "flops_per_step": 2.0 * N ** 3, "kernels_per_step": int(st.kernels),
           "tile": [int(st.block_m), int(st.block_n), int(st.block_k)],
           "products": int(st.products), "slices": int(st.slices)}
    if want_energy and energy is not None and energy.h is not None:
        per = t / steps
        reps = max(3, int(math.ceil(1.5 / max(per, 1e-6))))
        torch.cuda.synchronize()
        j0 = energy.read_j()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(reps):
                step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        j1 = energy.read_j()
        if j0 is not None and j1 is not None:
            out["energy"] = {"j_per_gemm": (j1 - j0) / reps, "window_s": t1 - t0, "reps": reps,
                             "avg_w": (j1 - j0) / (t1 - t0)}
    if want_e2e:
        out["e2e"] = bench_e2e(dt, A, B, C, N, max(6, steps), 3, stream, ws)
    if keep_rows is not None:
        out["rows_C"] = C.index_select(
            0, torch.as_tensor(keep_rows, dtype=torch.int64, device=C.device)).cpu()
    # spot check of a few rows of the timed output (parity proper is in tests/)
    try:
        if not check_rows:
            raise RuntimeError("skipped")
        out["rel_err_sampled_rows"] = sampled_rows_err(Ad, Bd, C, [0, N // 3, N - 1])
    except Exception as e:  # pragma: no cover - informational only
        out["rel_err_sampled_rows"] = f"unavailable: {e}"
    del Ad, Bd, C
    return out


def bench_e2e(dt, A, B, C, N, steps, warmup, stream, ws, lanes_n=3):
    """The same GEMM through the library's host-buffer entry (moa_gemm_host):
    every step the library copies that step's A and B from pinned host memory
    to the device, runs the GEMM and copies C back to pinned host memory, all
    inside the timed region.  Independent steps rotate over `lanes_n` streams,
    each with its own workspace and host C, so one step's copies overlap
    another's GEMM (the copy engines and the SMs work at once); with three
    lanes a lane's in-order upload, GEMM and download span three steps."""
    import torch
    from paper_2306_11148_b300 import moa
    Ah = A.pin_memory()
    Bh = B.pin_memory()
    need = moa.moa_gemm_host_workspace_size(N, N, N, dt, 0)
    lanes = []
    for _ in range(lanes_n):
        st = torch.cuda.Stream()
        Ch = torch.empty(C.shape, dtype=C.dtype, pin_memory=True)
        wsp = moa.Workspace(torch.device("cuda"))
        w, wb = wsp.get(need)
        lanes.append((st, Ch, wsp, w, wb))
    idx = [0]

    def step():
        st, Ch, _, w, wb = lanes[idx[0] % lanes_n]
        idx[0] += 1
        moa.check(moa.moa_gemm_host(N, N, N, dt, Ah.data_ptr(), Bh.data_ptr(), Ch.data_ptr(), 0,
                                    w, wb, int(st.cuda_stream), None))

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record(lanes[0][0])
    for ln in lanes[1:]:
        ln[0].wait_event(ev0)
    for _ in range(steps):
        step()
    ends = []
    for ln in lanes:
        e = torch.cuda.Event(enable_timing=True)
        e.record(ln[0])
        ends.append(e)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t0
    t = max(ev0.elapsed_time(e) for e in ends) / 1000.0
    for ln in lanes:
        moa.check(moa.moa_sync_status(int(ln[0].cuda_stream)))
    barrier(ws)
    h2d = A.numel() * A.element_size() + B.numel() * B.element_size()
    d2h = C.numel() * C.element_size()
    return {"seconds": t, "wall_seconds": t_wall, "steps": steps, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "streams": lanes_n, "api": "moa_gemm_host"}


def gpu_rows(mode, N, scaled, rows, stream):
    """Rows `rows` of C for the square workload of `mode` on the input kind
    `scaled` (None, "rows", "rowcol"), one untimed GEMM through moa_gemm_ex."""
    import torch
    from paper_2306_11148_b300 import moa
    dt, A, B = make_inputs(mode, N, scaled=scaled)
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.empty((N, N), dtype=moa.out_dtype(dt), device="cuda")
    with torch.cuda.stream(stream):
        moa.gemm(Ad, Bd, dt, C=C, stream=stream)
    moa.check(moa.moa_sync_status(int(stream.cuda_stream)))
    out = C.index_select(0, torch.as_tensor(rows, dtype=torch.int64, device="cuda")).cpu()
    del Ad, Bd, C
    return out


def cpu_baseline_split(mode, N, rows_c, rows, seconds_target=8.0):
    """CPU leg of the split-mode workloads: the oracle (FP64 i-k-j loop,
    OpenMP over rows, all host cores), as it stands, timed on a bounded
    sample of rows of the same N(0, 1) problem, then run on the sampled rows
    `rows` of each input kind, whose GPU results `rows_c[kind]` it checks
    (relative Frobenius error over those rows)."""
    import numpy as np
    import torch

    import oracle
    cores = os.cpu_count() or 1
    errs = {}
    t_all = 0.0
    flops_all = 0.0
    used = 0
    for kind, got in rows_c.items():
        _, A, B = make_inputs(mode, N, scaled=None if kind == "plain" else kind)
        A = A.double().numpy()
        B = B.double().numpy()
        t0 = time.perf_counter()
        ref, used = oracle.gemm_omp(A[rows], B, threads=0)
        dt = time.perf_counter() - t0
        t_all += dt
        flops_all += 2.0 * len(rows) * N * N
        g = got.double().numpy()
        errs[kind] = float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300))
        if kind == "plain":
            # a longer bounded sample of the same loop for the rate (rows
            # grown 4x until the sample takes a quarter of the target)
            extra = len(rows)
            from paper_2306_11148_b300 import inputs
            while t_all < seconds_target / 4 and extra < N:
                extra = min(N, extra * 4)
                idx = inputs.sample_rows(N, extra, seed=1)
                t0 = time.perf_counter()
                oracle.gemm_omp(A[idx], B, threads=0)
                t_all += time.perf_counter() - t0
                flops_all += 2.0 * extra * N * N
            # the same loop on one thread, 8 rows
            idx1 = inputs.sample_rows(N, 8, seed=1)
            t1 = time.perf_counter()
            oracle.gemm_omp(A[idx1], B, threads=1)
            dt1 = time.perf_counter() - t1
            single = {"value": 2.0 * 8 * N * N / dt1 / 1e12, "unit": "TFLOP/s",
                      "sample": f"8 rows on 1 thread, {dt1:.2f} s"}
        del A, B
    return {"value": flops_all / t_all / 1e12, "unit": "TFLOP/s", "cores": int(used),
            "kind": "oracle",
            "sample": f"sampled rows of the N={N} problem on {len(rows_c)} input kinds "
                      f"({', '.join(rows_c)}), FP64 i-k-j loop, OpenMP over rows, "
                      f"{flops_all / (2.0 * N * N):.0f} rows in {t_all:.2f} s",
            "host_cores": cores, "seconds": t_all, "single_thread": single,
            "rel_err_vs_oracle": errs, "rows_checked": len(rows)}


def cpu_operands(N, dtype_name, mode=None):
    """The square workload's operands as FP64 numpy arrays (exact
    conversion): a split mode's N(0, 1) FP32 operands, else uniform[-1, 1)."""
    import torch
    from paper_2306_11148_b300 import inputs
    tdt = torch.float32 if dtype_name != "f64" else torch.float64
    if mode in SPLIT_F32IN:
        _, A, B = make_inputs(mode, N)
    else:
        A, B = inputs.square_uniform(N, tdt, seed=0)
    return A.double().numpy(), B.double().numpy()


def cpu_baseline(N, dtype_name, seconds_target=8.0, mode=None, operands=None):
    """The oracle, as it stands, on sampled rows of the same N^3 problem, all
    host cores (OpenMP over rows); TFLOP/s of algorithmic work.  `operands`:
    (A, B) from cpu_operands, else drawn here."""
    import oracle
    from paper_2306_11148_b300 import inputs
    A, B = operands if operands is not None else cpu_operands(N, dtype_name, mode)
    rows = 8
    cores = os.cpu_count() or 1
    while True:
        idx = inputs.sample_rows(N, rows, seed=1)
        t0 = time.perf_counter()
        _, used = oracle.gemm_omp(A[idx], B, threads=0)
        dt = time.perf_counter() - t0
        if dt > seconds_target / 4 or rows >= N:
            break
        rows = min(N, rows * 4)
    flops = 2.0 * rows * N * N
    # the same loop on one thread, on a quarter of the rows (bounded)
    rows1 = max(1, rows // 4)
    idx1 = inputs.sample_rows(N, rows1, seed=1)
    t1 = time.perf_counter()
    oracle.gemm_omp(A[idx1], B, threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": int(used), "kind": "oracle",
            "sample": f"{rows} of {N} rows of the N={N} ONF GEMM in FP64 (i-k-j loop, OpenMP "
                      f"over rows), {dt:.2f} s", "host_cores": cores, "seconds": dt,
            "single_thread": {"value": 2.0 * rows1 * N * N / dt1 / 1e12, "unit": "TFLOP/s",
                              "sample": f"{rows1} rows on 1 thread, {dt1:.2f} s"}}


def bench_grouped(steps, warmup, ws, stream, count=512, compare=True):
    """Grouped batch: `count` BF16 GEMMs (m, n, p log-uniform in [32, 2048],
    multiples of 16, FP32 out) in one moa_gemm_grouped launch per step, and the
    same problems as `count` separate moa_gemm_ex launches."""
    import torch
    from paper_2306_11148_b300 import inputs, moa
    shapes = inputs.grouped_shapes(count, seed=0)
    probs = []
    flops = 0.0
    nbytes = 0
    for i, (m, n, p) in enumerate(shapes):
        A, B = inputs.uniform_pair(m, n, p, dtype=torch.bfloat16, seed=1000 + i)
        C = torch.empty((m, p), dtype=torch.float32, device="cuda")
        probs.append((A.cuda(), B.cuda(), C, moa.MOA_BF16))
        flops += 2.0 * m * n * p
        nbytes += 2 * (m * n + n * p) + 4 * m * p
    descs = moa.make_descs(probs)
    wspace = moa.Workspace(torch.device("cuda"))
    L = moa.lib()
    need = int(L.moa_gemm_grouped_workspace_size(len(probs), descs))
    wptr, wbytes = wspace.get(need)
    sh = int(stream.cuda_stream)

    def step():
        moa.check(L.moa_gemm_grouped(len(probs), descs, wptr, wbytes, sh))

    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)
    idx = [0]

    def step_timed():
        a, b = kev[idx[0]]
        L.moa_profile_events(a.cuda_event, b.cuda_event)
        step()
        idx[0] += 1

    with torch.cuda.stream(stream):
        t = time_device(step_timed, steps, warmup, stream, ws, warm_fn=step)
    L.moa_profile_events(None, None)
    kernel_s = sum(a.elapsed_time(b) for a, b in kev) / 1000.0
    moa.check(moa.moa_sync_status(sh))

    sws = moa.Workspace(torch.device("cuda"))

    def separate():
        for A, B, C, dt in probs:
            m, n = A.shape
            p = B.shape[1]
            w, wb = sws.get(moa.moa_gemm_workspace_size(m, n, p, dt, 0))
            moa.check(moa.moa_gemm_ex(m, n, p, dt, A.data_ptr(), B.data_ptr(), C.data_ptr(), 0,
                                      w, wb, sh, None))

    nsep = max(2, steps // 2)
    t_sep = float("nan")
    t_graph = float("nan")
    if compare:
        with torch.cuda.stream(stream):
            t_sep = time_device(separate, nsep, 2, stream, ws)
        # the same 512 launches captured once in a CUDA graph and replayed:
        # separate kernels without the host launch cost
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            separate()
        with torch.cuda.stream(stream):
            t_graph = time_device(graph.replay, nsep, 2, stream, ws)
        del graph
    e2e = bench_grouped_e2e(shapes, max(4, min(steps, 8)), 2, ws) if compare else {}
    return {"seconds": t, "kernel_seconds": kernel_s, "steps": steps, "flops_per_step": flops,
            "bytes_per_step": nbytes, "count": count, "e2e": e2e,
            "separate_seconds_per_step": t_sep / nsep,
            "graph_seconds_per_step": t_graph / nsep, "kernels_per_step": 1,
            "products": 1, "tile": [128, 0, 64]}


def bench_products(stream, steps=10, warmup=3):
    """The no-reduction members of the outer-product family through the one
    kernel (moa_product), FP32: the Kronecker product of 64 x 64 and 128 x 128
    operands (an 8192 x 8192 output) and the Hadamard product of two
    8192 x 8192 arrays.  HBM-bound: bytes = output written + operands read once;
    GB/s against the measured copy bandwidth."""
    import torch
    from paper_2306_11148_b300 import inputs, moa
    out = {}
    cases = [("kronecker", moa.MOA_PRODUCT_KRONECKER, (64, 64), (128, 128)),
             ("hadamard", moa.MOA_PRODUCT_HADAMARD, (8192, 8192), (8192, 8192))]
    for name, kind, sa, sb in cases:
        A, _ = inputs.uniform_pair(sa[0], sa[1], 1, dtype=torch.float32, seed=1)
        B, _ = inputs.uniform_pair(sb[0], sb[1], 1, dtype=torch.float32, seed=2)
        Ad, Bd = A.cuda(), B.cuda()
        C = moa.product(kind, Ad, Bd, moa.MOA_F32_SIMT, stream=stream)
        L = moa.lib()
        m, n = sa
        p, q = sb
        sh = int(stream.cuda_stream)

        def step():
            moa.check(L.moa_product(kind, m, n, p, q, moa.MOA_F32_SIMT, Ad.data_ptr(),
                                    Bd.data_ptr(), C.data_ptr(), sh))

        with torch.cuda.stream(stream):
            t = time_device(step, steps, warmup, stream, 1)
        moa.check(moa.moa_sync_status(sh))
        nbytes = 4 * (C.numel() + Ad.numel() + Bd.numel())
        out[name] = {"A": list(sa), "B": list(sb), "C": list(C.shape), "ms": t / steps * 1e3,
                     "bytes_per_launch": nbytes, "gbs": nbytes * steps / t / 1e9,
                     "kernel": "ipophp_kernel<float, float>"}
        del Ad, Bd, C
    return out


def bench_grouped_split(stream, count=64, div=1, steps=5, warmup=3, seed=3, mode="f64_crt_f32in"):
    """`count` split-precision GEMMs (FP32 N(0,1) inputs; `mode`: FP64-accuracy
    modular slices or FP32-accuracy split) with the serving stream's shapes
    (m, p log-uniform in [64, 4096], n in [64, 8192], each divided by `div`):
    one moa_gemm_grouped call per step against the same problems as `count`
    separate moa_gemm_ex calls (CUDA events)."""
    import torch
    from paper_2306_11148_b300 import inputs, moa
    dt = moa.MODES[mode]
    arr = inputs.serve_arrivals(rate=count * 4.0, seconds=1.0, seed=seed)[:count]
    probs = []
    flops = 0.0
    for i, (_, m, n, p, _) in enumerate(arr):
        m, n, p = max(1, m // div), max(1, n // div), max(1, p // div)
        A, B = inputs.normal_pair(m, n, p, dtype=torch.float32, seed=500 + i)
        probs.append((A.cuda(), B.cuda(), torch.empty((m, p), dtype=moa.out_dtype(dt),
                                                      device="cuda"), dt))
        flops += 2.0 * m * n * p
    paths = [moa.grouped_path(*pr) for pr in probs]
    descs = moa.make_descs(probs)
    wsp = moa.Workspace(torch.device("cuda"))
    L = moa.lib()
    w, wb = wsp.get(int(L.moa_gemm_grouped_workspace_size(len(probs), descs)))
    sh = int(stream.cuda_stream)

    def grouped():
        moa.check(L.moa_gemm_grouped(len(probs), descs, w, wb, sh))

    sws = moa.Workspace(torch.device("cuda"))
    sw, swb = sws.get(max(moa.moa_gemm_workspace_size(A.shape[0], A.shape[1], B.shape[1], dt, 0)
                          for A, B, _, dt in probs))

    def separate():
        for A, B, C, dt in probs:
            moa.check(moa.moa_gemm_ex(A.shape[0], A.shape[1], B.shape[1], dt, A.data_ptr(),
                                      B.data_ptr(), C.data_ptr(), 0, sw, swb, sh, None))

    with torch.cuda.stream(stream):
        t_g = time_device(grouped, steps, warmup, stream, 1)
        t_s = time_device(separate, steps, warmup, stream, 1)
    moa.check(moa.moa_sync_status(sh))
    what = {"f64_crt_f32in": "FP64-accuracy modular-slice",
            "f32_split": "FP32-accuracy split"}.get(mode, mode)
    return {"count": count, "shape_divisor": div, "flops_per_step": flops,
            "grouped_ms": t_g / steps * 1e3, "separate_ms": t_s / steps * 1e3,
            "grouped_tflops": flops * steps / t_g / 1e12,
            "separate_tflops": flops * steps / t_s / 1e12,
            "speedup": t_s / t_g,
            "on_grouped_path": sum(1 for x in paths if x != moa.MOA_GROUPED_ALONE),
            "workload": f"{count} {what} GEMMs, serving shapes / {div}"}


def bench_grouped_e2e(shapes, steps, warmup, ws):
    """The grouped batch end to end through moa_gemm_grouped with host
    buffers: every step copies all A and B operands from pinned host memory
    (one contiguous buffer per operand kind, each problem 256-byte aligned in
    it) to the device, runs the one grouped launch and copies every C back to
    pinned host memory, inside the timed region.  Independent steps alternate
    between two streams with their own device buffers, so one step's
    host-to-device copies overlap the previous step's launch and
    device-to-host copy (separate copy engines)."""
    import torch
    from paper_2306_11148_b300 import inputs, moa

    def al(x):
        return (x + 127) // 128 * 128   # elements: 256 B of BF16, 512 B of FP32

    offs, na, nb, nc = [], 0, 0, 0
    for m, n, p in shapes:
        offs.append((na, nb, nc))
        na += al(m * n)
        nb += al(n * p)
        nc += al(m * p)
    Ah = torch.zeros(na, dtype=torch.bfloat16, pin_memory=True)
    Bh = torch.zeros(nb, dtype=torch.bfloat16, pin_memory=True)
    for i, ((m, n, p), (oa, ob, _)) in enumerate(zip(shapes, offs)):
        A, B = inputs.uniform_pair(m, n, p, dtype=torch.bfloat16, seed=1000 + i)
        Ah[oa:oa + m * n] = A.reshape(-1)
        Bh[ob:ob + n * p] = B.reshape(-1)
    L = moa.lib()
    lanes = []
    for _ in range(2):
        st = torch.cuda.Stream()
        Ad = torch.empty(na, dtype=torch.bfloat16, device="cuda")
        Bd = torch.empty(nb, dtype=torch.bfloat16, device="cuda")
        Cd = torch.empty(nc, dtype=torch.float32, device="cuda")
        Ch = torch.empty(nc, dtype=torch.float32, pin_memory=True)
        probs = [(Ad[oa:oa + m * n].view(m, n), Bd[ob:ob + n * p].view(n, p),
                  Cd[oc:oc + m * p].view(m, p), moa.MOA_BF16)
                 for (m, n, p), (oa, ob, oc) in zip(shapes, offs)]
        descs = moa.make_descs(probs)
        wsp = moa.Workspace(torch.device("cuda"))
        w, wb = wsp.get(int(L.moa_gemm_grouped_workspace_size(len(probs), descs)))
        lanes.append((st, Ad, Bd, Cd, Ch, descs, len(probs), wsp, w, wb))
    idx = [0]

    def step():
        st, Ad, Bd, Cd, Ch, descs, count, _, w, wb = lanes[idx[0] % 2]
        idx[0] += 1
        with torch.cuda.stream(st):
            Ad.copy_(Ah, non_blocking=True)
            Bd.copy_(Bh, non_blocking=True)
            moa.check(L.moa_gemm_grouped(count, descs, w, wb, int(st.cuda_stream)))
            Ch.copy_(Cd, non_blocking=True)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record(lanes[0][0])
    lanes[1][0].wait_event(ev0)
    for _ in range(steps):
        step()
    ev1 = torch.cuda.Event(enable_timing=True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev1.record(lanes[0][0])
    ev2.record(lanes[1][0])
    torch.cuda.synchronize()
    t = max(ev0.elapsed_time(ev1), ev0.elapsed_time(ev2)) / 1000.0
    barrier(ws)
    for ln in lanes:
        moa.check(moa.moa_sync_status(int(ln[0].cuda_stream)))
    return {"seconds": t, "steps": steps, "h2d_bytes_per_step": 2 * (na + nb),
            "d2h_bytes_per_step": 4 * nc, "streams": 2}


class ServeOperands:
    """Device-resident operands of the serving stream, sized for its largest
    request.  `nbuf` pairs of FP32 N(0, 1) buffers (A: 4096 x 8192, B:
    8192 x 4096 elements) and `nout` output slots of 4096 x 4096 FP64.
    Arrival i reads its row-major m x n A and n x p B from pair i % nbuf at an
    offset that moves with i (256-byte aligned, so that successive requests
    touch different memory rather than one L2-resident prefix), and writes its
    m x p C to slot i % nout.  Every arrival thus runs its own shape."""

    MAX_MP, MAX_N = 4096, 8192

    def __init__(self, nbuf=2, nout=256, seed=0):
        import torch
        from paper_2306_11148_b300 import inputs
        self.nbuf, self.nout = nbuf, nout
        self.A, self.B = [], []
        for b in range(nbuf):
            A, B = inputs.normal_pair(self.MAX_MP, self.MAX_N, self.MAX_MP,
                                      dtype=torch.float32, seed=seed + 100 + b)
            self.A.append(A.reshape(-1).cuda())
            self.B.append(B.reshape(-1).cuda())
        self.C = torch.empty((nout, self.MAX_MP * self.MAX_MP), dtype=torch.float64,
                             device="cuda")

    def request(self, i, m, n, p, dt):
        """(A, B, C) views of arrival i with shape (m, n, p) for mode dt."""
        import torch
        from paper_2306_11148_b300 import moa
        size = self.MAX_MP * self.MAX_N
        b = i % self.nbuf
        span_a = max(1, (size - m * n) // 64 + 1)
        span_b = max(1, (size - n * p) // 64 + 1)
        oa = ((i * 7919) % span_a) * 64
        ob = ((i * 104729) % span_b) * 64
        A = self.A[b][oa:oa + m * n].view(m, n)
        B = self.B[b][ob:ob + n * p].view(n, p)
        slot = self.C[i % self.nout]
        C = slot[:m * p].view(m, p) if moa.out_dtype(dt) == torch.float64 else \
            slot.view(torch.float32)[:m * p].view(m, p)
        return A, B, C


def serve_dtype(tag, f64_mode="crt"):
    """Mode of a served request: FP32 accuracy -> the three-slice split;
    FP64 accuracy -> the modular slices ("crt") or the integer digits."""
    from paper_2306_11148_b300 import moa
    if tag == "f32":
        return moa.MOA_F32_SPLIT
    return moa.MOA_F64_CRT_F32IN if f64_mode == "crt" else moa.MOA_F64_SPLIT_F32IN


def serve_run(srv, ops, arrivals, f64_mode="crt"):
    """Submits every arrival (t, m, n, p, tag) at its time; returns the submit
    results [(status, ticket, i, flops)], the completions and the wall time."""
    from paper_2306_11148_b300 import moa
    t0 = time.perf_counter()
    codes = []
    for i, (t, m, n, p, tag) in enumerate(arrivals):
        delay = t - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        dt = serve_dtype(tag, f64_mode)
        A, B, C = ops.request(i, m, n, p, dt)
        rc, tk = srv.submit(A, B, C, dt)
        codes.append((rc, tk, i, 2.0 * m * n * p))
    submitted = [c for c in codes if c[0] == moa.MOA_OK]
    got = {}
    deadline = time.perf_counter() + 120
    while len(got) < len(submitted) and time.perf_counter() < deadline:
        for c in srv.poll():
            got[c[0]] = c
        time.sleep(0.001)
    wall = time.perf_counter() - t0
    return codes, got, wall


def bench_serve(ops, rate, seconds, seed=0, energy=None, n_streams=8, f64_mode="crt"):
    """Serving stream: Poisson arrivals at `rate` for `seconds`, each with its
    own (m, n, p) and precision tag from inputs.serve_arrivals, through one
    server (64 GB arena, 32 in flight, 8 streams, 2 s queue deadline).
    f64_mode: the mode of the FP64-accuracy requests ("crt": modular slices,
    "digits": integer digits)."""
    import torch
    from paper_2306_11148_b300 import inputs, moa
    arrivals = inputs.serve_arrivals(rate=rate, seconds=seconds, seed=seed)
    # a queued or running request owns its output slot until it completes
    srv = moa.Server(arena_bytes=64 << 30, max_inflight=32, n_streams=n_streams,
                     queue_capacity=ops.nout - 64, queue_deadline_s=2.0)
    j0 = energy.read_j() if energy else None
    try:
        codes, got, wall = serve_run(srv, ops, arrivals, f64_mode)
        st = srv.stats()
    finally:
        srv.close()
    j1 = energy.read_j() if energy else None
    done_ok = [c for c in got.values() if c[1] == moa.MOA_OK]
    ok_ticket = {c[0] for c in done_ok}
    flops = sum(f for rc, tk, i, f in codes if rc == moa.MOA_OK and tk in ok_ticket)
    span = (max(c[4] for c in done_ok) - min(c[2] for c in done_ok)) if done_ok else float("nan")

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(q * len(xs)))] * 1e3 if xs else float("nan")
    # latency split: queue wait (submit -> admission) and service (admission -> done)
    waits = [c[3] - c[2] for c in done_ok]
    service = [c[4] - c[3] for c in done_ok]
    # alone vs mix: arrivals whose output slot no later arrival reused, every
    # 8th of them, recomputed alone and compared bit for bit
    torch.cuda.synchronize()
    mism = checked = 0
    last = len(arrivals)
    for rc, tk, i, _ in codes[max(0, last - ops.nout):]:
        if i % 8 or rc != moa.MOA_OK or tk not in ok_ticket:
            continue
        _, m, n, p, tag = arrivals[i]
        dt = serve_dtype(tag, f64_mode)
        A, B, C = ops.request(i, m, n, p, dt)
        alone = moa.gemm(A, B, dt)
        torch.cuda.synchronize()
        checked += 1
        mism += 0 if torch.equal(alone, C) else 1
    n_f64 = sum(1 for a in arrivals if a[4] == "f64")
    return {"rate": rate, "seconds": seconds, "offered": len(arrivals),
            "offered_f64_accuracy": n_f64, "offered_f32_accuracy": len(arrivals) - n_f64,
            "submitted": st["submitted"], "completed": st["completed"],
            "rejected": st["rejected"], "busy": sum(1 for c in codes if c[0] == moa.MOA_ERR_BUSY),
            "failed": st["failed"], "served_per_s": len(done_ok) / span if done_ok else 0.0,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "mean_ms": st["mean_ms"], "batches": st["batches"],
            "queue_wait_p50_ms": pct(waits, 0.5), "queue_wait_p99_ms": pct(waits, 0.99),
            "service_p50_ms": pct(service, 0.5), "service_p99_ms": pct(service, 0.99),
            "inflight_peak": st["inflight_peak"], "arena_peak_gb": st["arena_peak"] / 1e9,
            "tflops_served": flops / span / 1e12 if done_ok else 0.0, "wall_s": wall,
            "j_per_request": (j1 - j0) / len(done_ok) if (j0 is not None and j1 is not None
                                                           and done_ok) else None,
            "avg_w": (j1 - j0) / wall if (j0 is not None and j1 is not None) else None,
            "alone_vs_mix_checked": checked, "alone_vs_mix_mismatch": mism,
            "f64_accuracy_mode": f64_mode}


def sampled_rows_err(Ad, Bd, C, rows):
    """Relative Frobenius error of rows `rows` of C against an FP64 torch
    matmul of the same device operands (an informational check printed with
    the timing; parity against the oracle is the job of tests/)."""
    import torch
    idx = torch.tensor(rows, dtype=torch.int64, device=C.device)
    ref = Ad.index_select(0, idx).double() @ Bd.double()
    got = C.index_select(0, idx).double()
    return float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))


def measure_window(step, energy, stream, t_est, min_window=1.5):
    """Back-to-back GEMMs for >= min_window seconds: (seconds per GEMM by CUDA
    events, joules per GEMM and average watts by the NVML energy counter,
    temperature at the end)."""
    import torch
    reps = max(2, int(math.ceil(min_window / max(t_est, 1e-6))))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    j0 = energy.read_j() if energy else None
    w0 = time.perf_counter()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(reps):
            step()
        ev1.record(stream)
    torch.cuda.synchronize()
    w1 = time.perf_counter()
    j1 = energy.read_j() if energy else None
    t = ev0.elapsed_time(ev1) / 1000.0 / reps
    out = {"s_per_gemm": t, "reps": reps, "window_s": w1 - w0}
    if j0 is not None and j1 is not None:
        out["j_per_gemm"] = (j1 - j0) / reps
        out["avg_w"] = (j1 - j0) / (w1 - w0)
    out["temp_c"] = energy.temp_c() if energy else None
    return out


def _prep(mode, N, seed=0):
    import torch
    from paper_2306_11148_b300 import inputs, moa
    dt = moa.MODES[mode]
    A, B = inputs.square_uniform(N, moa.in_dtype(dt), seed=seed)
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.empty((N, N), dtype=moa.out_dtype(dt), device="cuda")
    ws = moa.Workspace(torch.device("cuda"))
    w, wb = ws.get(moa.moa_gemm_workspace_size(N, N, N, dt, 0))
    return dt, A, B, Ad, Bd, C, ws, w, wb


def bench_energy_n(stream, energy, sizes=(1024, 2048, 4096, 8192, 16384),
                   modes=("tf32", "bf16", "f32_split", "f64_split_f64in",
                          "f64_split_f64in_e4m3", "f64_crt_f64in", "f64")):
    """Square sweep: per precision mode and N, time, TFLOP/s and NVML joules per
    GEMM, plus the least-squares slope of log J against log N (the paper
    claims energy quadratic in N)."""
    import numpy as np
    import torch

    from paper_2306_11148_b300 import moa
    res = {}
    for mode in modes:
        rows = []
        for N in sizes:
            dt, A, B, Ad, Bd, C, ws, w, wb = _prep(mode, N)
            sh = int(stream.cuda_stream)

            def step():
                moa.check(moa.moa_gemm_ex(N, N, N, dt, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(),
                                          0, w, wb, sh, None))
            with torch.cuda.stream(stream):
                step()                       # first call: one-time setup (maps, attributes)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                step()
                torch.cuda.synchronize()
                t_est = time.perf_counter() - t0
            m = measure_window(step, energy, stream, t_est)
            moa.check(moa.moa_sync_status(sh))
            m.update({"N": N, "tflops": 2.0 * N ** 3 / m["s_per_gemm"] / 1e12,
                      "rel_err_3_rows": sampled_rows_err(Ad, Bd, C, [0, N // 2, N - 1])})
            rows.append(m)
            del Ad, Bd, C, ws
            torch.cuda.empty_cache()
        fit = None
        pts = [(math.log(r["N"]), math.log(r["j_per_gemm"])) for r in rows if r.get("j_per_gemm")]
        if len(pts) >= 2:
            x = np.array([p[0] for p in pts])
            y = np.array([p[1] for p in pts])
            fit = float(np.polyfit(x, y, 1)[0])
        res[mode] = {"points": rows, "slope_logJ_logN": fit}
    return res


def bench_tiles(stream, energy, sizes=(2048, 4096, 8192), modes=("bf16", "tf32")):
    """Tile-width sweep (the paper's time/energy/power/temperature versus
    matrix size and block size): every block_n at every N."""
    import torch
    from paper_2306_11148_b300 import moa
    L = moa.lib()
    out = []
    for mode in modes:
        for N in sizes:
            dt, A, B, Ad, Bd, C, ws, w, wb = _prep(mode, N)
            sh = int(stream.cuda_stream)
            for bn in (64, 128, 256):
                moa.check(L.moa_set_block_n(bn))

                def step():
                    moa.check(moa.moa_gemm_ex(N, N, N, dt, Ad.data_ptr(), Bd.data_ptr(),
                                              C.data_ptr(), 0, w, wb, sh, None))
                with torch.cuda.stream(stream):
                    step()
                    t0 = time.perf_counter()
                    step()
                    torch.cuda.synchronize()
                    t_est = time.perf_counter() - t0
                m = measure_window(step, energy, stream, t_est, min_window=1.0)
                m.update({"mode": mode, "N": N, "block_n": bn,
                          "tflops": 2.0 * N ** 3 / m["s_per_gemm"] / 1e12})
                out.append(m)
            moa.check(L.moa_set_block_n(0))
            moa.check(moa.moa_sync_status(sh))
            del Ad, Bd, C, ws
            torch.cuda.empty_cache()
    return out


def bench_crt_tiles(stream, energy, sizes=(2048, 4096, 6144, 8192, 12288), rounds=2):
    """Tile shapes of the modular-slice mode (FP32 inputs) under sustained
    load: 128 x 256 tiles on one SM against 256 x 256 tiles on CTA pairs,
    alternating, each a >= 1.5 s window of back-to-back GEMMs (seconds per
    GEMM by CUDA events, joules by the NVML counter): the data behind the
    planner's choice."""
    import torch
    from paper_2306_11148_b300 import moa
    L = moa.lib()
    out = []
    for N in sizes:
        dt, A, B, Ad, Bd, C, ws, w, wb = _prep("f64_crt_f32in", N)
        sh = int(stream.cuda_stream)
        for r in range(rounds):
            for bm, bn in ((128, 256), (256, 256)):
                moa.check(L.moa_set_block_m(bm))
                moa.check(L.moa_set_block_n(bn))

                def step():
                    moa.check(moa.moa_gemm_ex(N, N, N, dt, Ad.data_ptr(), Bd.data_ptr(),
                                              C.data_ptr(), 0, w, wb, sh, None))
                with torch.cuda.stream(stream):
                    step()
                    t0 = time.perf_counter()
                    step()
                    torch.cuda.synchronize()
                    t_est = time.perf_counter() - t0
                m = measure_window(step, energy, stream, t_est, min_window=1.5)
                m.update({"N": N, "block_m": bm, "block_n": bn, "round": r,
                          "tflops": 2.0 * N ** 3 / m["s_per_gemm"] / 1e12})
                out.append(m)
        moa.check(L.moa_set_block_m(0))
        moa.check(L.moa_set_block_n(0))
        moa.check(moa.moa_sync_status(sh))
        del Ad, Bd, C, ws
        torch.cuda.empty_cache()
    return out


def fp64_rates(stream):
    """This device's FP64 rates (TFLOP/s) from the library's diagnostic:
    independent fused multiply-adds on the CUDA cores, and independent
    warp-level FP64 MMAs (the FP64 tensor path)."""
    import ctypes
    from paper_2306_11148_b300 import moa
    out = []
    for kind in (0, 1):
        v = ctypes.c_double(0.0)
        moa.check(moa.lib().moa_measure_fp64_rate(kind, int(stream.cuda_stream), ctypes.byref(v)))
        out.append(v.value)
    return tuple(out)


def bench_library_rates(N=8192, reps=10):
    """Dense GEMM rates of the vendor library (cuBLAS through torch) per data
    type on this GPU, next to this library's dense kernels: context for the
    roofline denominators (which stay MEASURED_PEAKS.json's BF16 figure times
    the nominal dtype ratio).  Not used on any product path."""
    import torch
    from paper_2306_11148_b300 import moa
    out = {}

    def best_ms(fn, r):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(r):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    def rate(n, ms):
        return 2.0 * n ** 3 / (ms / 1e3) / 1e12

    g = torch.Generator(device="cuda").manual_seed(0)
    a32 = torch.rand((N, N), generator=g, device="cuda") * 2 - 1
    b32 = torch.rand((N, N), generator=g, device="cuda") * 2 - 1
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        torch.backends.cuda.matmul.allow_tf32 = True
        out["cublas_tf32"] = rate(N, best_ms(lambda: a32 @ b32, reps))
        torch.backends.cuda.matmul.allow_tf32 = False
        n32 = N // 2
        out["cublas_fp32_n4096"] = rate(n32, best_ms(lambda: a32[:n32, :n32] @ b32[:n32, :n32], reps))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    a16, b16 = a32.bfloat16(), b32.bfloat16()
    out["cublas_bf16"] = rate(N, best_ms(lambda: a16 @ b16, reps))
    try:
        a8 = a32.to(torch.float8_e4m3fn)
        b8t = b32.t().contiguous().to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda")
        out["cublas_fp8_e4m3"] = rate(N, best_ms(
            lambda: torch._scaled_mm(a8, b8t.t(), scale_a=one, scale_b=one,
                                     out_dtype=torch.bfloat16), reps))
    except Exception as e:  # report, do not hide
        out["cublas_fp8_e4m3"] = f"unavailable: {e}"
    try:
        # INT8 x INT8 -> INT32 (cuBLASLt through torch._int_mm): the rate an
        # integer-digit slice variant would run at
        ai = torch.randint(-16, 17, (N, N), generator=g, device="cuda", dtype=torch.int8)
        bi = torch.randint(-16, 17, (N, N), generator=g, device="cuda", dtype=torch.int8)
        out["cublas_int8"] = rate(N, best_ms(lambda: torch._int_mm(ai, bi), reps))
        del ai, bi
    except Exception as e:  # report, do not hide
        out["cublas_int8"] = f"unavailable: {e}"
    n64 = N // 4
    a64, b64 = a32[:n64, :n64].double(), b32[:n64, :n64].double()
    out["cublas_fp64_n2048"] = rate(n64, best_ms(lambda: a64 @ b64, 3))
    # this library's dense kernels on the same operands
    c32 = torch.empty((N, N), device="cuda")
    out["moa_tf32"] = rate(N, best_ms(lambda: moa.gemm(a32, b32, moa.MOA_F32_TF32, C=c32), reps))
    out["moa_bf16"] = rate(N, best_ms(lambda: moa.gemm(a16, b16, moa.MOA_BF16, C=c32), reps))
    c64 = torch.empty((n64, n64), dtype=torch.float64, device="cuda")
    out["moa_fp64_n2048"] = rate(n64, best_ms(lambda: moa.gemm(a64, b64, moa.MOA_F64, C=c64), 3))
    # the device's own FP64 rates (library diagnostic kernels)
    fma, mma = fp64_rates(torch.cuda.current_stream())
    out["measured_fp64_fma"] = fma
    out["measured_fp64_mma"] = mma
    return out


# ------------------------------------------------------------------ reference arm
METRIC_OF = {
    "tf32": "GEMM TFLOP/s (FP32 ONF GEMM, TF32 tensor path)",
    "f64_split_f32in": "GEMM TFLOP/s (FP64-accurate ONF GEMM of FP32 inputs: BF16 integer-digit "
                       "slices on the tensor cores, exact integer accumulation)",
    "f64_split_f32in_e4m3": "GEMM TFLOP/s (FP64-accurate ONF GEMM of FP32 inputs: FP8 E4M3 "
                            "integer-digit slices on the tensor cores)",
    "f32_split": "GEMM TFLOP/s (FP32-accurate ONF GEMM: three BF16 slices, six products)",
    "f64_crt_f32in": "GEMM TFLOP/s (FP64-accurate ONF GEMM of FP32 inputs: BF16 modular slices "
                     "on the tensor cores, exact integer product by the Chinese remainder "
                     "theorem)",
}
INPUTS_OF = {m: "FP32 i.i.d. N(0,1), seed 0" for m in SPLIT_F32IN}


def square_metric_config(mode, N, ws):
    """Metric name and config of the square workloads (shared by both arms)."""
    metric = METRIC_OF.get(mode, f"GEMM TFLOP/s (ONF GEMM, {mode} path)")
    # bytes of A and B and of C per element, against the 126 MB L2
    in_b, out_b = {"bf16": (2, 4), "f64": (8, 8), "f64_split_f32in": (4, 8),
                   "f64_split_f32in_e4m3": (4, 8), "f64_crt_f32in": (4, 8),
                   "f64_crt_f64in": (8, 8)}.get(mode, (4, 4))
    mb = N * N * (2 * in_b + out_b) / 1e6
    l2 = (f"inputs larger than L2 (A, B, C: {mb:.0f} MB)" if mb > L2_MB else
          f"A, B, C fit in L2 ({mb:.1f} MB): not flushed between steps (warm-cache figure)")
    config = {"workload": f"square ONF GEMM m=n=p={N}, row-major, "
                          f"{INPUTS_OF.get(mode, 'uniform[-1,1), seed 0')}, mode {mode}",
              "N": N, "mode": mode, "parallelism": f"replicas x{ws}", "l2": l2}
    return metric, config


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle, as it stands, on the host cores; each
    step is a bounded sample of rows of the same square problem."""
    if rank != 0:
        return
    N = args.n
    mode = MODE_OF.get(args.workload, "f64_crt_f32in")
    per_step = []
    ops = cpu_operands(N, "f32", mode)
    for _ in range(args.warmup):
        cpu_baseline(N, "f32", seconds_target=2.0, operands=ops)
    for _ in range(args.steps):
        per_step.append(cpu_baseline(N, "f32", seconds_target=4.0, operands=ops))
    v = sum(x["value"] for x in per_step) / len(per_step)
    metric, config = square_metric_config(mode, N, args.gpus)
    config["arm"] = "CPU oracle (FP64 i-k-j loop, OpenMP over rows) on sampled rows"
    line = {"impl": "reference", "metric": metric, "value": v, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(x["seconds"] for x in per_step) / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": per_step[0]["cores"],
                             "kind": "oracle", "sample": per_step[0]["sample"],
                             "single_thread": per_step[0].get("single_thread")},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="moa", choices=["moa", "reference"])
    ap.add_argument("--workload", default="crt_f64", choices=list(MODE_OF))
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-sweep", type=lambda x: [float(v) for v in x.split(",") if v],
                    default=[], help="extra arrival rates (comma list) to find capacity")
    ap.add_argument("--energy-modes", type=lambda x: [v for v in x.split(",") if v], default=[],
                    help="modes of the energy_n sweep (comma list; default: all)")
    ap.add_argument("--serve-f64", default="crt", choices=["crt", "digits"],
                    help="mode of the FP64-accuracy serving requests")
    ap.add_argument("--no-extras", action="store_true", help="skip the other-mode measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--block-m", type=int, default=0, choices=[0, 128, 256],
                    help="force the modular-slice tile height (moa_set_block_m)")
    ap.add_argument("--profile", action="store_true",
                    help="timed GEMM steps only (no energy window, e2e, extras, CPU baseline)")
    args = ap.parse_args()
    if args.profile:
        args.no_extras = args.no_cpu = True
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    from paper_2306_11148_b300 import build as moa_build
    from paper_2306_11148_b300 import moa
    if rank == 0 and not os.path.exists(moa.LIB_PATH):
        moa_build.build()
    barrier(ws)
    torch.cuda.set_device(local)
    moa.lib()
    peaks = load_peaks()
    pci, uuid = gpu_identity(local)
    energy = Energy(pci, uuid)
    stream = torch.cuda.Stream()
    mode = MODE_OF[args.workload]
    N = args.n

    if args.block_m:
        moa.check(moa.lib().moa_set_block_m(args.block_m))

    if mode in ("energy_n", "tiles", "peaks", "products", "crt_tiles"):
        clocks = ClockSampler(pci)
        clocks.start()
        if mode == "products":
            res = bench_products(stream, steps=args.steps, warmup=args.warmup)
            for v in res.values():
                v["frac_of_hbm"] = v["gbs"] / peaks["hbm_gbs"]
            metric = "GB/s of the outer-product family's no-reduction members (one kernel)"
            value = res["kronecker"]["gbs"]
            unit = "GB/s (Kronecker product, FP32, 8192 x 8192 output)"
        elif mode == "peaks":
            res = bench_library_rates(args.n)
            metric = "dense GEMM TFLOP/s per dtype: vendor library vs this library"
            value = res["moa_tf32"]
            unit = "TFLOP/s (this library, TF32)"
        elif mode == "crt_tiles":
            res = bench_crt_tiles(stream, energy)
            metric = "modular-slice GEMM time and energy: one-SM vs CTA-pair tiles vs N"
            best = max(res, key=lambda r: r["tflops"])
            value = best["tflops"]
            unit = "TFLOP/s (best cell)"
        elif mode == "energy_n":
            res = bench_energy_n(stream, energy, **({"modes": tuple(args.energy_modes)}
                                                     if args.energy_modes else {}))
            metric = "joules per square ONF GEMM vs N (slope of log J vs log N)"
            value = res[next(iter(res))]["slope_logJ_logN"]
            unit = "dlogJ/dlogN"
        else:
            res = bench_tiles(stream, energy)
            metric = "time/energy/power/temperature vs N and tile width"
            best = max(res, key=lambda r: r["tflops"])
            value = best["tflops"]
            unit = "TFLOP/s (best cell)"
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": metric, "value": value, "unit": unit, "n_gpus": ws,
                              "higher_is_better": mode != "energy_n", "scaling": "weak",
                              "vs_baseline": None, "data": "synthetic",
                              "config": {"workload": mode, "parallelism": f"replicas x{ws}"},
                              "results": res, "clocks": clk}), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    if mode == "serve":
        ops = ServeOperands(nbuf=4)
        clocks = ClockSampler(pci)
        clocks.start()
        sat = bench_serve(ops, args.serve_rate, args.serve_seconds, energy=energy,
                          f64_mode=args.serve_f64)
        sweep = []
        for r in args.serve_sweep:
            sweep.append(bench_serve(ops, r, args.serve_seconds, energy=energy,
                                     f64_mode=args.serve_f64))
        clk = clocks.stop()
        # capacity: the highest served rate seen; a run at ~70 % of it
        cap = max([sat["served_per_s"]] + [x["served_per_s"] for x in sweep])
        light = bench_serve(ops, 0.7 * cap, args.serve_seconds, energy=energy,
                            f64_mode=args.serve_f64) \
            if args.serve_sweep else None
        if rank == 0:
            line = {"metric": "served GEMM requests/s (continuous batching), p50/p99 latency",
                    "value": sat["served_per_s"] * ws, "unit": "req/s", "n_gpus": ws,
                    "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "bf16-slices", "data": "synthetic",
                    "config": {"workload": f"Poisson arrivals {args.serve_rate}/s for "
                                           f"{args.serve_seconds} s, each its own (m, n, p): "
                                           "m,p logU[64,4096], n logU[64,8192]; FP32-acc or "
                                           "FP64-acc split requests; 64 GB arena; 32 in "
                                           "flight; 8 streams",
                               "parallelism": f"replicas x{ws}"},
                    "specified_rate": sat, "rate_sweep": sweep, "capacity_req_s": cap,
                    "at_70pct_capacity": light, "clocks": clk}
            print(json.dumps(line), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    clocks = ClockSampler(pci)
    clocks.start()
    # the split modes' error check: 64 sampled rows of C on each input kind
    check_idx = None
    if mode in SPLIT_F32IN and rank == 0 and not args.no_cpu:
        from paper_2306_11148_b300 import inputs as _inputs
        check_idx = _inputs.sample_rows(N, 64, seed=0)
    if mode == "grouped":
        main_res = bench_grouped(args.steps, args.warmup, ws, stream, compare=not args.profile)
    else:
        main_res = bench_mode(mode, N, args.steps, args.warmup, ws, stream,
                              want_energy=not args.profile, energy=energy,
                              want_e2e=not args.profile, check_rows=not args.profile,
                              keep_rows=check_idx)
    clk = clocks.stop()
    rows_c = None
    if check_idx is not None:
        rows_c = {"plain": main_res.pop("rows_C")}
        for kind in ("rows", "rowcol"):
            rows_c[kind] = gpu_rows(mode, N, kind, check_idx, stream)

    value, t_max = aggregate(main_res["flops_per_step"], args.steps, main_res["seconds"], ws)
    ms_per_step = t_max / args.steps * 1e3

    e2e = main_res.get("e2e", {})
    e2e_t = max_over_ranks(e2e.get("seconds", float("nan")), ws)
    e2e_val = main_res["flops_per_step"] * e2e.get("steps", 1) * ws / e2e_t / 1e12

    # roofline of the dominant kernel: algorithmic flops (or bytes) per launch
    # / that kernel's own CUDA-event duration, recorded by the library on the
    # launching stream.
    kdtype = {"tf32": "tf32", "bf16": "bf16", "f32_split": "bf16",
              "f64_split_f32in": "bf16", "f64_split_f32in_e4m3": "fp8", "f64_crt_f32in": "bf16",
              "f64_crt_f64in": "bf16",
              "grouped": "bf16"}.get(mode)
    kernel_ms = main_res["kernel_seconds"] / args.steps * 1e3
    if mode == "grouped":
        # mixed: small problems are HBM-bound, large ones tensor-bound; the
        # bound of the batch is max(flops / tensor peak, bytes / HBM peak)
        peak_t = peaks["bf16_tflops"]
        t_tensor = main_res["flops_per_step"] / (peak_t * 1e12)
        t_hbm = main_res["bytes_per_step"] / (peaks["hbm_gbs"] * 1e9)
        if t_tensor >= t_hbm:
            achieved = main_res["flops_per_step"] / (kernel_ms / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak_t, "unit": "TFLOP/s",
                    "frac": achieved / peak_t}
        else:
            achieved = main_res["bytes_per_step"] / (kernel_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"]}
        roof.update({"traffic": traffic_of(mode, N)[0], "kernel_ms": kernel_ms,
                     "kernel": "grouped_tc_kernel",
                     "bound_times_ms": {"tensor": t_tensor * 1e3, "hbm": t_hbm * 1e3},
                     "peak_source": peaks["source"]})
    elif kdtype:
        peak = peaks["bf16_tflops"] * NOMINAL_RATIO[kdtype]
        # tensor work per launch = products x 2N^3 (one per slice product)
        achieved = main_res["flops_per_step"] * max(1, main_res["products"]) / \
            (kernel_ms / 1e3) / 1e12
        # the burst figure is the peak of record; a launch of 10 ms or more runs
        # at the power-capped clock, which the sustained figure measures, so
        # that fraction is reported beside it for such launches only
        peak_s = peaks.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"]) * \
            NOMINAL_RATIO[kdtype]
        traffic, tnote = traffic_of(mode, N)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_note": tnote,
                "kernel_ms": kernel_ms,
                "work_per_launch": f"{max(1, main_res['products'])} slice products x 2N^3 "
                                   f"= {main_res['flops_per_step'] * max(1, main_res['products']):.4g}"
                                   " flop" if main_res["products"] > 1 else "2N^3 flop",
                "peak_source": f"{peaks['source']} bf16 burst x nominal {kdtype}/bf16 ratio",
                "kernel": {"tf32": "dense_tc_kernel", "bf16": "dense_tc_kernel",
                           "f64_crt_f32in": "crt_gemm_kernel",
                           "f64_crt_f64in": "crt_gemm_kernel"}.get(mode, "split_gemm_kernel")}
        if roof["kernel"] == "crt_gemm_kernel" and main_res["tile"][0] == 256:
            roof["kernel"] = "crt_gemm_pair_kernel"   # 256 x 256 tiles on CTA pairs
        if kernel_ms >= 10.0:
            roof.update({"peak_sustained": peak_s, "frac_sustained": achieved / peak_s})
    else:
        roof = {"bound": "alu", "achieved": value / ws, "peak": None, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "kernel_ms": kernel_ms}

    modes = {}
    if not args.no_extras and rank == 0 and ws == 1 and mode != "grouped":
        for m2, n2 in [("tf32", N), ("bf16", N), ("f32_split", N), ("f64_split_f32in", N),
                       ("f64_crt_f32in", N), ("f64_split_f32in_e4m3", N), ("f32_simt", N // 2),
                       ("f64", N // 4)]:
            if m2 == mode:
                continue
            try:
                r = bench_mode(m2, n2, 3, 2, 1, stream, want_energy=(n2 == N), energy=energy)
                r["tflops"] = r["flops_per_step"] * r["steps"] / r["seconds"] / 1e12
                modes[m2] = r
            except Exception as e:  # report, do not hide
                modes[m2] = {"error": str(e)}
        # the native FP64 GEMM against this device's measured FP64 rates
        if "tflops" in modes.get("f64", {}):
            try:
                fma, mma = fp64_rates(stream)
                modes["f64"].update({"fp64_fma_tflops_measured": fma,
                                     "fp64_mma_tflops_measured": mma,
                                     "frac_of_measured_fp64_fma": modes["f64"]["tflops"] / fma})
            except Exception as e:  # report, do not hide
                modes["f64"]["fp64_rates"] = {"error": str(e)}

        # the outer-product family's no-reduction members (HBM roofline)
        try:
            pr = bench_products(stream)
            for v in pr.values():
                v["frac_of_hbm"] = v["gbs"] / peaks["hbm_gbs"]
            modes["products"] = pr
        except Exception as e:  # report, do not hide
            modes["products"] = {"error": str(e)}
        # grouped modular-slice batches against separate launches
        for div in (1, 4):
            try:
                modes[f"grouped_crt_div{div}"] = bench_grouped_split(stream, count=64, div=div)
            except Exception as e:  # report, do not hide
                modes[f"grouped_crt_div{div}"] = {"error": str(e)}
            try:
                modes[f"grouped_f32_split_div{div}"] = bench_grouped_split(stream, count=64, div=div,
                                                                         mode="f32_split")
            except Exception as e:  # report, do not hide
                modes[f"grouped_f32_split_div{div}"] = {"error": str(e)}
        # a short run of the serving stream (each arrival its own shape)
        try:
            ops = ServeOperands(nbuf=2)
            modes["serve"] = bench_serve(ops, args.serve_rate, min(args.serve_seconds, 5.0),
                                         energy=energy, f64_mode=args.serve_f64)
            modes["serve"]["workload"] = (f"Poisson arrivals {args.serve_rate}/s for "
                                          f"{min(args.serve_seconds, 5.0)} s, each its own "
                                          "(m, n, p): m,p logU[64,4096], n logU[64,8192]; "
                                          "FP32-acc or FP64-acc split requests")
            del ops
        except Exception as e:  # report, do not hide
            modes["serve"] = {"error": str(e)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu and mode != "grouped":
        if rows_c is not None:
            cpu = cpu_baseline_split(mode, N, rows_c, check_idx)
        else:
            cpu = cpu_baseline(N, "f32")

    if rank == 0:
        if mode == "grouped":
            metric = "GEMM TFLOP/s (512 grouped BF16 GEMMs, one persistent launch)"
            config = {"workload": "512 ONF GEMMs, m,n,p log-uniform in [32,2048] rounded to 16, "
                                  "BF16 in (uniform[-1,1) seeds 1000+i), FP32 out, one "
                                  "moa_gemm_grouped launch per step",
                      "count": main_res["count"], "parallelism": f"replicas x{ws}",
                      "l2": "operands ~0.96 GB per step, larger than L2",
                      "separate_launches_ms": main_res["separate_seconds_per_step"] * 1e3,
                      "separate_tflops": main_res["flops_per_step"] /
                      main_res["separate_seconds_per_step"] / 1e12,
                      "separate_in_cuda_graph_ms": main_res["graph_seconds_per_step"] * 1e3,
                      "separate_in_cuda_graph_tflops": main_res["flops_per_step"] /
                      main_res["graph_seconds_per_step"] / 1e12}
        else:
            metric, config = square_metric_config(mode, N, ws)
        if cpu is not None and "rel_err_vs_oracle" in cpu:
            tol = 1e-5 if mode == "f32_split" else 1e-12
            config["error_check"] = (f"relative Frobenius error vs the FP64 oracle on "
                                     f"{cpu['rows_checked']} sampled rows per input kind, "
                                     f"tolerance {tol:g}")
        line = {
            "metric": metric,
            "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"tf32": "tf32", "bf16": "bf16", "f32_split": "bf16x6",
                      "f64_split_f32in": "f64 via bf16 integer digits (exact int accumulation)",
                      "f64_split_f32in_e4m3": "f64 via e4m3 integer digits",
                      "f64_crt_f32in": "f64 via bf16 modular slices (exact integer CRT)",
                      "f64_crt_f64in": "f64 via bf16 modular slices (exact integer CRT)",
                      "f64": "f64",
                      "f32_simt": "f32", "grouped": "bf16"}[mode],
            "data": "synthetic",
            "config": config,
            "rel_err_vs_oracle": (cpu or {}).get("rel_err_vs_oracle"),
            "rel_err_sampled_rows": main_res.get("rel_err_sampled_rows"),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val if math.isfinite(e2e_val) else None, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": e2e.get("h2d_bytes_per_step"),
                    "d2h_bytes_per_step": e2e.get("d2h_bytes_per_step"),
                    "api": e2e.get("api"), "streams": e2e.get("streams"),
                    "steps": e2e.get("steps")},
            "gpu_launches": main_res["kernels_per_step"] * args.steps,
            "clocks": clk,
            "energy": main_res.get("energy") or {"unavailable": energy.why},
            "tile": main_res["tile"],
            "modes": modes,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
