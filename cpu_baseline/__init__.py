"""Parallel float32 CPU baseline of the skeleton hot path -- MEASUREMENT ONLY.

The benchmark reports this multi-core CPU implementation (``cpu_parallel.cpp``,
std::thread over the cores of the process's affinity mask, float32 / int32
like the GPU) beside the GPU numbers, together with the host's CPU model and
core count.  It is not the oracle: the oracle (``oracle/``) is sequential
float64 code that checks results; this one exists to be timed.  Nothing of the
product path imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_parallel.cpp")
_LIB_PATH = os.path.join(_HERE, f"libcpu_parallel.{platform.machine()}.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile cpu_parallel.cpp (g++, portable flags: it also builds on Arm)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O3", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            f, i64, i32, vp = C.c_float, C.c_int64, C.c_int, C.c_void_p
            sig = {
                "cpu_map_axpy": (None, [vp, vp, vp, i64, f, i32]),
                "cpu_reduce_sum": (f, [vp, i64, i32]),
                "cpu_reduce_max": (f, [vp, i64, i32]),
                "cpu_dot": (f, [vp, vp, i64, i32]),
                "cpu_scan_i32": (None, [vp, vp, i64, i32, i32]),
                "cpu_scan_f32": (None, [vp, vp, i64, i32, i32]),
                "cpu_scan_bwd_f32": (None, [vp, vp, i64, i32]),
                "cpu_stencil2d": (None, [vp, vp, i64, i64, vp, i32]),
                "cpu_stencil1d": (None, [vp, vp, i64, i32, vp, i32]),
                "cpu_stencil2d_bwd": (None, [vp, vp, i64, i64, vp, i32]),
                "cpu_rowdot": (None, [vp, vp, i64, i64, vp, i32]),
                "cpu_gather": (None, [vp, i64, vp, i64, vp, i32]),
                "cpu_map_tanh_bwd": (None, [vp, vp, vp, i64, i32]),
                "cpu_batched": (None, [vp, vp, i64, vp, vp, i32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def cores() -> int:
    """Cores this process may run on (its affinity mask)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu() -> dict:
    """CPU model and core counts of this host (lscpu, else /proc/cpuinfo)."""
    names, vendor = [], None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k == "Model name" and v and v not in names:
                names.append(v)
            elif k == "Vendor ID" and v:
                vendor = v
    except (OSError, subprocess.SubprocessError):
        pass
    if not names:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    names.append(line.split(":", 1)[1].strip())
                    break
        except OSError:
            pass
    model = " ".join(x for x in [vendor, ", ".join(names)] if x) or platform.processor() or platform.machine()
    return {"model": model, "arch": platform.machine(), "cores_affinity": cores(), "cores_online": os.cpu_count()}


def _p(a: np.ndarray) -> C.c_void_p:
    return C.c_void_p(a.ctypes.data)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def map_axpy(x, y, a: float, out=None, nthreads: int | None = None):
    x, y = _f32(x), _f32(y)
    out = np.empty_like(x) if out is None else out
    _load().cpu_map_axpy(_p(x), _p(y), _p(out), x.size, a, nthreads or cores())
    return out


def reduce_sum(x, nthreads=None) -> float:
    x = _f32(x)
    return _load().cpu_reduce_sum(_p(x), x.size, nthreads or cores())


def reduce_max(x, nthreads=None) -> float:
    x = _f32(x)
    return _load().cpu_reduce_max(_p(x), x.size, nthreads or cores())


def dot(x, y, nthreads=None) -> float:
    x, y = _f32(x), _f32(y)
    return _load().cpu_dot(_p(x), _p(y), x.size, nthreads or cores())


def scan_i32(x, inclusive: bool, out=None, nthreads=None):
    x = np.ascontiguousarray(x, dtype=np.int32)
    out = np.empty_like(x) if out is None else out
    _load().cpu_scan_i32(_p(x), _p(out), x.size, int(inclusive), nthreads or cores())
    return out


def scan_f32(x, inclusive: bool, out=None, nthreads=None):
    x = _f32(x)
    out = np.empty_like(x) if out is None else out
    _load().cpu_scan_f32(_p(x), _p(out), x.size, int(inclusive), nthreads or cores())
    return out


def scan_bwd_f32(g, out=None, nthreads=None):
    g = _f32(g)
    out = np.empty_like(g) if out is None else out
    _load().cpu_scan_bwd_f32(_p(g), _p(out), g.size, nthreads or cores())
    return out


def stencil2d(x, w, out=None, nthreads=None):
    x, w = _f32(x), _f32(w).ravel()
    out = np.empty_like(x) if out is None else out
    _load().cpu_stencil2d(_p(x), _p(out), x.shape[0], x.shape[1], _p(w), nthreads or cores())
    return out


def stencil2d_bwd(g, w, out=None, nthreads=None):
    g, w = _f32(g), _f32(w).ravel()
    out = np.empty_like(g) if out is None else out
    _load().cpu_stencil2d_bwd(_p(g), _p(out), g.shape[0], g.shape[1], _p(w), nthreads or cores())
    return out


def stencil1d(x, r: int, w, out=None, nthreads=None):
    x, w = _f32(x), _f32(w)
    out = np.empty_like(x) if out is None else out
    _load().cpu_stencil1d(_p(x), _p(out), x.size, r, _p(w), nthreads or cores())
    return out


def rowdot(A, M, out=None, nthreads=None):
    A, M = _f32(A), _f32(M)
    out = np.empty(M.shape[0], np.float32) if out is None else out
    _load().cpu_rowdot(_p(A), _p(M), M.shape[0], M.shape[1], _p(out), nthreads or cores())
    return out


def gather(A, idx, out=None, nthreads=None):
    A, idx = _f32(A), np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(idx.size, np.float32) if out is None else out
    _load().cpu_gather(_p(A), A.size, _p(idx), idx.size, _p(out), nthreads or cores())
    return out


def map_tanh_bwd(x, g, out=None, nthreads=None):
    x, g = _f32(x), _f32(g)
    out = np.empty_like(x) if out is None else out
    _load().cpu_map_tanh_bwd(_p(x), _p(g), _p(out), x.size, nthreads or cores())
    return out


def batched(v, off, res=None, scan=None, nthreads=None):
    v, off = _f32(v), np.ascontiguousarray(off, dtype=np.int64)
    B = off.size - 1
    res = np.empty(B, np.float32) if res is None else res
    scan = np.empty_like(v) if scan is None else scan
    _load().cpu_batched(_p(v), _p(off), B, _p(res), _p(scan), nthreads or cores())
    return res, scan
