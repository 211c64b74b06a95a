"""CPU oracle of the skeleton hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product package never imports it and
it imports nothing of the product.  The arithmetic lives in ``oracle.c``
(plain sequential C, float64 / int64); this module compiles it with gcc and
marshals numpy arrays in and out.  ``coherence.py`` holds the plain model of
the smart-container protocol (Sec. IV).

Every function takes the same float32 / int32 arrays the GPU receives and
returns float64 / int64 results.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, f"liboracle.{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

# Oracle-local codes (must match the enums at the top of oracle.c).
FN = {"axpy": 0, "mul": 1, "add": 2, "tanh": 3, "sq": 4, "scale": 5, "copy": 6, "sub": 7, "max": 8}
BOUNDARY = {"clamp": 0, "zero": 1, "periodic": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
            sig = {
                "oracle_map_f32": (i32, [i32, d, vp, vp, i64, vp]),
                "oracle_map_bwd_f32": (i32, [i32, d, vp, vp, vp, i64, vp, vp]),
                "oracle_reduce_sum_f32": (d, [vp, i64, vp]),
                "oracle_reduce_max_f32": (d, [vp, i64]),
                "oracle_reduce_sum_i32": (i64, [vp, i64]),
                "oracle_reduce_max_i32": (C.c_int32, [vp, i64]),
                "oracle_mapreduce_f32": (d, [i32, d, vp, vp, i64, vp]),
                "oracle_scan_i32": (None, [vp, i64, i32, vp]),
                "oracle_scan_f32": (None, [vp, i64, i32, vp, vp]),
                "oracle_scan_bwd_f32": (None, [vp, i64, i32, vp, vp]),
                "oracle_mapoverlap1d_f32": (None, [vp, i64, i32, vp, i32, vp]),
                "oracle_mapoverlap2d_f32": (None, [vp, i64, i64, i32, vp, i32, vp]),
                "oracle_mapoverlap1d_bwd_f32": (None, [vp, i64, i32, vp, i32, vp]),
                "oracle_mapoverlap2d_bwd_f32": (None, [vp, i64, i64, i32, vp, i32, vp]),
                "oracle_gather_f32": (None, [vp, i64, vp, i64, vp]),
                "oracle_rowdot_f32": (None, [vp, i64, vp, i64, vp, vp]),
                "oracle_mapoverlap2d_chain_f32": (None, [vp, i64, i64, i32, vp, i32, i32, vp]),
                "oracle_coulomb_points_f32": (None, [vp, i64, vp, vp, i64, d, d, vp, vp]),
                "oracle_batched_f32": (None, [vp, vp, i64, i32, vp, vp, vp]),
                "oracle_composed_loss_f32": (d, [vp, i64, i64, i32, vp, i32, vp]),
                "oracle_composed_loss_f64": (d, [vp, i64, i64, i32, vp, i32]),
                "oracle_composed_loss_delta_f32": (d, [vp, i64, i64, i32, vp, i32, i64, i64, d]),
                "oracle_chain_map_stencil_sumsq_f32": (d, [i32, d, vp, i64, i64, i32, vp, i32, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------------ Map ---
def map_f32(fn: str, x, y=None, a: float = 0.0) -> np.ndarray:
    x, y = _f32(x), _f32(y)
    out = np.empty(x.size, dtype=np.float64)
    _load().oracle_map_f32(FN[fn], a, _p(x), _p(y), x.size, _p(out))
    return out.reshape(x.shape)


def map_bwd_f32(fn: str, g, x=None, y=None, a: float = 0.0):
    g, x, y = _f32(g), _f32(x), _f32(y)
    gx = np.empty(g.size, dtype=np.float64)
    gy = np.empty(g.size, dtype=np.float64) if y is not None else None
    _load().oracle_map_bwd_f32(FN[fn], a, _p(x), _p(y), _p(g), g.size, _p(gx), _p(gy))
    return gx.reshape(g.shape), (None if gy is None else gy.reshape(g.shape))


# --------------------------------------------------------------- Reduce ---
def reduce_f32(op: str, x):
    """Returns (value, sum |x|) for 'add'; (value, 0.0) for 'max'."""
    x = _f32(x)
    if op == "add":
        a = C.c_double()
        v = _load().oracle_reduce_sum_f32(_p(x), x.size, C.byref(a))
        return v, a.value
    if op == "max":
        return _load().oracle_reduce_max_f32(_p(x), x.size), 0.0
    raise ValueError(op)


def reduce_i32(op: str, x) -> int:
    x = _i32(x)
    if op == "add":
        return int(_load().oracle_reduce_sum_i32(_p(x), x.size))
    if op == "max":
        return int(_load().oracle_reduce_max_i32(_p(x), x.size))
    raise ValueError(op)


def mapreduce_f32(fn: str, x, y=None, a: float = 0.0):
    """Returns (sum_i f(x_i, y_i), sum_i |f(x_i, y_i)|)."""
    x, y = _f32(x), _f32(y)
    s = C.c_double()
    v = _load().oracle_mapreduce_f32(FN[fn], a, _p(x), _p(y), x.size, C.byref(s))
    return v, s.value


# ----------------------------------------------------------------- Scan ---
def scan_i32(x, inclusive: bool = True) -> np.ndarray:
    x = _i32(x)
    out = np.empty(x.size, dtype=np.int64)
    _load().oracle_scan_i32(_p(x), x.size, int(inclusive), _p(out))
    return out


def scan_f32(x, inclusive: bool = True):
    """Returns (scan, running sum of |x| over the same index range)."""
    x = _f32(x)
    out = np.empty(x.size, dtype=np.float64)
    ab = np.empty(x.size, dtype=np.float64)
    _load().oracle_scan_f32(_p(x), x.size, int(inclusive), _p(out), _p(ab))
    return out, ab


def scan_bwd_f32(g, inclusive: bool = True):
    """Returns (reverse scan of g, running sum of |g| over the same range)."""
    g = _f32(g)
    out = np.empty(g.size, dtype=np.float64)
    ab = np.empty(g.size, dtype=np.float64)
    _load().oracle_scan_bwd_f32(_p(g), g.size, int(inclusive), _p(out), _p(ab))
    return out, ab


# ----------------------------------------------------------- MapOverlap ---
def mapoverlap1d_f32(x, r: int, w, boundary: str = "clamp") -> np.ndarray:
    x, w = _f32(x), _f32(w)
    assert w.size == 2 * r + 1
    out = np.empty(x.size, dtype=np.float64)
    _load().oracle_mapoverlap1d_f32(_p(x), x.size, r, _p(w), BOUNDARY[boundary], _p(out))
    return out


def mapoverlap2d_f32(x, r: int, w, boundary: str = "clamp") -> np.ndarray:
    """x: 2D (rows, cols); w: (2r+1, 2r+1) weights."""
    x, w = _f32(x), _f32(w)
    assert x.ndim == 2 and w.size == (2 * r + 1) ** 2
    out = np.empty(x.shape, dtype=np.float64)
    _load().oracle_mapoverlap2d_f32(_p(x), x.shape[0], x.shape[1], r, _p(w),
                                    BOUNDARY[boundary], _p(out))
    return out


def mapoverlap2d_chain_f32(x, r: int, w, boundary: str, steps: int) -> np.ndarray:
    """S^steps(x) for the 2D stencil S of mapoverlap2d_f32, in float64 throughout."""
    x, w = _f32(x), _f32(w)
    assert x.ndim == 2 and w.size == (2 * r + 1) ** 2 and steps >= 0
    out = np.empty(x.shape, dtype=np.float64)
    _load().oracle_mapoverlap2d_chain_f32(_p(x), x.shape[0], x.shape[1], r, _p(w), BOUNDARY[boundary], int(steps),
                                          _p(out))
    return out


def mapoverlap1d_bwd_f32(g, r: int, w, boundary: str = "clamp") -> np.ndarray:
    g, w = _f32(g), _f32(w)
    out = np.empty(g.size, dtype=np.float64)
    _load().oracle_mapoverlap1d_bwd_f32(_p(g), g.size, r, _p(w), BOUNDARY[boundary], _p(out))
    return out


def mapoverlap2d_bwd_f32(g, r: int, w, boundary: str = "clamp") -> np.ndarray:
    g, w = _f32(g), _f32(w)
    out = np.empty(g.shape, dtype=np.float64)
    _load().oracle_mapoverlap2d_bwd_f32(_p(g), g.shape[0], g.shape[1], r, _p(w),
                                        BOUNDARY[boundary], _p(out))
    return out


# ------------------------------------------------------------- MapArray ---
def gather_f32(A, idx) -> np.ndarray:
    A, idx = _f32(A), _i32(idx)
    out = np.empty(idx.size, dtype=np.float64)
    _load().oracle_gather_f32(_p(A), A.size, _p(idx), idx.size, _p(out))
    return out


def rowdot_f32(A, M):
    """Returns (M @ A row by row, sum_k |A_k M_ik| per row)."""
    A, M = _f32(A), _f32(M)
    n, m = M.shape
    assert A.size == m
    out = np.empty(n, dtype=np.float64)
    ab = np.empty(n, dtype=np.float64)
    _load().oracle_rowdot_f32(_p(A), m, _p(M), n, _p(out), _p(ab))
    return out, ab


def coulomb_points_f32(atoms, ii, jj, h: float, z0: float):
    """Potential of the atoms (m x 4 float32: x, y, z, q) at grid points
    (ii[p], jj[p]) placed at (jj*h, ii*h, z0).  Returns (value, sum |q|/r)."""
    atoms = _f32(atoms).reshape(-1, 4)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    assert ii.shape == jj.shape
    out = np.empty(ii.size, dtype=np.float64)
    ab = np.empty(ii.size, dtype=np.float64)
    _load().oracle_coulomb_points_f32(_p(atoms), atoms.shape[0], _p(ii), _p(jj), ii.size, float(h), float(z0),
                                      _p(out), _p(ab))
    return out, ab


def coulomb_grid_f32(atoms, rows: int, cols: int, h: float, z0: float):
    """The whole grid (rows x cols) of coulomb_points_f32."""
    ii, jj = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    v, ab = coulomb_points_f32(atoms, ii.ravel(), jj.ravel(), h, z0)
    return v.reshape(rows, cols), ab.reshape(rows, cols)


# -------------------------------------------------------------- Batched ---
def batched_f32(v, offsets, inclusive: bool = True):
    """Returns (sumsq per instance, per-instance scan, per-instance |x| prefix)."""
    v = _f32(v)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    B = off.size - 1
    sumsq = np.empty(B, dtype=np.float64)
    out = np.empty(v.size, dtype=np.float64)
    ab = np.empty(v.size, dtype=np.float64)
    _load().oracle_batched_f32(_p(v), _p(off), B, int(inclusive), _p(sumsq), _p(out), _p(ab))
    return sumsq, out, ab


# --------------------------------------------------------- Composed loss ---
def composed_loss_f32(x, r: int, w, boundary: str = "clamp", grad: bool = True):
    """Returns (L, dL/dx or None) of the composed loss on a 2D float32 grid."""
    x, w = _f32(x), _f32(w)
    g = np.empty(x.shape, dtype=np.float64) if grad else None
    L = _load().oracle_composed_loss_f32(_p(x), x.shape[0], x.shape[1], r, _p(w),
                                         BOUNDARY[boundary], _p(g))
    return L, g


def chain_map_stencil_sumsq_f32(fn: str, x, r: int, w, boundary: str = "clamp", a: float = 0.0):
    """Returns (sum_p (S f(x))_p^2, sum_p (sum_taps |w| |f(x)|)^2): the chain
    Map -> 2D MapOverlap -> MapReduce(sq, +) on a 2D float32 grid, and the
    scale of its float32 rounding bound."""
    x, w = _f32(x), _f32(w)
    bound = C.c_double(0.0)
    v = _load().oracle_chain_map_stencil_sumsq_f32(FN[fn], float(a), _p(x), x.shape[0], x.shape[1], r, _p(w),
                                                   BOUNDARY[boundary], C.byref(bound))
    return v, bound.value


def composed_loss_f64(x, r: int, w, boundary: str = "clamp") -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = _f32(w)
    return _load().oracle_composed_loss_f64(_p(x), x.shape[0], x.shape[1], r, _p(w),
                                            BOUNDARY[boundary])


def composed_loss_delta_f32(x, r: int, w, i: int, j: int, h: float, boundary: str = "clamp") -> float:
    x, w = _f32(x), _f32(w)
    return _load().oracle_composed_loss_delta_f32(_p(x), x.shape[0], x.shape[1], r, _p(w),
                                                  BOUNDARY[boundary], i, j, h)


# ------------------------------------------------------- Default weights ---
def stencil_weights(kind: str) -> np.ndarray:
    """The stencil weights of the workloads (a reading of the unspecified
    'weights summing to 1'; exact binary fractions, so the float32 weights the
    GPU receives equal these):
      '5pt': centre 1/2, N/S/W/E 1/8 each (3x3 with zero corners);
      '9pt': [1 2 1]^T [1 2 1] / 16."""
    if kind == "5pt":
        return np.array([[0, 1, 0], [1, 4, 1], [0, 1, 0]], dtype=np.float32) / np.float32(8)
    if kind == "9pt":
        v = np.array([1, 2, 1], dtype=np.float32)
        return np.outer(v, v).astype(np.float32) / np.float32(16)
    raise ValueError(kind)
