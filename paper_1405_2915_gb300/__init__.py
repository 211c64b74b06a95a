"""Python binding of libskel.so: data-parallel skeletons over smart
containers on one GB300 (sm_103a).

Every function named ``skel_*`` here is a thin wrapper of the C function of
the same name in include/skel.h: it converts Python arguments (containers,
function names, torch streams) into the C arguments and raises SkelError on a
non-zero status.  All computation happens in the CUDA kernels of libskel.so;
if the library is missing, importing this package fails.

PyTorch supplies device memory and streams only: by default the library's
device allocations go through torch's caching allocator, and calls are
enqueued on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from typing import Iterable, Sequence

import numpy as np

from . import _lib
from ._lib import BOUNDARY, FN, SK, SkelError, F32, I32, I64, READ, WRITE, READWRITE, UNIT_HOST, UNIT_DEVICE

lib = _lib.load()

_NP2DT = {np.dtype(np.float32): F32, np.dtype(np.int32): I32, np.dtype(np.int64): I64}
_DT2NP = {F32: np.float32, I32: np.int32, I64: np.int64}


def check(rc: int) -> None:
    if rc != 0:
        raise SkelError(rc, lib.skel_last_error().decode())


def _torch():
    import torch
    return torch


def current_stream() -> int:
    """cudaStream_t of torch's current stream (0 = legacy default stream)."""
    return _torch().cuda.current_stream().cuda_stream


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = current_stream()
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    return C.c_void_p(stream)


# ------------------------------------------------------------- allocator ---
_alloc_refs = []


def use_torch_allocator(enable: bool = True) -> None:
    """Routes the library's device allocations through torch's caching
    allocator (enable=True) or back to the library's built-in
    cudaMallocAsync pool (enable=False)."""
    if not enable:
        check(lib.skel_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None))
        _alloc_refs.clear()
        return
    torch = _torch()

    def _alloc(size, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    a, f = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
    _alloc_refs[:] = [a, f]
    check(lib.skel_set_allocator(a, f, None))


# ------------------------------------------------------------- containers ---
class Container:
    """Owning Python handle of a skel container (Sec. IV smart container).

    Keeps alive whatever Python object owns wrapped memory (a torch tensor or
    a numpy array)."""

    def __init__(self, handle: int, keep=(), parent: "Container | None" = None):
        self.handle = C.c_void_p(handle)
        self._keep = list(keep)
        self._parent = parent
        self._views = 0
        if parent is not None:
            parent._views += 1

    # constructors ---------------------------------------------------------
    @classmethod
    def empty(cls, shape, dtype=np.float32) -> "Container":
        shape = tuple(int(s) for s in (shape if isinstance(shape, Iterable) else (shape,)))
        arr = (C.c_int64 * 2)(*shape, *([1] * (2 - len(shape))))
        h = C.c_void_p()
        check(lib.skel_container_create(_NP2DT[np.dtype(dtype)], len(shape), arr, C.byref(h)))
        return cls(h.value)

    @classmethod
    def from_tensor(cls, t, host=None) -> "Container":
        """Wraps a contiguous CUDA tensor (its device copy is valid)."""
        torch = _torch()
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("from_tensor needs a contiguous CUDA tensor")
        dt = {torch.float32: F32, torch.int32: I32, torch.int64: I64}[t.dtype]
        shape = tuple(t.shape) if t.dim() in (1, 2) else (t.numel(),)
        arr = (C.c_int64 * 2)(*shape, *([1] * (2 - len(shape))))
        h = C.c_void_p()
        hp = None if host is None else host.ctypes.data
        check(lib.skel_container_wrap(dt, len(shape), arr, C.c_void_p(hp), C.c_void_p(t.data_ptr()),
                                      UNIT_DEVICE, C.byref(h)))
        return cls(h.value, keep=[t] + ([host] if host is not None else []))

    @classmethod
    def from_host(cls, a: np.ndarray, valid: bool = True) -> "Container":
        """Wraps a contiguous host array (pinned or pageable); its host copy
        is valid when `valid`; device storage is allocated lazily."""
        if not a.flags.c_contiguous:
            raise ValueError("from_host needs a C-contiguous array")
        shape = a.shape if a.ndim in (1, 2) else (a.size,)
        arr = (C.c_int64 * 2)(*shape, *([1] * (2 - len(shape))))
        h = C.c_void_p()
        check(lib.skel_container_wrap(_NP2DT[a.dtype], len(shape), arr, C.c_void_p(a.ctypes.data), None,
                                      UNIT_HOST if valid else 0, C.byref(h)))
        return cls(h.value, keep=[a])

    def view(self, offset: int, shape) -> "Container":
        shape = tuple(int(s) for s in (shape if isinstance(shape, Iterable) else (shape,)))
        arr = (C.c_int64 * 2)(*shape, *([1] * (2 - len(shape))))
        h = C.c_void_p()
        check(lib.skel_container_view(self.handle, int(offset), len(shape), arr, C.byref(h)))
        return Container(h.value, parent=self)

    # accessors ------------------------------------------------------------
    def info(self):
        dt, nd, v = C.c_int(), C.c_int(), C.c_int()
        shp = (C.c_int64 * 2)()
        check(lib.skel_container_info(self.handle, C.byref(dt), C.byref(nd), shp, C.byref(v)))
        shape = (shp[0],) if nd.value == 1 else (shp[0], shp[1])
        return _DT2NP[dt.value], shape, v.value

    @property
    def shape(self):
        return self.info()[1]

    def stats(self):
        v = [C.c_int64() for _ in range(4)]
        check(lib.skel_container_stats(self.handle, *[C.byref(x) for x in v]))
        return {"h2d": v[0].value, "d2h": v[1].value, "h2d_bytes": v[2].value, "d2h_bytes": v[3].value}

    def host_ptr(self, mode: int = READ, stream=None) -> int:
        p = C.c_void_p()
        check(lib.skel_container_host_ptr(self.handle, mode, _stream(stream), C.byref(p)))
        return p.value

    def device_ptr(self, mode: int = READ, stream=None) -> int:
        p = C.c_void_p()
        check(lib.skel_container_device_ptr(self.handle, mode, _stream(stream), C.byref(p)))
        return p.value

    def mark(self, units: int) -> None:
        check(lib.skel_container_mark(self.handle, units))

    def prefetch(self, unit: int, stream=None) -> None:
        """Starts the copy that makes `unit` valid, on `stream`, without waiting."""
        check(lib.skel_container_prefetch(self.handle, unit, _stream(stream)))

    def to_numpy(self, stream=None) -> np.ndarray:
        """Host read access (lazy device->host copy), returned as a copy."""
        dt, shape, _ = self.info()
        n = int(np.prod(shape))
        p = self.host_ptr(READ, stream)
        buf = (C.c_char * (n * np.dtype(dt).itemsize)).from_address(p) if n else b""
        return np.frombuffer(bytes(buf), dtype=dt).reshape(shape).copy()

    def close(self) -> None:
        if self.handle is not None and self.handle.value:
            if self._views:
                raise SkelError(_lib.ERR_INVALID_ARG, "container still has live views")
            check(lib.skel_container_destroy(self.handle))
            if self._parent is not None:
                self._parent._views -= 1
        self.handle = None
        self._keep = []

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value and not self._views:
                lib.skel_container_destroy(self.handle)
                if self._parent is not None:
                    self._parent._views -= 1
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _handles(cs: Sequence[Container | None]):
    arr = (C.c_void_p * max(1, len(cs)))()
    for i, c in enumerate(cs):
        arr[i] = None if c is None else c.handle.value
    return arr


def _fn(name) -> int:
    return name if isinstance(name, int) else FN[name]


def _params(p):
    p = list(p or [])
    return (C.c_double * max(1, len(p)))(*p), len(p)


def _weights(w):
    if w is None:
        return None, 0
    w = np.ascontiguousarray(w, dtype=np.float32).ravel()
    return w.ctypes.data_as(C.POINTER(C.c_float)), w.size, w


# -------------------------------------------------------- skeleton calls ---
def skel_map(fn, ins: Sequence[Container], out: Container, params=(), stream=None) -> None:
    p, n = _params(params)
    check(lib.skel_map(_fn(fn), p, n, _handles(ins), len(ins), out.handle, _stream(stream)))


def skel_reduce(op, x: Container, result_dev: Container | None = None, host: bool = True, stream=None):
    dt = x.info()[0]
    res = np.zeros(1, dtype=dt)
    check(lib.skel_reduce(_fn(op), x.handle, C.c_void_p(res.ctypes.data) if host else None,
                          None if result_dev is None else result_dev.handle, _stream(stream)))
    return res[0] if host else None


def skel_mapreduce(map_fn, red_op, ins: Sequence[Container], result_dev: Container | None = None,
                   host: bool = True, stream=None):
    res = np.zeros(1, dtype=np.float32)
    check(lib.skel_mapreduce(_fn(map_fn), _fn(red_op), _handles(ins), len(ins),
                             C.c_void_p(res.ctypes.data) if host else None,
                             None if result_dev is None else result_dev.handle, _stream(stream)))
    return res[0] if host else None


def skel_scan(op, inclusive: bool, x: Container, out: Container, stream=None) -> None:
    check(lib.skel_scan(_fn(op), int(inclusive), x.handle, out.handle, _stream(stream)))


def skel_scan_noalloc(op, inclusive: bool, x, out, stream=None) -> None:
    """Allocation-free scan of a contiguous 1D CUDA tensor (float32 or int32)
    into `out` (same dtype and length); see skel_scan_noalloc in skel.h."""
    torch = _torch()
    dt = {torch.float32: F32, torch.int32: I32}[x.dtype]
    if out.dtype != x.dtype or out.numel() != x.numel() or not x.is_contiguous() or not out.is_contiguous():
        raise ValueError("skel_scan_noalloc: contiguous tensors of equal dtype and length")
    check(lib.skel_scan_noalloc(_fn(op), int(inclusive), dt, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                x.numel(), _stream(stream)))


def skel_mapoverlap(fn, radius: int, weights, boundary, x: Container, out: Container, stream=None) -> None:
    w = _weights(weights)
    check(lib.skel_mapoverlap(_fn(fn), radius, w[0], w[1], BOUNDARY[boundary] if isinstance(boundary, str) else boundary,
                              x.handle, out.handle, _stream(stream)))


def skel_mapoverlap_chain(fn, weights, boundary, steps: int, x: Container, tmp, out: Container, stream=None) -> None:
    """out = S^steps(x) for the 2D stencil S; tmp (a container of x's shape,
    or None) holds intermediate steps."""
    w = _weights(weights)
    check(lib.skel_mapoverlap_chain(_fn(fn), w[0], w[1], BOUNDARY[boundary] if isinstance(boundary, str) else boundary,
                                    int(steps), x.handle, tmp.handle if tmp is not None else None, out.handle,
                                    _stream(stream)))


def skel_compose_map_stencil_sumsq(map_fn, stencil, x: Container, params=(), weights=None, boundary="clamp",
                                   result_dev: Container | None = None, host: bool = True, stream=None):
    """sum_{i,j} (S map_fn(x))[i,j]^2 as one composed call (Map -> 2D
    MapOverlap -> MapReduce); returns the value when host is True."""
    res = np.zeros(1, dtype=np.float32)
    p, np_ = _params(params)
    w = _weights(weights)
    check(lib.skel_compose_map_stencil_sumsq(_fn(map_fn), p, np_, _fn(stencil), w[0], w[1],
                                             BOUNDARY[boundary] if isinstance(boundary, str) else boundary, x.handle,
                                             C.c_void_p(res.ctypes.data) if host else None,
                                             None if result_dev is None else result_dev.handle, _stream(stream)))
    return res[0] if host else None


def skel_maparray(fn, whole: Container, elem: Container, out: Container, stream=None) -> None:
    check(lib.skel_maparray(_fn(fn), whole.handle, elem.handle, out.handle, _stream(stream)))


def skel_maparray_grid(fn, whole: Container, out: Container, params, stream=None) -> None:
    """MapArray over out's grid positions (fn "coulomb": params = (h, z0))."""
    p = (C.c_double * len(params))(*params)
    check(lib.skel_maparray_grid(_fn(fn), whole.handle, out.handle, p, len(params), _stream(stream)))


def skel_batched(values: Container, offsets: Container, results: Container | None,
                 scan_out: Container | None, inclusive: bool = True, map_fn="sq", red_op="add",
                 scan_op="add", stream=None) -> None:
    check(lib.skel_batched(_fn(map_fn), _fn(red_op), _fn(scan_op), int(inclusive), values.handle,
                           offsets.handle, None if results is None else results.handle,
                           None if scan_out is None else scan_out.handle, _stream(stream)))


class Plan:
    """A batched call captured once into a CUDA graph (skel_batched_plan_create)."""

    def __init__(self, values, offsets, results, scan_out, inclusive=True, map_fn="sq", red_op="add",
                 scan_op="add", stream=None):
        h = C.c_void_p()
        check(lib.skel_batched_plan_create(_fn(map_fn), _fn(red_op), _fn(scan_op), int(inclusive),
                                           values.handle, offsets.handle,
                                           None if results is None else results.handle,
                                           None if scan_out is None else scan_out.handle,
                                           _stream(stream), C.byref(h)))
        self.handle = h
        self._keep = [values, offsets, results, scan_out]

    def launch(self, stream=None) -> None:
        check(lib.skel_plan_launch(self.handle, _stream(stream)))

    def close(self) -> None:
        if self.handle is not None and self.handle.value:
            check(lib.skel_plan_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- backward ---
def skel_map_bwd(fn, ins: Sequence[Container], gout: Container, gins: Sequence[Container | None],
                 params=(), stream=None) -> None:
    p, n = _params(params)
    check(lib.skel_map_bwd(_fn(fn), p, n, _handles(ins), len(ins), gout.handle, _handles(gins), _stream(stream)))


def skel_map_bwd_sum(fn, ins: Sequence[Container], gouts: Sequence[Container], gins: Sequence[Container | None],
                     params=(), stream=None) -> None:
    p, n = _params(params)
    check(lib.skel_map_bwd_sum(_fn(fn), p, n, _handles(ins), len(ins), _handles(gouts), len(gouts), _handles(gins),
                               _stream(stream)))


def skel_reduce_bwd(op, gr: Container | None, gin: Container, gr_host: float | None = None, stream=None) -> None:
    g = None if gr_host is None else C.byref(C.c_float(gr_host))
    check(lib.skel_reduce_bwd(_fn(op), None if gr is None else gr.handle, g, gin.handle, _stream(stream)))


def skel_mapreduce_bwd(map_fn, red_op, ins: Sequence[Container], gr: Container | None,
                       gins: Sequence[Container | None], gr_host: float | None = None, stream=None) -> None:
    g = None if gr_host is None else C.byref(C.c_float(gr_host))
    check(lib.skel_mapreduce_bwd(_fn(map_fn), _fn(red_op), _handles(ins), len(ins),
                                 None if gr is None else gr.handle, g, _handles(gins), _stream(stream)))


def skel_scan_bwd(op, inclusive: bool, gout: Container, gin: Container, stream=None) -> None:
    check(lib.skel_scan_bwd(_fn(op), int(inclusive), gout.handle, gin.handle, _stream(stream)))


def skel_mapoverlap_bwd(fn, radius: int, weights, boundary, gout: Container, gin: Container, stream=None) -> None:
    w = _weights(weights)
    check(lib.skel_mapoverlap_bwd(_fn(fn), radius, w[0], w[1],
                                  BOUNDARY[boundary] if isinstance(boundary, str) else boundary,
                                  gout.handle, gin.handle, _stream(stream)))


# -------------------------------------------------------------- dispatch ---
def skel_load_dispatch_table(path: str | None) -> None:
    check(lib.skel_load_dispatch_table(None if path is None else path.encode()))


def skel_dispatch_set(skeleton, fn, dtype, bucket, radius, residency, variant, block=0, ept=0, tile=0) -> None:
    check(lib.skel_dispatch_set(SK[skeleton] if isinstance(skeleton, str) else skeleton, fn, dtype, bucket,
                                radius, residency, variant, block, ept, tile))


def skel_dispatch_size() -> int:
    return lib.skel_dispatch_size()


def skel_force_variant(skeleton, variant: int, block: int = 0, ept: int = 0, tile: int = 0) -> None:
    check(lib.skel_force_variant(SK[skeleton] if isinstance(skeleton, str) else skeleton, variant, block, ept, tile))


def skel_last_variant(skeleton):
    v = [C.c_int() for _ in range(4)]
    check(lib.skel_last_variant(SK[skeleton] if isinstance(skeleton, str) else skeleton, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def skel_variant_count(skeleton) -> int:
    return lib.skel_variant_count(SK[skeleton] if isinstance(skeleton, str) else skeleton)


def skel_variant_name(skeleton, v: int) -> str:
    return lib.skel_variant_name(SK[skeleton] if isinstance(skeleton, str) else skeleton, v).decode()


def skel_check_device(stream=None) -> None:
    check(lib.skel_check_device(_stream(stream)))


def skel_set_debug(key: int, value: int) -> None:
    check(lib.skel_set_debug(key, value))


def skel_coherence_step(valid: int, unit: int, mode: int):
    nv, tr = C.c_int(), C.c_int()
    check(lib.skel_coherence_step(valid, unit, mode, C.byref(nv), C.byref(tr)))
    return nv.value, tr.value


def skel_version() -> str:
    return lib.skel_version().decode()


# ------------------------------------------------------- measurement probes ---
def skel_probe_empty_launches(count: int, stream=None) -> None:
    check(lib.skel_probe_empty_launches(int(count), _stream(stream)))


def skel_probe_l2_random(table, reads: int, sink, stream=None) -> int:
    """table, sink: float32 CUDA tensors (table length a power of two).
    Returns the number of reads the launch makes."""
    made = C.c_int64()
    check(lib.skel_probe_l2_random(C.c_void_p(table.data_ptr()), table.numel(), int(reads),
                                   C.c_void_p(sink.data_ptr()), C.byref(made), _stream(stream)))
    return made.value


def skel_probe_call_overhead(calls: int, n: int, stream=None):
    """(microseconds per skel_map call, microseconds per bare launch of its kernel)."""
    a, b = C.c_double(), C.c_double()
    check(lib.skel_probe_call_overhead(int(calls), int(n), C.byref(a), C.byref(b), _stream(stream)))
    return a.value, b.value
