"""ctypes declarations of every function in include/skel.h.

This module only loads libskel.so and declares argument types; it never
computes anything.  Loading fails loudly when the library has not been
built (there is no other implementation to fall back to).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libskel.so")

# enums of skel.h
F32, I32, I64 = 0, 1, 2
OK, ERR_INVALID_ARG, ERR_SHAPE, ERR_DTYPE, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_TABLE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
FN = {"add": 0, "mul": 1, "max": 2, "axpy": 3, "tanh": 4, "sq": 5, "scale": 6, "sub": 7, "copy": 8,
      "stencil5": 9, "stencil9": 10, "stencil1d": 11, "gather": 12, "rowdot": 13, "coulomb": 14}
BOUNDARY = {"clamp": 0, "zero": 1, "periodic": 2}
READ, WRITE, READWRITE = 1, 2, 3
UNIT_HOST, UNIT_DEVICE = 1, 2
SK = {"map": 0, "reduce": 1, "mapreduce": 2, "scan": 3, "mapoverlap1d": 4, "mapoverlap2d": 5,
      "maparray": 6, "batched": 7, "chain2d": 8, "edge": 9, "compose": 10}

vp, i32, i64, dbl, f32p = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.POINTER(C.c_float)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# name: (restype, argtypes) -- one line per declaration of skel.h
SIGNATURES = {
    "skel_version": (C.c_char_p, []),
    "skel_last_error": (C.c_char_p, []),
    "skel_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
    "skel_release_cached": (i32, []),
    "skel_launch_count": (i64, []),
    "skel_container_create": (i32, [i32, i32, C.POINTER(i64), C.POINTER(vp)]),
    "skel_container_wrap": (i32, [i32, i32, C.POINTER(i64), vp, vp, i32, C.POINTER(vp)]),
    "skel_container_view": (i32, [vp, i64, i32, C.POINTER(i64), C.POINTER(vp)]),
    "skel_container_host_ptr": (i32, [vp, i32, vp, C.POINTER(vp)]),
    "skel_container_device_ptr": (i32, [vp, i32, vp, C.POINTER(vp)]),
    "skel_container_mark": (i32, [vp, i32]),
    "skel_container_prefetch": (i32, [vp, i32, vp]),
    "skel_container_info": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]),
    "skel_container_stats": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
    "skel_container_destroy": (i32, [vp]),
    "skel_coherence_step": (i32, [i32, i32, i32, C.POINTER(i32), C.POINTER(i32)]),
    "skel_map": (i32, [i32, C.POINTER(dbl), i32, C.POINTER(vp), i32, vp, vp]),
    "skel_reduce": (i32, [i32, vp, vp, vp, vp]),
    "skel_mapreduce": (i32, [i32, i32, C.POINTER(vp), i32, vp, vp, vp]),
    "skel_scan": (i32, [i32, i32, vp, vp, vp]),
    "skel_scan_noalloc": (i32, [i32, i32, i32, vp, vp, i64, vp]),
    "skel_mapoverlap": (i32, [i32, i32, f32p, i32, i32, vp, vp, vp]),
    "skel_maparray": (i32, [i32, vp, vp, vp, vp]),
    "skel_mapoverlap_chain": (i32, [i32, f32p, i32, i32, i32, vp, vp, vp, vp]),
    "skel_maparray_grid": (i32, [i32, vp, vp, C.POINTER(dbl), i32, vp]),
    "skel_compose_map_stencil_sumsq": (i32, [i32, C.POINTER(dbl), i32, i32, f32p, i32, i32, vp, vp, vp, vp]),
    "skel_batched": (i32, [i32, i32, i32, i32, vp, vp, vp, vp, vp]),
    "skel_batched_plan_create": (i32, [i32, i32, i32, i32, vp, vp, vp, vp, vp, C.POINTER(vp)]),
    "skel_plan_launch": (i32, [vp, vp]),
    "skel_plan_destroy": (i32, [vp]),
    "skel_map_bwd": (i32, [i32, C.POINTER(dbl), i32, C.POINTER(vp), i32, vp, C.POINTER(vp), vp]),
    "skel_map_bwd_sum": (i32, [i32, C.POINTER(dbl), i32, C.POINTER(vp), i32, C.POINTER(vp), i32, C.POINTER(vp), vp]),
    "skel_reduce_bwd": (i32, [i32, vp, f32p, vp, vp]),
    "skel_mapreduce_bwd": (i32, [i32, i32, C.POINTER(vp), i32, vp, f32p, C.POINTER(vp), vp]),
    "skel_scan_bwd": (i32, [i32, i32, vp, vp, vp]),
    "skel_mapoverlap_bwd": (i32, [i32, i32, f32p, i32, i32, vp, vp, vp]),
    "skel_load_dispatch_table": (i32, [C.c_char_p]),
    "skel_dispatch_set": (i32, [i32] * 10),
    "skel_dispatch_size": (i32, []),
    "skel_force_variant": (i32, [i32, i32, i32, i32, i32]),
    "skel_last_variant": (i32, [i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    "skel_variant_count": (i32, [i32]),
    "skel_variant_name": (C.c_char_p, [i32, i32]),
    "skel_check_device": (i32, [vp]),
    "skel_set_debug": (i32, [i32, i64]),
    "skel_probe_empty_launches": (i32, [i32, vp]),
    "skel_probe_l2_random": (i32, [vp, i64, i64, vp, C.POINTER(i64), vp]),
    "skel_probe_call_overhead": (i32, [i32, i64, C.POINTER(dbl), C.POINTER(dbl), vp]),
}


class SkelError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"skel error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python paper_1405_2915_gb300/build.py` "
                          "(the CUDA library is the only implementation)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib
