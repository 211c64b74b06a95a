"""Parity at the benchmark's full sizes, in its launch configuration: every
call of the benchmark step at n = 2^28 (grids 16384^2, rowdot 16384 x 16384,
gather from 2^20 values), dispatched through the committed GB300 execution
plan table exactly as the benchmark runs it, against the oracle on the whole
output.  (The batched call at its full 4096-instance size is covered in
test_gpu_maparray_batched.)"""
import os

import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import SUM_REL, assert_elem_close, assert_prefix_close, assert_sum_close, skel, to_np, wrap

pytestmark = pytest.mark.gpu

N = 1 << 28
SIDE = 1 << 14
TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1405_2915_gb300",
                     "dispatch_gb300.tbl")


@pytest.fixture(scope="module")
def sk():
    s = skel()
    if os.path.exists(TABLE):
        s.skel_load_dispatch_table(TABLE)
    yield s
    s.skel_load_dispatch_table(None)


def dev(a):
    import torch
    return torch.from_numpy(a).cuda()


def empty(shape, dtype=None):
    import torch
    return torch.empty(shape, dtype=dtype or torch.float32, device="cuda")


def test_full_map_axpy_and_tanh_bwd(sk):
    x = syn.uniform_f32(syn.SEED_X, N)
    y = syn.uniform_f32(syn.SEED_Y, N)
    dx, dy, o = dev(x), dev(y), empty(N)
    sk.skel_map("axpy", [wrap(dx), wrap(dy)], wrap(o), [2.5])
    assert_elem_close(to_np(o), oracle.map_f32("axpy", x, y, 2.5), "axpy 2^28")
    # tanh adjoint at input x with incoming gradient y: y * (1 - tanh(x)^2)
    sk.skel_map_bwd("tanh", [wrap(dx)], wrap(dy), [wrap(o)])
    gx, _ = oracle.map_bwd_f32("tanh", y, x)
    assert_elem_close(to_np(o), gx, "tanh bwd 2^28")


def test_full_reduce_and_dot(sk):
    import torch
    x = syn.uniform_f32(syn.SEED_X, N)
    y = syn.uniform_f32(syn.SEED_Y, N)
    cx, cy = wrap(dev(x)), wrap(dev(y))
    r = torch.zeros(1, device="cuda")
    sk.skel_reduce("add", cx, wrap(r), host=False)
    v, ab = oracle.reduce_f32("add", x)
    assert_sum_close(float(to_np(r)[0]), v, ab, "sum 2^28")
    sk.skel_reduce("max", cx, wrap(r), host=False)
    assert float(to_np(r)[0]) == oracle.reduce_f32("max", x)[0]
    sk.skel_mapreduce("mul", "add", [cx, cy], wrap(r), host=False)
    v, ab = oracle.mapreduce_f32("mul", x, y)
    assert_sum_close(float(to_np(r)[0]), v, ab, "dot 2^28")


def test_full_scan_i32_inclusive_exact(sk):
    import torch
    x = syn.uniform_int(syn.SEED_INT, N, 0, 100)
    o = empty(N, torch.int32)
    sk.skel_scan("add", True, wrap(dev(x)), wrap(o))
    ref = oracle.scan_i32(x, True).astype(np.int32)   # int64 result modulo 2^32
    assert np.array_equal(to_np(o), ref)


def test_full_scan_f32_exclusive_and_reverse(sk):
    x = syn.uniform_f32(syn.SEED_X, N)
    dx, o = dev(x), empty(N)
    sk.skel_scan("add", False, wrap(dx), wrap(o))
    ref, ab = oracle.scan_f32(x, False)
    assert_prefix_close(to_np(o), ref, ab, "exclusive scan 2^28")
    del ref, ab
    sk.skel_scan_bwd("add", True, wrap(dx), wrap(o))
    ref, ab = oracle.scan_bwd_f32(x, True)
    assert_prefix_close(to_np(o), ref, ab, "reverse scan 2^28")


@pytest.mark.parametrize("kind", ["stencil9", "stencil5"])
def test_full_mapoverlap2d(sk, kind):
    g = syn.uniform_f32(syn.SEED_GRID, N, 0.0, 1.0).reshape(SIDE, SIDE)
    dg, o = dev(g), empty((SIDE, SIDE))
    sk.skel_mapoverlap(kind, 1, None, "clamp", wrap(dg), wrap(o))
    w = oracle.stencil_weights("9pt" if kind == "stencil9" else "5pt")
    assert_elem_close(to_np(o), oracle.mapoverlap2d_f32(g, 1, w, "clamp"), f"{kind} 16384^2")
    if kind == "stencil9":
        sk.skel_mapoverlap_bwd(kind, 1, None, "clamp", wrap(dg), wrap(o))
        assert_elem_close(to_np(o), oracle.mapoverlap2d_bwd_f32(g, 1, w, "clamp"), "9pt adjoint 16384^2")


def test_full_mapoverlap1d_r8(sk):
    import math
    x = syn.uniform_f32(syn.SEED_X, N)
    o = empty(N)
    sk.skel_mapoverlap("stencil1d", 8, None, "clamp", wrap(dev(x)), wrap(o))
    w = (np.array([math.comb(16, k) for k in range(17)], np.float64) / 4 ** 8).astype(np.float32)
    assert_elem_close(to_np(o), oracle.mapoverlap1d_f32(x, 8, w, "clamp"), "1D r=8 2^28")


def test_full_maparray(sk):
    m = SIDE
    A = syn.uniform_f32(syn.SEED_X + 7, m)
    M = syn.uniform_f32(syn.SEED_MAT, N).reshape(N // m, m)
    rd = empty(N // m)
    sk.skel_maparray("rowdot", wrap(dev(A)), wrap(dev(M)), wrap(rd))
    ref, ab = oracle.rowdot_f32(A, M)
    err = np.abs(to_np(rd).astype(np.float64) - ref)
    assert np.all(err <= SUM_REL * ab)
    del M
    Ag = syn.uniform_f32(syn.SEED_X + 8, 1 << 20)
    idx = syn.uniform_int(syn.SEED_IDX, N, 0, (1 << 20) - 1)
    o = empty(N)
    sk.skel_maparray("gather", wrap(dev(Ag)), wrap(dev(idx)), wrap(o))
    assert np.array_equal(to_np(o).astype(np.float64), oracle.gather_f32(Ag, idx))   # a copy: exact
