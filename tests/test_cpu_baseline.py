"""The parallel float32 CPU baseline (timed by the benchmark beside the GPU)
computes the same skeleton calls: checked against the float64 oracle with
several threads.  Its float32 sums run sequentially within each thread's
chunk, so their rounding bound is the sequential one: depth * 2^-24 times
the sum of |terms| (depth = the longest chain of float32 additions)."""
import math

import numpy as np
import pytest

import cpu_baseline as cb
import oracle
import synthetic as syn

EPS = 2.0 ** -24
T = 4            # threads


def test_host_cpu_reports_model_and_cores():
    h = cb.host_cpu()
    assert h["model"] and h["cores_affinity"] >= 1 and h["cores_online"] >= h["cores_affinity"]


@pytest.mark.parametrize("n", [7, 5000, 100_003])
def test_map_reduce_dot(n):
    x, y = syn.uniform_f32(1, n), syn.uniform_f32(2, n)
    assert np.max(np.abs(cb.map_axpy(x, y, 2.5, nthreads=T) - oracle.map_f32("axpy", x, y, a=2.5))) <= 1e-6
    depth = -(-n // T) + T
    ref, ab = oracle.reduce_f32("add", x)
    assert abs(cb.reduce_sum(x, nthreads=T) - ref) <= depth * EPS * ab
    assert cb.reduce_max(x, nthreads=T) == oracle.reduce_f32("max", x)[0]
    ref, ab = oracle.mapreduce_f32("mul", x, y)
    assert abs(cb.dot(x, y, nthreads=T) - ref) <= 2 * depth * EPS * ab


@pytest.mark.parametrize("n", [1, 4099, 100_003])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scans(n, inclusive):
    xi = syn.uniform_int(3, n, 0, 100)
    assert np.array_equal(cb.scan_i32(xi, inclusive, nthreads=T), oracle.scan_i32(xi, inclusive).astype(np.int32))
    x = syn.uniform_f32(4, n)
    ref, ab = oracle.scan_f32(x, inclusive)
    depth = -(-n // T) + T
    assert np.all(np.abs(cb.scan_f32(x, inclusive, nthreads=T) - ref) <= depth * EPS * ab)
    refb, abb = oracle.scan_bwd_f32(x, True)
    assert np.all(np.abs(cb.scan_bwd_f32(x, nthreads=T) - refb) <= depth * EPS * abb)


def test_int32_scan_wraps():
    x = np.full(70_000, 2 ** 30, np.int32)
    got = cb.scan_i32(x, True, nthreads=T)
    assert np.array_equal(got, oracle.scan_i32(x, True).astype(np.int32))


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 1), (64, 100), (300, 257)])
@pytest.mark.parametrize("kind", ["5pt", "9pt"])
def test_stencils_and_adjoint(shape, kind):
    x = syn.uniform_f32(5, shape[0] * shape[1], 0.0, 1.0).reshape(shape)
    w = oracle.stencil_weights(kind)
    assert np.max(np.abs(cb.stencil2d(x, w, nthreads=T) - oracle.mapoverlap2d_f32(x, 1, w, "clamp"))) <= 1e-6
    assert np.max(np.abs(cb.stencil2d_bwd(x, w, nthreads=T) - oracle.mapoverlap2d_bwd_f32(x, 1, w, "clamp"))) <= 1e-6


@pytest.mark.parametrize("n,r", [(3, 2), (10_000, 8), (100_003, 16)])
def test_stencil1d(n, r):
    x = syn.uniform_f32(6, n)
    w = (np.array([math.comb(2 * r, k) for k in range(2 * r + 1)], np.float64) / 4 ** r).astype(np.float32)
    assert np.max(np.abs(cb.stencil1d(x, r, w, nthreads=T) - oracle.mapoverlap1d_f32(x, r, w, "clamp"))) <= 1e-6


def test_maparray_and_tanh_bwd():
    m = 1024
    A = syn.uniform_f32(7, m)
    M = syn.uniform_f32(8, 64 * m).reshape(64, m)
    ref, ab = oracle.rowdot_f32(A, M)
    assert np.all(np.abs(cb.rowdot(A, M, nthreads=T) - ref) <= m * EPS * ab)
    idx = syn.uniform_int(9, 50_000, -5, m + 5)
    assert np.array_equal(cb.gather(A, idx, nthreads=T), oracle.gather_f32(A, idx).astype(np.float32))
    x, g = syn.uniform_f32(10, 9999, -3, 3), syn.uniform_f32(11, 9999)
    assert np.max(np.abs(cb.map_tanh_bwd(x, g, nthreads=T) - oracle.map_bwd_f32("tanh", g, x)[0])) <= 1e-6


def test_batched():
    lens = syn.loguniform_lengths(12, 40, 1, 5000)
    lens[3] = 0
    off = syn.csr_offsets(lens)
    v = syn.uniform_f32(13, int(off[-1]))
    res, scan = cb.batched(v, off, nthreads=T)
    rres, rscan = oracle.batched_f32(v, off, True)[:2]
    for b in range(40):
        a, e = int(off[b]), int(off[b + 1])
        seg = v[a:e].astype(np.float64)
        d = e - a
        assert abs(res[b] - rres[b]) <= 2 * d * EPS * float((seg * seg).sum()) + 1e-30
        assert np.all(np.abs(scan[a:e] - rscan[a:e]) <= d * EPS * np.cumsum(np.abs(seg)))
