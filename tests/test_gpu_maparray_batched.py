"""Parity of MapArray (gather, rowdot) and of the batched uneven instances
(persistent launch and its CUDA-graph plan) against the oracle."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import (SUM_REL, assert_prefix_close, dev_empty, dev_tensor, forced, skel, to_np, wrap)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant,ept", [(0, 0), (1, 0), (2, 2), (2, 4), (2, 8)])
@pytest.mark.parametrize("m,n", [(1, 1), (7, 5), (1000, 4099), (1 << 16, 1 << 20), (3, 100_003)])
def test_gather(variant, ept, m, n):
    import torch
    sk = skel()
    A = syn.uniform_f32(syn.SEED_X, m)
    idx = syn.uniform_int(syn.SEED_IDX, n, -5, m + 5)          # includes out-of-range indices (clamped)
    dout = dev_empty((n,), torch.float32)
    with forced("maparray", variant, 0, ept):
        sk.skel_maparray("gather", wrap(dev_tensor(A)), wrap(dev_tensor(idx)), wrap(dout))
    assert np.array_equal(to_np(dout).astype(np.float64), oracle.gather_f32(A, idx))   # a copy: exact


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (37, 64), (1000, 1000), (64, 65536), (4096, 4096), (5, 1 << 20),
                                 (2, 3_000_001), (3, 0)])
def test_rowdot(variant, n, m):
    import torch
    sk = skel()
    A = syn.uniform_f32(syn.SEED_X, m)
    M = syn.uniform_f32(syn.SEED_MAT, n * m).reshape(n, m)
    dout = dev_empty((n,), torch.float32)
    with forced("maparray", variant):
        sk.skel_maparray("rowdot", wrap(dev_tensor(A)), wrap(dev_tensor(M)), wrap(dout))
    ref, ab = oracle.rowdot_f32(A, M)
    err = np.abs(to_np(dout).astype(np.float64) - ref)
    assert np.all(err <= SUM_REL * ab), float((err / np.maximum(ab, 1e-30)).max())


def batched_inputs(B, seed=syn.SEED_BATCH_LEN, lo=64, hi=1 << 20, extra=None):
    lens = syn.loguniform_lengths(seed, B, lo, hi)
    if extra is not None:
        lens = np.concatenate([lens, np.asarray(extra, np.int64)])
    off = syn.csr_offsets(lens)
    v = syn.uniform_f32(syn.SEED_BATCH_VAL, int(off[-1]))
    return lens, off, v


def check_batched(v, off, res, scan, inclusive):
    sumsq, ref, ab = oracle.batched_f32(v, off, inclusive)
    B = len(off) - 1
    if res is not None:
        for b in range(B):
            lo, hi = off[b], off[b + 1]
            absq = float(np.sum(v[lo:hi].astype(np.float64) ** 2))
            assert abs(float(res[b]) - sumsq[b]) <= SUM_REL * absq + 1e-30, (b, res[b], sumsq[b])
    if scan is not None:
        assert_prefix_close(scan, ref, ab, "batched scan")


@pytest.mark.parametrize("variant,ept,tile", [(0, 4, 0), (1, 4, 0), (0, 2, 0), (0, 8, 0), (2, 4, 0), (1, 8, 0), (3, 4, 0),
                                              (4, 4, 0), (4, 8, 0), (5, 4, 0), (5, 8, 0), (6, 4, 0), (6, 4, 1), (7, 4, 0),
                                              (7, 4, 1)])
@pytest.mark.parametrize("inclusive", [True, False])
def test_batched_small_mixed(variant, ept, tile, inclusive):
    """Empty, tiny, unaligned and multi-tile instances mixed (for the flat
    variants' tiles of 4096, 24576 and 32768 elements: instances that cross
    one and two tile boundaries, a start exactly on a 32768-element boundary,
    and trailing empties)."""
    import torch
    sk = skel()
    lens = np.array([0, 1, 3, 4, 5, 0, 64, 4095, 4096, 4097, 13, 20000, 0, 1, 70001, 2, 28690,   # next starts at 4 x 32768
                     3, 65536, 0, 0], np.int64)
    off = syn.csr_offsets(lens)
    v = syn.uniform_f32(syn.SEED_BATCH_VAL, int(off[-1]))
    res = torch.full((len(lens),), -7.0, device="cuda")
    sc = torch.full((int(off[-1]),), -7.0, device="cuda")
    with forced("batched", variant, 0, ept, tile):
        sk.skel_batched(wrap(dev_tensor(v)), wrap(dev_tensor(off)), wrap(res), wrap(sc), inclusive)
    sk.skel_check_device()
    check_batched(v, off, to_np(res), to_np(sc), inclusive)


@pytest.mark.parametrize("variant,tile", [(6, 0), (6, 1), (7, 0), (7, 1)])
@pytest.mark.parametrize("inclusive", [True, False])
def test_batched_flat_tile_boundaries(variant, tile, inclusive):
    """The flat variants when instances start exactly on tile boundaries
    (122880 = 5 x 24576 = 30 x 4096, 110592 = 27 x 4096) and when the array
    is a whole number of tiles (no partial tile)."""
    import torch
    sk = skel()
    for lens in ([0, 110592, 12288, 0], [110592, 12288, 7, 0, 1]):
        lens = np.array(lens, np.int64)
        off = syn.csr_offsets(lens)
        v = syn.uniform_f32(syn.SEED_BATCH_VAL, int(off[-1]))
        res = torch.full((len(lens),), -7.0, device="cuda")
        sc = torch.full((int(off[-1]),), -7.0, device="cuda")
        with forced("batched", variant, 0, 4, tile):
            sk.skel_batched(wrap(dev_tensor(v)), wrap(dev_tensor(off)), wrap(res), wrap(sc), inclusive)
        sk.skel_check_device()
        check_batched(v, off, to_np(res), to_np(sc), inclusive)


@pytest.mark.parametrize("variant", [0, 3, 5, 6, 7])
def test_batched_only_reduce_and_only_scan(variant):
    import torch
    sk = skel()
    sk.skel_force_variant("batched", variant)
    try:
        _only_reduce_only_scan(sk, torch)
    finally:
        sk.skel_force_variant("batched", -1)


def _only_reduce_only_scan(sk, torch):
    lens, off, v = batched_inputs(300, hi=1 << 16)
    res = torch.zeros(len(lens), device="cuda")
    sc = torch.zeros(int(off[-1]), device="cuda")
    cv, co = wrap(dev_tensor(v)), wrap(dev_tensor(off))
    sk.skel_batched(cv, co, wrap(res), None, True)
    sk.skel_batched(cv, co, None, wrap(sc), True)
    check_batched(v, off, to_np(res), to_np(sc), True)


@pytest.mark.parametrize("variant", [0, 3, 5, 6, 7])
def test_batched_full_workload_and_graph_plan(variant):
    """4096 instances, log-uniform lengths in [64, 2^20] (~4.4e8 elements):
    direct call, captured plan replayed twice, and per-instance calls on a
    sample of instances all agree with the oracle."""
    import torch
    sk = skel()
    sk.skel_force_variant("batched", variant)
    try:
        _full_workload(sk, torch)
    finally:
        sk.skel_force_variant("batched", -1)


def _full_workload(sk, torch):
    lens, off, v = batched_inputs(4096)
    dv, doff = dev_tensor(v), dev_tensor(off)
    res = torch.zeros(len(lens), device="cuda")
    sc = torch.zeros(int(off[-1]), device="cuda")
    cv, co, cr, cs = wrap(dv), wrap(doff), wrap(res), wrap(sc)
    sk.skel_batched(cv, co, cr, cs, True)
    sk.skel_check_device()
    r1, s1 = to_np(res), to_np(sc)
    check_batched(v, off, r1, s1, True)
    plan = sk.Plan(cv, co, cr, cs, True)
    for _ in range(2):
        res.zero_()
        sc.zero_()
        plan.launch()
        torch.cuda.synchronize()
        check_batched(v, off, to_np(res), to_np(sc), True)
    plan.close()
    # per-instance skeleton calls on views (the one-launch-per-instance path)
    for b in [0, 1, 17, 1000, 4095]:
        lo, hi = int(off[b]), int(off[b + 1])
        view = cv.view(lo, (hi - lo,))
        out = torch.empty(hi - lo, device="cuda")
        q = sk.skel_mapreduce("sq", "add", [view])
        sk.skel_scan("add", True, view, wrap(out))
        ref, ab = oracle.scan_f32(v[lo:hi], True)
        assert_prefix_close(to_np(out), ref, ab, f"instance {b}")
        absq = float(np.sum(v[lo:hi].astype(np.float64) ** 2))
        assert abs(float(q) - oracle.mapreduce_f32("sq", v[lo:hi])[0]) <= SUM_REL * absq
        view.close()


@pytest.mark.parametrize("variant", [-1, 5, 6, 7])
def test_batched_rejects_bad_offsets(variant):
    import torch
    sk = skel()
    v = torch.zeros(100, device="cuda")
    off = torch.tensor([0, 50, 40, 100], dtype=torch.int64, device="cuda")   # decreasing
    res = torch.zeros(3, device="cuda")
    sc = torch.zeros(100, device="cuda")
    sk.skel_force_variant("batched", variant)
    try:
        sk.skel_batched(wrap(v), wrap(off), wrap(res), wrap(sc), True)
    finally:
        sk.skel_force_variant("batched", -1)
    with pytest.raises(sk.SkelError):
        sk.skel_check_device()
    sk.skel_check_device()   # the status was cleared by the previous check
