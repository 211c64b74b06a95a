"""Degenerate inputs through the dispatched calls: empty containers for every
skeleton (reduce returns its identity, the others leave nothing to do),
batches of empty instances, and one-element grids."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import assert_elem_close, dev_empty, dev_tensor, skel, to_np, wrap

pytestmark = pytest.mark.gpu


def test_empty_containers_every_skeleton():
    import torch
    sk = skel()
    e = lambda dt=torch.float32: wrap(torch.empty(0, dtype=dt, device="cuda"))
    sk.skel_map("axpy", [e(), e()], e(), [2.5])
    assert sk.skel_reduce("add", e()) == 0.0
    assert sk.skel_reduce("max", e()) == -np.inf
    assert sk.skel_reduce("add", e(torch.int32)) == 0
    assert sk.skel_reduce("max", e(torch.int32)) == np.iinfo(np.int32).min
    assert sk.skel_mapreduce("mul", "add", [e(), e()]) == 0.0
    sk.skel_scan("add", True, e(), e())
    sk.skel_scan("add", False, e(torch.int32), e(torch.int32))
    sk.skel_scan_bwd("add", True, e(), e())
    sk.skel_mapoverlap("stencil1d", 4, None, "clamp", e(), e())
    g0 = lambda: wrap(torch.empty((0, 16), device="cuda"))
    sk.skel_mapoverlap("stencil9", 1, None, "clamp", g0(), g0())
    sk.skel_mapoverlap_chain("stencil9", None, "clamp", 3, g0(), g0(), g0())
    sk.skel_maparray("gather", wrap(dev_tensor(np.ones(4, np.float32))), e(torch.int32), e())
    sk.skel_maparray("rowdot", wrap(dev_tensor(np.ones(8, np.float32))),
                     wrap(torch.empty((0, 8), device="cuda")), e())
    sk.skel_check_device()


@pytest.mark.parametrize("variant", [-1, 0, 3, 5])
def test_batched_only_empty_instances(variant):
    import torch
    sk = skel()
    off = np.zeros(6, np.int64)                      # five empty instances
    res = torch.full((5,), 7.0, device="cuda")
    v = torch.empty(0, device="cuda")
    sk.skel_force_variant("batched", variant)
    try:
        sk.skel_batched(wrap(v), wrap(dev_tensor(off)), wrap(res), wrap(torch.empty(0, device="cuda")), True)
    finally:
        sk.skel_force_variant("batched", -1)
    sk.skel_check_device()
    assert np.array_equal(to_np(res), np.zeros(5, np.float32))   # the sum of squares of nothing


@pytest.mark.parametrize("kind", ["stencil5", "stencil9"])
@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
def test_one_cell_grids(kind, boundary):
    import torch
    sk = skel()
    x = np.array([[0.625]], np.float32)
    w = oracle.stencil_weights("5pt" if kind == "stencil5" else "9pt")
    out = dev_empty((1, 1), torch.float32)
    sk.skel_mapoverlap(kind, 1, None, boundary, wrap(dev_tensor(x)), wrap(out))
    assert_elem_close(to_np(out), oracle.mapoverlap2d_f32(x, 1, w, boundary), f"1x1 {kind} {boundary}")
    tmp = dev_empty((1, 1), torch.float32)
    sk.skel_mapoverlap_chain(kind, None, boundary, 5, wrap(dev_tensor(x)), wrap(tmp), wrap(out))
    assert_elem_close(to_np(out), oracle.mapoverlap2d_chain_f32(x, 1, w, boundary, 5), f"1x1 chain {boundary}")


def test_single_element_scans_and_reduces():
    import torch
    sk = skel()
    for dt, x in ((torch.float32, syn.uniform_f32(3, 1)), (torch.int32, np.array([-5], np.int32))):
        dx = wrap(dev_tensor(x))
        o = dev_empty((1,), dt)
        sk.skel_scan("add", True, dx, wrap(o))
        assert to_np(o)[0] == x[0]
        sk.skel_scan("add", False, dx, wrap(o))
        assert to_np(o)[0] == 0
        assert sk.skel_reduce("max", dx) == x[0]
