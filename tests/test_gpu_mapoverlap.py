"""Parity of MapOverlap 1D/2D and its adjoint (every variant, forced) against
the oracle: elementwise within 1e-6 (outputs of magnitude <= 1 here), for
clamp, zero and periodic boundaries, ragged and tiny grids."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import assert_elem_close, dev_empty, dev_tensor, forced, skel, to_np, wrap

pytestmark = pytest.mark.gpu

SHAPES_2D = [(1, 4), (1, 1), (3, 5), (4, 4), (7, 12), (33, 36), (129, 260), (300, 1000), (512, 512),
             (1031, 2052)]
BOUNDS = ["clamp", "zero", "periodic"]


def weights(kind):
    return oracle.stencil_weights(kind)


@pytest.mark.parametrize("variant,tile", [(0, 0), (1, 0), (2, 0), (3, 16), (3, 32), (3, 64), (3, 128)])
@pytest.mark.parametrize("shape", SHAPES_2D)
@pytest.mark.parametrize("kind", ["5pt", "9pt"])
@pytest.mark.parametrize("boundary", BOUNDS)
def test_mapoverlap2d(variant, tile, shape, kind, boundary):
    import torch
    sk = skel()
    x = syn.uniform_f32(syn.SEED_GRID, shape[0] * shape[1], 0.0, 1.0).reshape(shape)
    dout = dev_empty(shape, torch.float32)
    fn = "stencil5" if kind == "5pt" else "stencil9"
    with forced("mapoverlap2d", variant, 0, 0, tile):
        if variant != 0 and shape[1] % 4:
            # selectability constraint of the tiled variants; a forced call does not fall back
            with pytest.raises(sk.SkelError) as e:
                sk.skel_mapoverlap(fn, 1, None, boundary, wrap(dev_tensor(x)), wrap(dout))
            assert e.value.code == -4
            return
        sk.skel_mapoverlap(fn, 1, None, boundary, wrap(dev_tensor(x)), wrap(dout))
    ref = oracle.mapoverlap2d_f32(x, 1, weights(kind), boundary)
    assert_elem_close(to_np(dout), ref, f"{kind} {boundary} {shape} v{variant}")


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 4), (2, 8), (5, 4), (64, 68), (257, 516), (3, 1028)])
@pytest.mark.parametrize("boundary", BOUNDS)
def test_mapoverlap2d_general_weights_and_adjoint(variant, shape, boundary):
    import torch
    sk = skel()
    w = syn.uniform_f32(77, 9, -1.0, 1.0).reshape(3, 3)
    x = syn.uniform_f32(78, shape[0] * shape[1]).reshape(shape)
    dout = dev_empty(shape, torch.float32)
    with forced("mapoverlap2d", variant, 0, 0, 32 if variant == 3 else 0):
        sk.skel_mapoverlap("stencil9", 1, w, boundary, wrap(dev_tensor(x)), wrap(dout))
        assert_elem_close(to_np(dout), oracle.mapoverlap2d_f32(x, 1, w, boundary), "forward", atol=3e-6)
        sk.skel_mapoverlap_bwd("stencil9", 1, w, boundary, wrap(dev_tensor(x)), wrap(dout))
    assert_elem_close(to_np(dout), oracle.mapoverlap2d_bwd_f32(x, 1, w, boundary), "adjoint", atol=3e-6)


@pytest.mark.parametrize("kind", ["5pt", "9pt"])
@pytest.mark.parametrize("boundary", BOUNDS)
def test_mapoverlap2d_adjoint_default_weights(kind, boundary):
    import torch
    sk = skel()
    shape = (97, 132)
    g = syn.uniform_f32(79, shape[0] * shape[1]).reshape(shape)
    dout = dev_empty(shape, torch.float32)
    sk.skel_mapoverlap_bwd("stencil5" if kind == "5pt" else "stencil9", 1, None, boundary,
                           wrap(dev_tensor(g)), wrap(dout))
    assert_elem_close(to_np(dout), oracle.mapoverlap2d_bwd_f32(g, 1, weights(kind), boundary), "adjoint")


def test_mapoverlap2d_unaligned_falls_back():
    """cols % 4 != 0: the tiled variants' constraint fails; the call still
    succeeds through a variant without constraints."""
    import torch
    sk = skel()
    shape = (50, 37)
    x = syn.uniform_f32(80, shape[0] * shape[1]).reshape(shape)
    dout = dev_empty(shape, torch.float32)
    sk.skel_dispatch_set("mapoverlap2d", 10, 0, 0, 1, 0, 3, 0, 0, 32)   # ask for column_walk
    try:
        sk.skel_mapoverlap("stencil9", 1, None, "clamp", wrap(dev_tensor(x)), wrap(dout))
    finally:
        sk.skel_load_dispatch_table(None)
    assert_elem_close(to_np(dout), oracle.mapoverlap2d_f32(x, 1, weights("9pt"), "clamp"), "fallback")
    assert sk.skel_last_variant("mapoverlap2d")[0] in (0,)


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("r", [0, 1, 2, 3, 5, 8, 16])
@pytest.mark.parametrize("n", [1, 2, 7, 33, 2048, 2049, 4096 * 3 + 5, 100_003])
@pytest.mark.parametrize("boundary", BOUNDS)
def test_mapoverlap1d(variant, r, n, boundary):
    import torch
    sk = skel()
    x = syn.uniform_f32(90 + r, n)
    w = syn.uniform_f32(91 + r, 2 * r + 1, 0.0, 1.0)
    w = (w / w.astype(np.float64).sum()).astype(np.float32)
    dout = dev_empty((n,), torch.float32)
    with forced("mapoverlap1d", variant):
        sk.skel_mapoverlap("stencil1d", r, w, boundary, wrap(dev_tensor(x)), wrap(dout))
        assert_elem_close(to_np(dout), oracle.mapoverlap1d_f32(x, r, w, boundary), f"1d r={r} n={n}")
        sk.skel_mapoverlap_bwd("stencil1d", r, w, boundary, wrap(dev_tensor(x)), wrap(dout))
    assert_elem_close(to_np(dout), oracle.mapoverlap1d_bwd_f32(x, r, w, boundary), f"1d adjoint r={r} n={n}")


def test_mapoverlap1d_bulk_needs_alignment():
    """The bulk-copy variant refuses a 4-byte-offset input when forced; the
    dispatched call falls back to a variant without the constraint."""
    import torch
    sk = skel()
    n, r = 50_001, 3
    x = syn.uniform_f32(96, n + 1)
    w = syn.uniform_f32(97, 2 * r + 1, 0.0, 1.0)
    dx = dev_tensor(x)
    dout = dev_empty((n,), torch.float32)
    cx = wrap(dx)
    view = cx.view(1, (n,))
    with forced("mapoverlap1d", 2):
        with pytest.raises(sk.SkelError):
            sk.skel_mapoverlap("stencil1d", r, w, "clamp", view, wrap(dout))
    sk.skel_mapoverlap("stencil1d", r, w, "clamp", view, wrap(dout))
    assert_elem_close(to_np(dout), oracle.mapoverlap1d_f32(x[1:], r, w, "clamp"), "offset input")
    view.close()


def test_mapoverlap1d_default_binomial_weights():
    import math
    import torch
    sk = skel()
    n, r = 5000, 4
    x = syn.uniform_f32(95, n)
    dout = dev_empty((n,), torch.float32)
    sk.skel_mapoverlap("stencil1d", r, None, "clamp", wrap(dev_tensor(x)), wrap(dout))
    w = np.array([math.comb(2 * r, k) for k in range(2 * r + 1)], np.float64) / 4 ** r
    assert_elem_close(to_np(dout), oracle.mapoverlap1d_f32(x, r, w.astype(np.float32), "clamp"), "binomial")


def test_mapoverlap_rejects_aliasing_and_bad_radius():
    import torch
    sk = skel()
    t = torch.zeros(64, 64, device="cuda")
    c = wrap(t)
    with pytest.raises(sk.SkelError):
        sk.skel_mapoverlap("stencil9", 1, None, "clamp", c, c)
    with pytest.raises(sk.SkelError):
        sk.skel_mapoverlap("stencil9", 2, None, "clamp", c, wrap(torch.zeros(64, 64, device="cuda")))
    v = torch.zeros(100, device="cuda")
    with pytest.raises(sk.SkelError):
        sk.skel_mapoverlap("stencil1d", 17, None, "clamp", wrap(v), wrap(torch.zeros(100, device="cuda")))
