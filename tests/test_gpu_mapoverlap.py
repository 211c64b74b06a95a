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


# ------------------------------------------------ chains of 2D calls --
CHAIN_CASES = [((1, 1), 3), ((5, 7), 2), ((33, 130), 5), ((130, 257), 10), ((300, 520), 4), ((64, 128), 1)]


def run_chain(sk, kind, boundary, steps, x, with_tmp=True):
    import torch
    out = dev_empty(x.shape, torch.float32)
    tmp = wrap(dev_empty(x.shape, torch.float32)) if with_tmp else None
    sk.skel_mapoverlap_chain(kind, None, boundary, steps, wrap(dev_tensor(x)), tmp, wrap(out))
    return to_np(out)


# every steps-per-pass factor the tuner may choose (1..8) and the per-call variant
@pytest.mark.parametrize("variant,k", [(0, 0)] + [(1, k) for k in range(1, 9)])
@pytest.mark.parametrize("shape,steps", CHAIN_CASES)
@pytest.mark.parametrize("kind", ["stencil5", "stencil9"])
@pytest.mark.parametrize("boundary", ["clamp", "zero"])
def test_mapoverlap_chain_matches_oracle(variant, k, shape, steps, kind, boundary):
    """out = S^steps(x) against the float64 chain; each step adds at most a
    few float32 roundings of values <= 1 (the stencils average)."""
    sk = skel()
    x = syn.uniform_f32(syn.SEED_GRID + steps, shape[0] * shape[1], 0.0, 1.0).reshape(shape)
    with forced("chain2d", variant, 0, 0, k):
        g = run_chain(sk, kind, boundary, steps, x)
    w = oracle.stencil_weights("5pt" if kind == "stencil5" else "9pt")
    ref = oracle.mapoverlap2d_chain_f32(x, 1, w, boundary, steps)
    assert_elem_close(g, ref, f"chain {kind} {boundary} {shape} x{steps} v{variant} k{k}", atol=1e-6 * steps)


@pytest.mark.parametrize("k", list(range(1, 9)))
@pytest.mark.parametrize("boundary", ["clamp", "zero"])
def test_mapoverlap_chain_time_blocked_is_bitwise_per_call(k, boundary):
    """The fused passes evaluate every cell with the single-step tap order:
    the result equals the chain of single calls bit for bit."""
    sk = skel()
    x = syn.uniform_f32(syn.SEED_GRID, 211 * 390, 0.0, 1.0).reshape(211, 390)
    for kind in ("stencil5", "stencil9"):
        with forced("chain2d", 0):
            a = run_chain(sk, kind, boundary, 7, x)
        with forced("chain2d", 1, 0, 0, k):
            b = run_chain(sk, kind, boundary, 7, x)
        assert np.array_equal(a, b), (kind, boundary, k)


def test_mapoverlap_chain_periodic_falls_back_and_tmp_rules():
    sk = skel()
    x = syn.uniform_f32(syn.SEED_GRID, 40 * 64, 0.0, 1.0).reshape(40, 64)
    w = oracle.stencil_weights("9pt")
    with forced("chain2d", 1, 0, 0, 4):
        with pytest.raises(sk.SkelError):                 # periodic is not time-blocked
            run_chain(sk, "stencil9", "periodic", 3, x)
    g = run_chain(sk, "stencil9", "periodic", 3, x)       # dispatched: falls back to per call
    assert sk.skel_last_variant("chain2d")[0] == 0
    assert_elem_close(g, oracle.mapoverlap2d_chain_f32(x, 1, w, "periodic", 3), "periodic chain", atol=3e-6)
    with forced("chain2d", 0):
        with pytest.raises(sk.SkelError):                 # per call needs tmp for 2+ steps
            run_chain(sk, "stencil9", "clamp", 2, x, with_tmp=False)
    with forced("chain2d", 1, 0, 0, 4):                   # one pass covers 3 steps: no tmp needed
        g = run_chain(sk, "stencil9", "clamp", 3, x, with_tmp=False)
    assert_elem_close(g, oracle.mapoverlap2d_chain_f32(x, 1, w, "clamp", 3), "single pass", atol=3e-6)
