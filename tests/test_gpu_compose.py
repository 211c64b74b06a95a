"""Parity of the composed chain Map -> MapOverlap -> MapReduce(sq, +) as one
call, per-call and fused variants, against the float64 oracle.

Tolerance: |gpu - oracle| <= 2^-18 * B, B = sum_p (sum_taps |w| |t|)^2 from
the oracle.  A float32 evaluation rounds t = f(x) (at most 2 ulp for tanhf,
1 for the others), each stencil output over its 9 taps (at most 9 roundings,
each relative to sum_taps |w||t|), squares it, and sums the squares over a
tree of depth well under 16: about (2 * (9 + 2) + 16) * 2^-24 * B < 2^-18.7 * B
in the worst case."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import dev_tensor, forced, skel, to_np, wrap

pytestmark = pytest.mark.gpu

TOL = 2.0 ** -18
MAPS = [("copy", 0.0), ("sq", 0.0), ("scale", 2.5), ("tanh", 0.0)]
VARIANTS = [(0, 0), (1, 0), (1, 1), (1, 2)]   # (variant, tile)
GENERAL_W = syn.uniform_f32(70, 9, -1.0, 1.0)


def weights_for(kind):
    if kind == "general":
        return "stencil9", GENERAL_W
    return kind, None


def ref_weights(kind):
    if kind == "general":
        return GENERAL_W.reshape(3, 3)
    return oracle.stencil_weights("5pt" if kind == "stencil5" else "9pt")


def check(gpu, ref, bound, what):
    assert abs(float(gpu) - ref) <= TOL * bound + 1e-30, \
        f"{what}: |gpu - oracle| = {abs(float(gpu) - ref):.3e} > 2^-18 * B = {TOL * bound:.3e}"


@pytest.mark.parametrize("variant,tile", VARIANTS)
@pytest.mark.parametrize("fn,a", MAPS)
@pytest.mark.parametrize("kind", ["stencil5", "stencil9", "general"])
@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("shape", [(1, 4), (3, 8), (33, 100), (130, 516)])
def test_chain_small(variant, tile, fn, a, kind, boundary, shape):
    sk = skel()
    x = syn.uniform_f32(71 + shape[0], shape[0] * shape[1]).reshape(shape)
    stencil, w = weights_for(kind)
    with forced("compose", variant, 0, 0, tile):
        got = sk.skel_compose_map_stencil_sumsq(fn, stencil, wrap(dev_tensor(x)), [a] if fn == "scale" else (),
                                                w, boundary)
        assert sk.skel_last_variant("compose")[0] == variant
    ref, bound = oracle.chain_map_stencil_sumsq_f32(fn, x, 1, ref_weights(kind), boundary, a)
    check(got, ref, bound, f"{fn} {kind} {boundary} {shape} v{variant}")


def test_chain_device_result_and_empty():
    import torch
    sk = skel()
    x = syn.uniform_f32(80, 64 * 128).reshape(64, 128)
    r = torch.full((1,), 7.0, device="cuda")
    for v in (0, 1):
        with forced("compose", v):
            assert sk.skel_compose_map_stencil_sumsq("tanh", "stencil9", wrap(dev_tensor(x)), result_dev=wrap(r),
                                                     host=False) is None
        ref, bound = oracle.chain_map_stencil_sumsq_f32("tanh", x, 1, oracle.stencil_weights("9pt"), "clamp")
        check(to_np(r)[0], ref, bound, f"device result v{v}")
        e = wrap(torch.empty((0, 8), device="cuda"))
        with forced("compose", v):
            assert sk.skel_compose_map_stencil_sumsq("copy", "stencil5", e) == 0.0


def test_fused_refuses_unaligned_rows_and_table_falls_back():
    sk = skel()
    x = syn.uniform_f32(81, 9 * 7).reshape(9, 7)            # cols % 4 != 0
    ref, bound = oracle.chain_map_stencil_sumsq_f32("sq", x, 1, oracle.stencil_weights("9pt"), "zero")
    with forced("compose", 1):
        with pytest.raises(sk.SkelError) as e:
            sk.skel_compose_map_stencil_sumsq("sq", "stencil9", wrap(dev_tensor(x)), boundary="zero")
        assert e.value.code == -4
    sk.skel_dispatch_set("compose", sk.FN["stencil9"], sk.F32, 0, 1, 0, 1)   # the table picks fused
    try:
        got = sk.skel_compose_map_stencil_sumsq("sq", "stencil9", wrap(dev_tensor(x)), boundary="zero")
        assert sk.skel_last_variant("compose")[0] == 0                     # ... and falls back
        check(got, ref, bound, "fallback")
    finally:
        sk.skel_load_dispatch_table(None)


def test_chain_rejects_bad_arguments():
    import torch
    sk = skel()
    x = wrap(torch.zeros((8, 8), device="cuda"))
    with pytest.raises(sk.SkelError):
        sk.skel_compose_map_stencil_sumsq("axpy", "stencil9", x)        # a two-input map
    with pytest.raises(sk.SkelError):
        sk.skel_compose_map_stencil_sumsq("scale", "stencil9", x)       # SCALE without its parameter
    with pytest.raises(sk.SkelError):
        sk.skel_compose_map_stencil_sumsq("copy", "stencil1d", x)       # 2D stencils only
    with pytest.raises(sk.SkelError):
        sk.skel_compose_map_stencil_sumsq("copy", "stencil9", wrap(torch.zeros(64, device="cuda")))   # 2D input
    with pytest.raises(sk.SkelError):
        sk.skel_compose_map_stencil_sumsq("copy", "stencil9", x, weights=np.ones(5, np.float32))


@pytest.mark.parametrize("variant,tile", [(0, 0), (1, 0), (1, 2)])
def test_chain_8192sq(variant, tile):
    """The composed-loss shape: tanh, 9-point clamp stencil, 8192 x 8192."""
    sk = skel()
    side = 8192
    x = syn.uniform_f32(syn.SEED_GRAD, side * side).reshape(side, side)
    with forced("compose", variant, 0, 0, tile):
        got = sk.skel_compose_map_stencil_sumsq("tanh", "stencil9", wrap(dev_tensor(x)))
    ref, bound = oracle.chain_map_stencil_sumsq_f32("tanh", x, 1, oracle.stencil_weights("9pt"), "clamp")
    check(got, ref, bound, f"8192^2 v{variant}")
