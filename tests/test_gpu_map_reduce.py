"""Parity of Map, Reduce and MapReduce (every variant, forced) against the
CPU oracle at the stated tolerances: map elementwise within 1e-6; float32
sums within 2^-20 * sum |terms|; max and int32 sums bit-exact."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import (assert_elem_close, assert_sum_close, dev_empty, dev_tensor, forced, skel, to_np,
                     wrap)

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 4, 5, 31, 33, 127, 1023, 1025, 4097, 65537, (1 << 20) + 3, 3_000_001]
MAP_CONFIGS = [(0, 256, 0), (1, 256, 1), (1, 128, 2), (1, 256, 4), (2, 256, 1), (2, 512, 4),
               (3, 256, 1), (3, 256, 4)]


@pytest.mark.parametrize("variant,block,ept", MAP_CONFIGS)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("pad", [0, 1])
def test_map_axpy(variant, block, ept, n, pad):
    import torch
    sk = skel()
    x, y = syn.uniform_f32(syn.SEED_X, n), syn.uniform_f32(syn.SEED_Y, n)
    dx, dy = dev_tensor(x, pad), dev_tensor(y, pad)
    dout = dev_empty((n,), torch.float32, pad)
    with forced("map", variant, block, ept):
        sk.skel_map("axpy", [wrap(dx), wrap(dy)], wrap(dout), params=[2.5])
    assert_elem_close(to_np(dout), oracle.map_f32("axpy", x, y, a=2.5), f"axpy n={n}")


@pytest.mark.parametrize("fn", ["add", "sub", "mul", "max", "tanh", "sq", "scale", "copy"])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_map_functors(fn, variant):
    import torch
    sk = skel()
    n = 100_003
    x, y = syn.uniform_f32(11, n, -3.0, 3.0), syn.uniform_f32(12, n)
    nin = 2 if fn in ("add", "sub", "mul", "max") else 1
    ins = [wrap(dev_tensor(x))] + ([wrap(dev_tensor(y))] if nin == 2 else [])
    dout = dev_empty((n,), torch.float32)
    with forced("map", variant, 256, 2 if variant else 0):
        sk.skel_map(fn, ins, wrap(dout), params=[-1.5] if fn == "scale" else [])
    ref = oracle.map_f32(fn, x, y if nin == 2 else None, a=-1.5)
    assert_elem_close(to_np(dout), ref, fn, atol=1e-6 * max(1.0, float(np.abs(ref).max())))


def test_map_in_place_and_mismatched_alignment():
    import torch
    sk = skel()
    n = 10_001
    x, y = syn.uniform_f32(21, n), syn.uniform_f32(22, n)
    dx = dev_tensor(x)
    dy = dev_tensor(y, pad_front=1)     # different offset modulo 16 bytes than dx
    cx = wrap(dx)
    sk.skel_map("axpy", [cx, wrap(dy)], cx, params=[2.5])   # in place; vector variants fall back
    assert_elem_close(to_np(dx), oracle.map_f32("axpy", x, y, a=2.5), "in-place axpy")
    assert sk.skel_last_variant("map")[0] == 0


@pytest.mark.parametrize("variant,block,ept", MAP_CONFIGS)
@pytest.mark.parametrize("same_container", [True, False])
@pytest.mark.parametrize("which", [0, 1])
def test_map_in_place_every_variant(variant, block, ept, same_container, which):
    """out is input `which` at the same alignment (the vector variants apply):
    either the same container, or a second container wrapping the same
    device memory.  Results equal the oracle's for every forced variant."""
    sk = skel()
    n = 1_000_003
    x, y = syn.uniform_f32(23, n), syn.uniform_f32(24, n)
    dx, dy = dev_tensor(x, 1), dev_tensor(y, 1)       # equal offsets modulo 16 bytes
    cx, cy = wrap(dx), wrap(dy)
    target = (dx, cx) if which == 0 else (dy, cy)
    cout = target[1] if same_container else wrap(target[0])
    with forced("map", variant, block, ept):
        sk.skel_map("axpy", [cx, cy], cout, params=[2.5])
        assert sk.skel_last_variant("map")[0] == variant
    assert_elem_close(to_np(target[0]), oracle.map_f32("axpy", x, y, a=2.5), f"in-place axpy into input {which}")


def test_map_partial_overlap_is_rejected():
    import torch
    sk = skel()
    n = 4096
    base = torch.zeros(n + 8, device="cuda")
    a, b = base[:n], base[3:n + 3]                   # two wrapped pointers, 3 elements apart
    ca = wrap(a)
    with pytest.raises(sk.SkelError) as e:
        sk.skel_map("scale", [ca], wrap(b), params=[2.0])
    assert e.value.code == -1
    parent = sk.Container.from_tensor(base)         # views of one container, shifted
    v0, v1 = parent.view(0, (n,)), parent.view(5, (n,))
    with pytest.raises(sk.SkelError) as e:
        sk.skel_map("scale", [v0], v1, params=[2.0])
    assert e.value.code == -1
    v0.close(); v1.close()


def test_map_empty_is_noop():
    import torch
    sk = skel()
    e = torch.empty(0, device="cuda")
    sk.skel_map("axpy", [wrap(e), wrap(e)], wrap(e), params=[2.5])


RED_CONFIGS = [(0, 256, 4), (0, 128, 1), (0, 512, 8), (1, 256, 4), (1, 256, 2), (1, 512, 8),
               (2, 256, 4), (2, 512, 1)]


@pytest.mark.parametrize("variant,block,ept", RED_CONFIGS)
@pytest.mark.parametrize("n", [0] + SIZES)
@pytest.mark.parametrize("pad", [0, 3])
def test_reduce_f32(variant, block, ept, n, pad):
    sk = skel()
    x = syn.uniform_f32(syn.SEED_X + n, n)
    cx = wrap(dev_tensor(x, pad))
    with forced("reduce", variant, block, ept):
        s = sk.skel_reduce("add", cx)
        m = sk.skel_reduce("max", cx)
    ref, ab = oracle.reduce_f32("add", x)
    assert_sum_close(s, ref, ab, f"sum n={n}")
    assert float(m) == oracle.reduce_f32("max", x)[0]


@pytest.mark.parametrize("variant,block,ept", RED_CONFIGS[::2])
@pytest.mark.parametrize("n", [0, 1, 5, 4097, 1 << 20, 3_000_001])
def test_reduce_i32_exact(variant, block, ept, n):
    sk = skel()
    x = syn.uniform_int(syn.SEED_INT + n, n, -(2**31), 2**31 - 1)
    cx = wrap(dev_tensor(x))
    with forced("reduce", variant, block, ept):
        s = sk.skel_reduce("add", cx)
        m = sk.skel_reduce("max", cx)
    assert int(s) == int(np.int64(oracle.reduce_i32("add", x)).astype(np.int32))   # modulo 2^32
    assert int(m) == oracle.reduce_i32("max", x)


def test_reduce_deterministic_and_device_result():
    import torch
    sk = skel()
    n = (1 << 22) + 7
    x = syn.uniform_f32(31, n)
    cx = wrap(dev_tensor(x))
    r = torch.zeros(1, device="cuda")
    cr = wrap(r)
    vals = set()
    for _ in range(20):
        vals.add(float(sk.skel_reduce("add", cx)))
    assert len(vals) == 1
    sk.skel_reduce("add", cx, result_dev=cr, host=False)
    assert float(to_np(r)[0]) in vals


@pytest.mark.parametrize("variant,block,ept", RED_CONFIGS)
@pytest.mark.parametrize("n", [0, 1, 7, 1 << 20, (1 << 20) + 5])
def test_mapreduce_dot_and_sumsq(variant, block, ept, n):
    sk = skel()
    x, y = syn.uniform_f32(syn.SEED_X, n), syn.uniform_f32(syn.SEED_Y, n)
    cx, cy = wrap(dev_tensor(x)), wrap(dev_tensor(y))
    with forced("mapreduce", variant, block, ept):
        d = sk.skel_mapreduce("mul", "add", [cx, cy])
        q = sk.skel_mapreduce("sq", "add", [cx])
    ref, ab = oracle.mapreduce_f32("mul", x, y)
    assert_sum_close(d, ref, ab, f"dot n={n}")
    ref, ab = oracle.mapreduce_f32("sq", x)
    assert_sum_close(q, ref, ab, f"sumsq n={n}")


def test_dot_config_2pow20_default_dispatch():
    """The dot-product workload: two float32 vectors of 2^20, U[-1,1]."""
    sk = skel()
    n = 1 << 20
    x, y = syn.uniform_f32(syn.SEED_X, n), syn.uniform_f32(syn.SEED_Y, n)
    d = sk.skel_mapreduce("mul", "add", [wrap(dev_tensor(x)), wrap(dev_tensor(y))])
    ref, ab = oracle.mapreduce_f32("mul", x, y)
    assert_sum_close(d, ref, ab, "dot 2^20")
