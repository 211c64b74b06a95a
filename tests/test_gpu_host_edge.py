"""The host edge (Sec. IV lazy copying, keyed by residency): Map, Reduce and
MapReduce calls on inputs valid only in host memory, through the whole copy,
the chunked copy pipeline and direct reads of pinned host memory.  Results
against the oracle, the containers' valid units and transfer counts after
each variant, the refusals (pageable memory, views, an output aliasing a
host-only input) and their fallback, and ordering against earlier work on
the device copy."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import assert_elem_close, assert_sum_close, forced, skel, to_np

pytestmark = pytest.mark.gpu

CHUNK = 1 << 21                          # float32 elements per chunk at tile 0 (8 MiB)
SIZES = [0, 1, 5, 4097, CHUNK, CHUNK + 3, 3 * CHUNK + 5]
EDGES = [(0, 0), (1, 0), (1, 1), (2, 0)]   # (variant, tile)
HOST, DEV = 1, 2


def pinned(a: np.ndarray) -> np.ndarray:
    """A numpy view of a copy of `a` in page-locked host memory (kept alive
    by the returned array's base)."""
    import torch
    if a.size == 0:
        return np.empty(0, a.dtype)
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    v = t.numpy()
    assert v.ctypes.data == t.data_ptr()
    return v


def host_container(a):
    sk = skel()
    return sk.Container.from_host(pinned(a))


def check_units(c, variant):
    _, _, valid = c.info()
    st = c.stats()
    if variant == 2:
        assert valid == HOST and st["h2d"] == 0
    else:
        assert valid == HOST | DEV and st["h2d"] == 1


@pytest.mark.parametrize("variant,tile", EDGES)
@pytest.mark.parametrize("n", SIZES)
def test_map_axpy_and_tanh(variant, tile, n):
    import torch
    sk = skel()
    x = syn.uniform_f32(syn.SEED_X + n, n)
    y = syn.uniform_f32(syn.SEED_Y + n, n)
    cx, cy = host_container(x), host_container(y)
    out = torch.empty(n, device="cuda")
    co = sk.Container.from_tensor(out)
    with forced("edge", variant, 0, 0, tile):
        sk.skel_map("axpy", [cx, cy], co, [2.5])
        assert sk.skel_last_variant("edge")[0] == variant
    assert_elem_close(to_np(out), oracle.map_f32("axpy", x, y, 2.5), f"axpy edge {variant} n={n}")
    check_units(cx, variant)
    check_units(cy, variant)
    # a second call on the now device-valid inputs (chunked, copy) takes the
    # ordinary path and copies nothing more
    cx.mark(HOST)
    with forced("edge", variant, 0, 0, tile):
        sk.skel_map("tanh", [cx], co)
    assert_elem_close(to_np(out), oracle.map_f32("tanh", x, None, 0.0), f"tanh edge {variant} n={n}")


@pytest.mark.parametrize("variant,tile", EDGES)
@pytest.mark.parametrize("n", SIZES)
def test_reduce_and_mapreduce(variant, tile, n):
    import torch
    sk = skel()
    x = syn.uniform_f32(syn.SEED_X + 3 * n, n)
    y = syn.uniform_f32(syn.SEED_Y + 3 * n, n)
    xi = syn.uniform_int(syn.SEED_INT + n, n, 0, 100)
    with forced("edge", variant, 0, 0, tile):
        cx = host_container(x)
        v, ab = oracle.reduce_f32("add", x)
        assert_sum_close(sk.skel_reduce("add", cx), v, ab, f"sum edge {variant} n={n}")
        check_units(cx, variant)
        cx.mark(HOST)
        assert sk.skel_reduce("max", cx) == (oracle.reduce_f32("max", x)[0] if n else -np.inf)
        ci = host_container(xi)
        assert sk.skel_reduce("add", ci) == int(np.int64(oracle.reduce_i32("add", xi)).astype(np.int32))
        cx.mark(HOST)
        cy = host_container(y)
        r = torch.zeros(1, device="cuda")
        sk.skel_mapreduce("mul", "add", [cx, cy], sk.Container.from_tensor(r), host=False)
        v, ab = oracle.mapreduce_f32("mul", x, y)
        assert_sum_close(float(to_np(r)[0]), v, ab, f"dot edge {variant} n={n}")
        assert sk.skel_last_variant("edge")[0] == variant
        cy.mark(HOST)
        v, ab = oracle.mapreduce_f32("sq", y, None)
        assert_sum_close(sk.skel_mapreduce("sq", "add", [cy]), v, ab, f"sumsq edge {variant} n={n}")


def test_mixed_residency_and_shared_input():
    """One host-only input next to a device-valid one; the same host-only
    container passed twice (copied once)."""
    import torch
    sk = skel()
    n = 2 * CHUNK + 7
    x = syn.uniform_f32(21, n)
    y = syn.uniform_f32(22, n)
    for variant, tile in EDGES[1:]:
        cx = host_container(x)
        cy = sk.Container.from_tensor(torch.from_numpy(y).cuda())
        out = torch.empty(n, device="cuda")
        with forced("edge", variant, 0, 0, tile):
            sk.skel_map("mul", [cx, cy], sk.Container.from_tensor(out))
            assert_elem_close(to_np(out), oracle.map_f32("mul", x, y, 0.0), f"mixed {variant}")
            cz = host_container(x)
            sk.skel_map("mul", [cz, cz], sk.Container.from_tensor(out))
            assert_elem_close(to_np(out), oracle.map_f32("mul", x, x, 0.0), f"shared {variant}")
            assert cz.stats()["h2d"] == (0 if variant == 2 else 1)


def test_refusals_and_fallback():
    import torch
    sk = skel()
    n = 4096
    x = syn.uniform_f32(31, n)
    out = torch.empty(n, device="cuda")
    co = sk.Container.from_tensor(out)
    pageable = sk.Container.from_host(x.copy())
    with forced("edge", 2):                         # direct reads need pinned memory
        with pytest.raises(sk.SkelError) as e:
            sk.skel_map("tanh", [pageable], co)
        assert e.value.code == -4
    big = host_container(np.concatenate([x, x]))
    view = big.view(n, (n,))
    with forced("edge", 1):                         # the chunked copy keeps whole storages only
        with pytest.raises(sk.SkelError) as e:
            sk.skel_map("tanh", [view], co)
        assert e.value.code == -4
    del view
    inplace = host_container(x)
    with forced("edge", 1):                         # an output that is a host-only input
        with pytest.raises(sk.SkelError) as e:
            sk.skel_map("scale", [inplace], inplace, [2.0])
        assert e.value.code == -4
    # through the table (not forced) the same calls fall back to the whole copy
    sk.skel_dispatch_set("edge", sk.SK["map"], sk.F32, 6, 0, 1, 2)
    try:
        sk.skel_map("tanh", [pageable], co)
        assert sk.skel_last_variant("edge")[0] == 0
        assert_elem_close(to_np(out), oracle.map_f32("tanh", x, None, 0.0), "fallback")
        sk.skel_map("scale", [inplace], inplace, [2.0])
        assert sk.skel_last_variant("edge")[0] == 0
        assert np.array_equal(inplace.to_numpy(), (x * np.float32(2.0)).astype(np.float32))
        sk.skel_map("tanh", [host_container(x)], co)   # pinned: the table's direct variant runs
        assert sk.skel_last_variant("edge")[0] == 2
    finally:
        sk.skel_load_dispatch_table(None)


@pytest.mark.parametrize("variant", [1, 2])
def test_ordering_after_earlier_device_work(variant):
    """Calls still queued on the stream read a container's device copy when
    its host copy gets new values and the next call reads it through the
    edge: the queued calls must see the old values (the chunked copy into
    the device copy waits for them), the new call the new ones."""
    import torch
    sk = skel()
    n = 4 * CHUNK
    old = syn.uniform_f32(41, n)
    new = syn.uniform_f32(42, n)
    buf = pinned(old)
    cx = sk.Container.from_host(buf)
    o1 = torch.empty(n, device="cuda")
    c1 = sk.Container.from_tensor(o1)
    sk.skel_map("scale", [cx], c1, [3.0])     # the whole lazy copy of the old values
    torch.cuda.current_stream().synchronize()  # ... has landed: the host copy is free to change
    for _ in range(8):                         # queued reads of the device copy
        sk.skel_map("scale", [cx], c1, [3.0])
    buf[:] = new                               # nothing queued reads the host copy
    cx.mark(HOST)
    o2 = torch.empty(n, device="cuda")
    with forced("edge", variant):
        sk.skel_map("scale", [cx], sk.Container.from_tensor(o2), [3.0])
    assert np.array_equal(to_np(o1), (old * np.float32(3.0)).astype(np.float32))
    assert np.array_equal(to_np(o2), (new * np.float32(3.0)).astype(np.float32))


def test_second_touch_copies_a_reused_input():
    """With the table choosing direct reads, an input read in place once and
    then read again (its host copy unchanged) is copied whole instead, so the
    calls after it find it on the device; writing its host copy starts over."""
    import torch
    sk = skel()
    n = 1 << 16
    x = syn.uniform_f32(51, n)
    cx = host_container(x)
    out = torch.empty(n, device="cuda")
    co = sk.Container.from_tensor(out)
    sk.skel_dispatch_set("edge", sk.SK["map"], sk.F32, 8, 0, 1, 2)
    try:
        sk.skel_map("tanh", [cx], co)
        assert sk.skel_last_variant("edge")[0] == 2 and cx.stats()["h2d"] == 0
        sk.skel_map("sq", [cx], co)                     # second touch: the whole copy
        assert sk.skel_last_variant("edge")[0] == 0 and cx.stats()["h2d"] == 1
        assert_elem_close(to_np(out), oracle.map_f32("sq", x, None, 0.0), "second touch")
        sk.skel_map("tanh", [cx], co)                   # on the device now: no transfer
        assert cx.stats()["h2d"] == 1
        cx.mark(HOST)                                   # the host copy is new again
        sk.skel_map("tanh", [cx], co)
        assert sk.skel_last_variant("edge")[0] == 2 and cx.stats()["h2d"] == 1
        assert_elem_close(to_np(out), oracle.map_f32("tanh", x, None, 0.0), "after mark")
    finally:
        sk.skel_load_dispatch_table(None)
