"""Smart containers on the GPU (Sec. IV lazy copying): transfer counts
against the plain protocol model, stale copies never read, cross-stream
ordering, views, and the library-owned storage through torch's allocator."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from oracle import coherence as coh
from helpers import assert_elem_close, skel

pytestmark = pytest.mark.gpu


def test_stencil_chain_copies_once_each_way():
    """Ten chained stencil calls ping-pong between two containers; the host
    copy is read once at the end: one H2D and one D2H in total."""
    sk = skel()
    side = 512
    x = syn.uniform_f32(syn.SEED_GRID, side * side, 0.0, 1.0).reshape(side, side)
    a = sk.Container.from_host(x.copy())
    b = sk.Container.empty((side, side))
    w = oracle.stencil_weights("9pt")
    ref = x.astype(np.float32)
    for k in range(10):
        src, dst = (a, b) if k % 2 == 0 else (b, a)
        sk.skel_mapoverlap("stencil9", 1, None, "clamp", src, dst)
        ref = oracle.mapoverlap2d_f32(ref, 1, w, "clamp").astype(np.float32)   # per-call oracle on float32 input
    out = a.to_numpy()
    assert a.stats()["h2d"] == 1 and a.stats()["d2h"] == 1
    assert b.stats()["h2d"] == 0 and b.stats()["d2h"] == 0
    assert_elem_close(out, ref.astype(np.float64), "chain", atol=2e-6)


def test_random_access_sequences_match_protocol_model():
    sk = skel()
    rng = np.random.default_rng(5)
    n = 1000
    for trial in range(20):
        a = sk.Container.from_host(np.zeros(n, np.float32), valid=False)
        tmp = sk.Container.empty((n,))
        model = coh.Model()
        for op in rng.integers(0, 5, size=12):
            if op == 0:      # host write
                a.host_ptr(sk.WRITE)
                model.access(coh.HOST, coh.WRITE)
            elif op == 1:    # host read
                a.host_ptr(sk.READ)
                model.access(coh.HOST, coh.READ)
            elif op == 2:    # device read (a skeleton reads a)
                sk.skel_map("copy", [a], tmp)
                model.access(coh.DEVICE, coh.READ)
            elif op == 3:    # device write (a skeleton writes a)
                sk.skel_map("copy", [tmp], a)
                model.access(coh.DEVICE, coh.WRITE)
            else:            # device read-write (in place)
                sk.skel_map("scale", [a], a, [1.0])
                model.access(coh.DEVICE, coh.READWRITE)
            st = a.stats()
            assert (st["h2d"], st["d2h"]) == (model.h2d, model.d2h), trial
            assert a.info()[2] == model.valid
        a.close()
        tmp.close()


def test_host_write_invalidates_device_copy():
    sk = skel()
    n = 4096
    h = np.arange(n, dtype=np.float32)
    c = sk.Container.from_host(h)
    out = sk.Container.empty((n,))
    sk.skel_map("scale", [c], out, [2.0])
    assert np.array_equal(out.to_numpy(), 2 * h)
    import ctypes
    p = c.host_ptr(sk.WRITE)                 # host takes the only valid copy
    arr = np.ctypeslib.as_array((ctypes.c_float * n).from_address(p))
    arr[:] = -1.0
    sk.skel_map("scale", [c], out, [2.0])    # must copy the new host data
    assert np.all(out.to_numpy() == -2.0)
    assert c.stats()["h2d"] == 2


def test_cross_stream_ordering():
    import torch
    sk = skel()
    n = 1 << 24
    x = torch.from_numpy(syn.uniform_f32(3, n)).cuda()
    a = sk.Container.empty((n,))
    b = sk.Container.empty((n,))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    cx = sk.Container.from_tensor(x)
    sk.skel_map("scale", [cx], a, [3.0], stream=s1)       # writes a on s1
    sk.skel_map("scale", [a], b, [0.5], stream=s2)        # reads a on s2: must wait for s1
    got = b.to_numpy(stream=s2)
    assert np.array_equal(got, (x.cpu().numpy() * np.float32(3.0)) * np.float32(0.5))


def test_views_share_state_and_data():
    sk = skel()
    n = 10_000
    h = syn.uniform_f32(4, n)
    c = sk.Container.from_host(h.copy())
    v = c.view(1000, (2000,))
    out = sk.Container.empty((2000,))
    sk.skel_map("scale", [v], out, [2.0])
    assert np.array_equal(out.to_numpy(), 2 * h[1000:3000])
    sk.skel_map("scale", [out], v, [0.5])                 # writes through the view: device-only now
    assert c.info()[2] == sk.UNIT_DEVICE
    full = c.to_numpy()
    assert np.array_equal(full[1000:3000], h[1000:3000]) and np.array_equal(full[:1000], h[:1000])
    v.close()
    c.close()


def test_library_owned_storage_through_torch_allocator():
    import torch
    sk = skel()
    sk.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        n = 1 << 20
        c = sk.Container.from_host(syn.uniform_f32(5, n))
        out = sk.Container.empty((n,))
        sk.skel_map("sq", [c], out)
        assert torch.cuda.memory_allocated() >= before + 2 * 4 * n
        ref = oracle.map_f32("sq", syn.uniform_f32(5, n))
        assert_elem_close(out.to_numpy(), ref, "sq")
        c.close()
        out.close()
        sk.lib.skel_release_cached()
    finally:
        sk.use_torch_allocator(False)


def test_residency_enters_dispatch_key():
    """A call whose input still lives on the host looks up the residency-1
    entry of the table (falling back to residency 0 when untuned)."""
    sk = skel()
    n = 1 << 16
    sk.skel_load_dispatch_table(None)
    sk.skel_dispatch_set("map", 8, 0, 8, 0, 1, 0, 256, 0, 0)   # COPY, host-resident input -> scalar
    sk.skel_dispatch_set("map", 8, 0, 8, 0, 0, 2, 256, 1, 0)   # COPY, device-resident -> vec4_hint
    try:
        c = sk.Container.from_host(np.ones(n, np.float32))
        out = sk.Container.empty((n,))
        sk.skel_map("copy", [c], out)
        assert sk.skel_last_variant("map")[0] == 0
        sk.skel_map("copy", [c], out)                          # now device-valid
        assert sk.skel_last_variant("map")[0] == 2
    finally:
        sk.skel_load_dispatch_table(None)


def test_prefetch_both_directions_overlaps_and_counts():
    """Prefetch copies on their own streams; the skeleton on the current
    stream and the host read order after them; each copy happens once."""
    import torch
    sk = skel()
    n = 1 << 22
    x = syn.uniform_f32(syn.SEED_X, n)
    y = syn.uniform_f32(syn.SEED_Y, n)
    cx, cy = sk.Container.from_host(x.copy()), sk.Container.from_host(y.copy())
    out = sk.Container.empty((n,))
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    cx.prefetch(sk.UNIT_DEVICE, s_in)
    cy.prefetch(sk.UNIT_DEVICE, s_in)
    cy.prefetch(sk.UNIT_DEVICE, s_in)                  # already on its way: no second copy
    sk.skel_map("axpy", [cx, cy], out, [2.5])
    out.prefetch(sk.UNIT_HOST, s_out)
    got = out.to_numpy()
    assert_elem_close(got, oracle.map_f32("axpy", x, y, 2.5), "axpy after prefetch")
    assert cx.stats()["h2d"] == 1 and cy.stats()["h2d"] == 1
    assert out.stats()["d2h"] == 1                      # the host read found the prefetched copy
    out.prefetch(sk.UNIT_HOST, s_out)                   # valid already: nothing to do
    assert out.stats()["d2h"] == 1
    # a later device write after the prefetch waits for it (write-after-read)
    sk.skel_map("scale", [cx], out, [0.5])
    assert_elem_close(out.to_numpy(), oracle.map_f32("scale", x, None, 0.5), "write after prefetch")
    for c in (cx, cy, out):
        c.close()


def test_prefetch_rejects_bad_unit():
    sk = skel()
    c = sk.Container.from_host(np.zeros(16, np.float32))
    with pytest.raises(sk.SkelError):
        c.prefetch(3)
    c.close()
