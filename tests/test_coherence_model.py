"""Pins of the plain coherence model (Sec. IV, lazy memory copying) to the
transfer counts that the protocol's description fixes by hand."""
from oracle import coherence as coh


def test_chain_of_device_calls_copies_once_each_way():
    """Host fills a container, ten device calls ping-pong between two
    containers, host reads the result: one H2D per operand, one D2H."""
    a, b = coh.Model(), coh.Model()
    a.access(coh.HOST, coh.WRITE)
    for k in range(10):
        src, dst = (a, b) if k % 2 == 0 else (b, a)
        src.access(coh.DEVICE, coh.READ)
        dst.access(coh.DEVICE, coh.WRITE)
    a.access(coh.HOST, coh.READ)
    assert (a.h2d, a.d2h, b.h2d, b.d2h) == (1, 1, 0, 0)


def test_stale_copy_never_read():
    m = coh.Model()
    m.access(coh.HOST, coh.WRITE)
    assert m.access(coh.DEVICE, coh.READ) == coh.H2D
    assert m.access(coh.DEVICE, coh.READ) == coh.NONE          # reuse valid device copy
    m.access(coh.HOST, coh.WRITE)                               # host write invalidates device
    assert m.valid == coh.HOST
    assert m.access(coh.DEVICE, coh.READWRITE) == coh.H2D
    assert m.valid == coh.DEVICE
    assert m.access(coh.HOST, coh.READ) == coh.D2H
    assert m.valid == coh.HOST | coh.DEVICE
    assert m.access(coh.HOST, coh.READ) == coh.NONE


def test_fresh_container_reads_nothing():
    m = coh.Model()
    assert m.access(coh.DEVICE, coh.READ) == coh.NONE
    assert m.access(coh.HOST, coh.READ) == coh.NONE
    assert (m.h2d, m.d2h) == (0, 0)


def test_write_only_access_skips_copy():
    m = coh.Model(coh.HOST)
    assert m.access(coh.DEVICE, coh.WRITE) == coh.NONE
    assert m.valid == coh.DEVICE
    assert m.access(coh.HOST, coh.WRITE) == coh.NONE
    assert m.valid == coh.HOST
