"""Parity of Scan (every variant, forced): int32 bit-exact modulo 2^32;
float32 per element within 2^-20 * sum_{j<=i} |x_j| (the prefix of |x| over
the same index range)."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import assert_prefix_close, dev_empty, dev_tensor, forced, skel, to_np, wrap

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 4, 5, 31, 1023, 1024, 1025, 4095, 4096, 4097, 8193, 65537, (1 << 20) + 3, 3_000_001]
# (variant, ept, tile); variant 5: tile bit 0 publishes the tile aggregate
# early, bit 1 selects 48 KiB tiles; variant 6: tile 0 = four 48 KiB stages,
# 1 = six 32 KiB stages; variant 7: tile 0 = 96 KiB staged + 64 KiB in
# registers, 1 = 64 + 32 KiB, 2 = 64 + 48 KiB, 3 = 96 + 80 KiB; variant 8:
# ring tiles + scanner warps 0 = 6 + 6, 1 = 4 + 8, 2 = 6 + 8, 3 = 5 + 8
SCAN_CONFIGS = [(0, 4, 0), (0, 2, 0), (1, 4, 0), (1, 2, 0), (1, 8, 0), (2, 4, 0), (2, 8, 0), (3, 4, 0), (3, 2, 0),
                (3, 8, 0), (4, 4, 0), (5, 4, 0), (5, 4, 1), (5, 4, 2), (5, 4, 3), (6, 4, 0), (6, 4, 1), (7, 4, 0),
                (7, 4, 1), (7, 4, 2), (7, 4, 3), (8, 4, 0), (8, 4, 1), (8, 4, 2), (8, 4, 3)]


def mod32(a):
    return np.asarray(a, dtype=np.int64).astype(np.int32)


@pytest.mark.parametrize("variant,ept,tile", SCAN_CONFIGS)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("inclusive", [True, False])
@pytest.mark.parametrize("pad", [0, 1])
def test_scan_i32_exact(variant, ept, tile, n, inclusive, pad):
    import torch
    sk = skel()
    x = syn.uniform_int(syn.SEED_INT + n, n, 0, 100)
    dx = dev_tensor(x, pad)
    dout = dev_empty((n,), torch.int32, pad)
    with forced("scan", variant, 0, ept, tile):
        if variant in (4, 5, 6, 7, 8) and pad % 4:
            # bulk copies need 16-byte aligned operands; a forced call does not fall back
            with pytest.raises(sk.SkelError) as e:
                sk.skel_scan("add", inclusive, wrap(dx), wrap(dout))
            assert e.value.code == -4
            return
        sk.skel_scan("add", inclusive, wrap(dx), wrap(dout))
    assert np.array_equal(to_np(dout), mod32(oracle.scan_i32(x, inclusive)))


@pytest.mark.parametrize("variant,ept,tile", SCAN_CONFIGS)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_f32(variant, ept, tile, n, inclusive):
    import torch
    sk = skel()
    x = syn.uniform_f32(syn.SEED_X + n, n)
    dx = dev_tensor(x)
    dout = dev_empty((n,), torch.float32)
    with forced("scan", variant, 0, ept, tile):
        sk.skel_scan("add", inclusive, wrap(dx), wrap(dout))
    ref, ab = oracle.scan_f32(x, inclusive)
    assert_prefix_close(to_np(dout), ref, ab, f"scan f32 n={n} incl={inclusive}")


def test_scan_i32_wraps_modulo_2pow32():
    import torch
    sk = skel()
    n = 100_000
    x = syn.uniform_int(5, n, 2**30, 2**31 - 1)
    dout = dev_empty((n,), torch.int32)
    for variant in (0, 1, 2):
        with forced("scan", variant):
            sk.skel_scan("add", True, wrap(dev_tensor(x)), wrap(dout))
        assert np.array_equal(to_np(dout), mod32(oracle.scan_i32(x, True)))


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("rows,cols", [(1, 1), (5, 1), (3, 5000), (7, 4096), (4, 4097), (64, 1000)])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_rows(variant, rows, cols, inclusive):
    """A 2D container is scanned along each row independently."""
    import torch
    sk = skel()
    x = syn.uniform_f32(41, rows * cols).reshape(rows, cols)
    xi = syn.uniform_int(42, rows * cols, 0, 100).reshape(rows, cols)
    dout = dev_empty((rows, cols), torch.float32)
    douti = dev_empty((rows, cols), torch.int32)
    with forced("scan", variant):
        sk.skel_scan("add", inclusive, wrap(dev_tensor(x)), wrap(dout))
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xi)), wrap(douti))
    g, gi = to_np(dout), to_np(douti)
    for r in range(rows):
        ref, ab = oracle.scan_f32(x[r], inclusive)
        assert_prefix_close(g[r], ref, ab, f"row {r}")
        assert np.array_equal(gi[r], mod32(oracle.scan_i32(xi[r], inclusive)))


@pytest.mark.parametrize("variant,tile", [(1, 0), (6, 0), (6, 1), (7, 0), (7, 1), (8, 0), (8, 1)])
def test_scan_lookback_repeated_runs_identical_int(variant, tile):
    """Races in the look-back (or, for the warp-specialised variant, in the
    hand-over of stages between its roles) would show up as run-to-run
    differences."""
    import torch
    sk = skel()
    n = (1 << 22) + 16
    x = syn.uniform_int(7, n, 0, 100)
    dx = wrap(dev_tensor(x))
    ref = mod32(oracle.scan_i32(x, True))
    dout = dev_empty((n,), torch.int32)
    with forced("scan", variant, 0, 4 if variant == 6 else 0, tile):
        for _ in range(20):
            dout.fill_(-1)
            sk.skel_scan("add", True, dx, wrap(dout))
            assert np.array_equal(to_np(dout), ref)


@pytest.mark.parametrize("variant", [1, 3, 4, 5, 6, 7, 8])
def test_scan_types_interleaved_share_lookback_words(variant):
    """int32 and float32 look-back scans alternate on one stream and reuse the
    same descriptor words; a stale word of one type must never read as a
    published value for the other (tested over many calls and tile counts)."""
    import torch
    sk = skel()
    for k in range(12):
        n = 3_000_001 - 4096 * k
        xi = syn.uniform_int(700 + k, n, 0, 100)
        xf = syn.uniform_f32(800 + k, n)
        oi = dev_empty((n,), torch.int32)
        of = dev_empty((n,), torch.float32)
        with forced("scan", variant):
            sk.skel_scan("add", True, wrap(dev_tensor(xi)), wrap(oi))
            sk.skel_scan("add", k % 2 == 0, wrap(dev_tensor(xf)), wrap(of))
        assert np.array_equal(to_np(oi), mod32(oracle.scan_i32(xi, True)))
        ref, ab = oracle.scan_f32(xf, k % 2 == 0)
        assert_prefix_close(to_np(of), ref, ab, f"interleaved f32 call {k}")


@pytest.mark.parametrize("variant", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("rows,cols", [(3, 5000), (7, 4096), (64, 1000), (2, 12), (3, 40000), (2, 163840), (3, 200000)])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_rows_tma(variant, rows, cols, inclusive):
    """Row-wise scans through the bulk-copy variants (segments of a multiple
    of 4 elements)."""
    import torch
    sk = skel()
    x = syn.uniform_f32(43, rows * cols).reshape(rows, cols)
    dout = dev_empty((rows, cols), torch.float32)
    with forced("scan", variant):
        sk.skel_scan("add", inclusive, wrap(dev_tensor(x)), wrap(dout))
    g = to_np(dout)
    for r in range(rows):
        ref, ab = oracle.scan_f32(x[r], inclusive)
        assert_prefix_close(g[r], ref, ab, f"row {r}")


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_ws_many_ring_turns(tile, inclusive):
    """2^25 + 4 elements: every persistent block of the warp-specialised
    variant goes round its ring of stages several times."""
    import torch
    sk = skel()
    n = (1 << 25) + 4
    xi = syn.uniform_int(900 + tile, n, 0, 100)
    oi = dev_empty((n,), torch.int32)
    xf = syn.uniform_f32(901 + tile, n)
    of = dev_empty((n,), torch.float32)
    with forced("scan", 6, 0, 4, tile):
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xi)), wrap(oi))
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xf)), wrap(of))
    assert np.array_equal(to_np(oi), mod32(oracle.scan_i32(xi, inclusive)))
    ref, ab = oracle.scan_f32(xf, inclusive)
    assert_prefix_close(to_np(of), ref, ab, f"ws f32 2^25 tile={tile}")


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_hybrid_many_tiles_and_ragged_tail(tile, inclusive):
    """The hybrid-staged variant over 2^25 + 3 elements: thousands of tiles in
    flight, a last tile that ends inside its register part, and a last group
    of fewer than four elements."""
    import torch
    sk = skel()
    n = (1 << 25) + 3
    xi = syn.uniform_int(910 + tile, n, 0, 100)
    oi = dev_empty((n,), torch.int32)
    xf = syn.uniform_f32(911 + tile, n)
    of = dev_empty((n,), torch.float32)
    with forced("scan", 7, 0, 4, tile):
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xi)), wrap(oi))
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xf)), wrap(of))
    assert np.array_equal(to_np(oi), mod32(oracle.scan_i32(xi, inclusive)))
    ref, ab = oracle.scan_f32(xf, inclusive)
    assert_prefix_close(to_np(of), ref, ab, f"hybrid f32 2^25+3 tile={tile}")


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_reread_many_tiles_and_ragged_tail(tile, inclusive):
    """The re-reading variant over 2^25 + 3 elements: every persistent block
    goes round its ring of tiles many times, the queue to the scanner warps
    fills, and the last tile is partial with a last group of three."""
    import torch
    sk = skel()
    n = (1 << 25) + 3
    xi = syn.uniform_int(920 + tile, n, 0, 100)
    oi = dev_empty((n,), torch.int32)
    xf = syn.uniform_f32(921 + tile, n)
    of = dev_empty((n,), torch.float32)
    with forced("scan", 8, 0, 4, tile):
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xi)), wrap(oi))
        sk.skel_scan("add", inclusive, wrap(dev_tensor(xf)), wrap(of))
    assert np.array_equal(to_np(oi), mod32(oracle.scan_i32(xi, inclusive)))
    ref, ab = oracle.scan_f32(xf, inclusive)
    assert_prefix_close(to_np(of), ref, ab, f"reread f32 2^25+3 tile={tile}")


@pytest.mark.parametrize("tile", [0, 2])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_reread_rows_and_refusal(tile, inclusive):
    """Row-wise scans through the re-reading variant: rows of whole tiles
    (8192 = 2 x 4096, as in the composed loss), a partial tile per row, and a
    row length that is not a multiple of 4 (refused before any launch; an
    unforced call falls back)."""
    import torch
    sk = skel()
    for rows, cols in [(64, 8192), (5, 12300), (9, 100)]:
        x = syn.uniform_f32(45 + cols, rows * cols).reshape(rows, cols)
        dout = dev_empty((rows, cols), torch.float32)
        with forced("scan", 8, 0, 4, tile):
            sk.skel_scan("add", inclusive, wrap(dev_tensor(x)), wrap(dout))
        g = to_np(dout)
        for r in range(rows):
            ref, ab = oracle.scan_f32(x[r], inclusive)
            assert_prefix_close(g[r], ref, ab, f"row {r} of {rows} x {cols}")
    x = syn.uniform_f32(44, 3 * 4097).reshape(3, 4097)
    dout = dev_empty((3, 4097), torch.float32)
    with forced("scan", 8):
        with pytest.raises(sk.SkelError) as e:
            sk.skel_scan("add", True, wrap(dev_tensor(x)), wrap(dout))
        assert e.value.code == -4
