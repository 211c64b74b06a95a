"""Failure detection without a GPU fault: a scan tile that never publishes
makes its successors' bounded look-back waits run out; the kernel records the
status, every launch still finishes, the host reads the status, and the
context stays usable."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import SUM_REL, assert_prefix_close, dev_empty, dev_tensor, forced, skel, to_np, wrap

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [1, 3, 4, 5, 6, 7, 8])   # warp, block, pipelined, wide, warp-specialised, hybrid, re-read
def test_lookback_wait_runs_out_and_is_reported(variant):
    import torch
    sk = skel()
    n = 20 * 40960 + 5                  # at least 20 tiles for every variant (the hybrid's are 40960 elements)
    x = syn.uniform_int(1, n, 0, 100)
    out = dev_empty((n,), torch.int32)
    sk.skel_check_device()
    sk.skel_set_debug(2, 50_000)        # 50 ms wait limit
    sk.skel_set_debug(1, 3)             # tile 3 never publishes
    try:
        with forced("scan", variant):
            sk.skel_scan("add", True, wrap(dev_tensor(x)), wrap(out))
        with pytest.raises(sk.SkelError) as e:
            sk.skel_check_device()
        assert e.value.code == -7
    finally:
        sk.skel_set_debug(1, -1)
        sk.skel_set_debug(2, 2_000_000)
    # the status was cleared and the context works
    sk.skel_check_device()
    with forced("scan", variant):
        sk.skel_scan("add", True, wrap(dev_tensor(x)), wrap(out))
    sk.skel_check_device()
    assert np.array_equal(to_np(out), oracle.scan_i32(x, True).astype(np.int32))


def test_batched_reread_wait_runs_out_and_is_reported():
    """The re-reading batched variant: a tile in the middle of a long
    instance never publishes, the tiles after it that continue the instance
    give up their bounded walks, the status is reported, and the next call
    (hook off) is correct."""
    import torch
    sk = skel()
    lens = np.array([50 * 4096 + 7, 3 * 4096, 20 * 4096 + 1], np.int64)
    off = syn.csr_offsets(lens)
    v = syn.uniform_f32(syn.SEED_BATCH_VAL, int(off[-1]))
    res = torch.zeros(len(lens), device="cuda")
    sc = torch.zeros(int(off[-1]), device="cuda")
    cv, co, cr, cs = wrap(dev_tensor(v)), wrap(dev_tensor(off)), wrap(res), wrap(sc)
    sk.skel_check_device()
    sk.skel_set_debug(2, 50_000)        # 50 ms wait limit
    sk.skel_set_debug(1, 5)             # tile 5 (inside the first instance) never publishes
    try:
        with forced("batched", 7, 0, 4, 0):
            sk.skel_batched(cv, co, cr, cs, True)
        with pytest.raises(sk.SkelError) as e:
            sk.skel_check_device()
        assert e.value.code == -7
    finally:
        sk.skel_set_debug(1, -1)
        sk.skel_set_debug(2, 2_000_000)
    sk.skel_check_device()
    with forced("batched", 7, 0, 4, 0):
        sk.skel_batched(cv, co, cr, cs, True)
    sk.skel_check_device()
    sumsq, ref, ab = oracle.batched_f32(v, off, True)
    assert_prefix_close(to_np(sc), ref, ab, "batched scan after the timeout")
    r = to_np(res)
    for b in range(len(lens)):   # the sum of squares of positive terms: 2^-20 of itself
        assert abs(float(r[b]) - sumsq[b]) <= SUM_REL * sumsq[b], (b, r[b], sumsq[b])


def test_errors_are_reported_not_raised_across_the_abi():
    import torch
    sk = skel()
    a = wrap(torch.zeros(10, device="cuda"))
    b = wrap(torch.zeros(11, device="cuda"))
    with pytest.raises(sk.SkelError) as e:
        sk.skel_map("add", [a, b], a)
    assert e.value.code == -2
    with pytest.raises(sk.SkelError) as e:
        sk.skel_scan("max", True, a, wrap(torch.zeros(10, device="cuda")))
    assert e.value.code == -4
    i = wrap(torch.zeros(10, dtype=torch.int64, device="cuda"))
    with pytest.raises(sk.SkelError) as e:
        sk.skel_reduce("add", i)
    assert e.value.code == -3
