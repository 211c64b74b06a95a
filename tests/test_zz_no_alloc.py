"""The allocation-free scan entry point (skel_scan_noalloc), for callers that
cannot allocate device memory (a fixed budget owned by the host, or a
latency-critical path that must avoid allocator locks and the synchronisation
cudaMalloc/cudaFree can cause).  Its scratch is a static device array inside
libskel.so, so this test checks it against the regular skel_scan and the
oracle on two calls in a row (the second call reuses what the first left in
the array), over enough calls that the look-back tag kept in the array wraps,
that a bounded wait that gives up is reported by skel_check_device, and that
sizes beyond the array's capacity are refused.  It is collected last so that
it also runs after every other test in the same process."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import SUM_REL, dev_empty, dev_tensor, skel, to_np, wrap

pytestmark = pytest.mark.gpu


def _call(sk, inclusive, dt_code, x, out, n):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    return sk.lib.skel_scan_noalloc(0, int(inclusive), dt_code, C.c_void_p(x.data_ptr()),
                                    C.c_void_p(out.data_ptr()), n, C.c_void_p(stream))


@pytest.mark.parametrize("dtype", ["int32", "float32"])
@pytest.mark.parametrize("inclusive", [True, False])
@pytest.mark.parametrize("n", [1, 4097, 3_000_001])
def test_noalloc_scan_matches_skel_scan_on_two_calls(dtype, inclusive, n):
    import torch
    sk = skel()
    tdt = torch.int32 if dtype == "int32" else torch.float32
    dt_code = 1 if dtype == "int32" else 0
    x = syn.uniform_int(900 + n, n, 0, 100) if dtype == "int32" else syn.uniform_f32(900 + n, n)
    dx = dev_tensor(x)
    ref = dev_empty((n,), tdt)
    sk.skel_scan("add", inclusive, wrap(dx), wrap(ref))          # the existing entry point
    ref_h = to_np(ref)
    for call in range(2):
        out = dev_empty((n,), tdt)
        out.fill_(-1)
        rc = _call(sk, inclusive, dt_code, dx, out, n)
        assert rc == 0, sk.lib.skel_last_error().decode()
        got = to_np(out)
        if dtype == "int32":
            assert np.array_equal(got, ref_h), f"call {call}"
            assert np.array_equal(got, oracle.scan_i32(x, inclusive).astype(np.int32)), f"call {call}"
        else:
            # the existing entry point's output and the oracle's values, each
            # within the scan bound 2^-20 * sum of |x| over the prefix
            val, ab = oracle.scan_f32(x, inclusive)
            for what, want in (("oracle", val), ("skel_scan", ref_h.astype(np.float64))):
                err = np.abs(got.astype(np.float64) - want)
                bound = SUM_REL * ab
                assert np.all(err <= bound), f"call {call} vs {what}: max excess {float(np.max(err - bound))}"
    sk.skel_check_device()


def test_noalloc_scan_many_calls_wrap_the_tag():
    """300 calls alternating two inputs and both scan kinds: the tag kept in
    the static array passes its 255-call wrap (words cleared on the device)
    and the tile ticket resets after every call."""
    import torch
    sk = skel()
    n = 3 * 4096 + 17
    xs = [syn.uniform_int(31, n, 0, 100), syn.uniform_int(32, n, 0, 100)]
    dxs = [dev_tensor(x) for x in xs]
    want = {(k, incl): oracle.scan_i32(xs[k], incl).astype(np.int32) for k in (0, 1) for incl in (True, False)}
    out = dev_empty((n,), torch.int32)
    for call in range(300):
        k, incl = call % 2, (call // 2) % 2 == 0
        out.fill_(-1)
        assert _call(sk, incl, 1, dxs[k], out, n) == 0, sk.lib.skel_last_error().decode()
        got = to_np(out)
        assert np.array_equal(got, want[(k, incl)]), f"call {call}"
    sk.skel_check_device()


def test_noalloc_scan_timeout_is_reported():
    """A tile that never publishes (test hook) makes its successors' bounded
    waits run out; skel_check_device reports SKEL_ERR_TIMEOUT and clears it,
    and the next call is correct."""
    import torch
    sk = skel()
    n = 20 * 4096 + 5
    x = syn.uniform_int(41, n, 0, 100)
    dx = dev_tensor(x)
    out = dev_empty((n,), torch.int32)
    sk.skel_check_device()
    sk.skel_set_debug(2, 50_000)        # 50 ms wait limit
    sk.skel_set_debug(1, 3)             # tile 3 never publishes
    try:
        assert _call(sk, True, 1, dx, out, n) == 0
        with pytest.raises(sk.SkelError) as e:
            sk.skel_check_device()
        assert e.value.code == -7
    finally:
        sk.skel_set_debug(1, -1)
        sk.skel_set_debug(2, 2_000_000)
    sk.skel_check_device()              # cleared
    assert _call(sk, True, 1, dx, out, n) == 0
    sk.skel_check_device()
    assert np.array_equal(to_np(out), oracle.scan_i32(x, True).astype(np.int32))


def test_noalloc_scan_refuses_sizes_beyond_its_static_scratch():
    import torch
    sk = skel()
    x = torch.zeros(8, device="cuda")
    too_big = (1 << 27) + 1
    rc = sk.lib.skel_scan_noalloc(0, 1, 0, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr() + 4096),
                                  too_big, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -2
    assert "SKEL_SCAN_NOALLOC_MAX_N" in sk.lib.skel_last_error().decode()


def test_noalloc_scan_python_wrapper_and_allocator_untouched():
    import torch
    sk = skel()
    n = 1 << 20
    x = dev_tensor(syn.uniform_int(7, n, 0, 100))
    out = torch.empty_like(x)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    sk.skel_scan_noalloc("add", True, x, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    assert np.array_equal(to_np(out), oracle.scan_i32(to_np(x), True).astype(np.int32))
