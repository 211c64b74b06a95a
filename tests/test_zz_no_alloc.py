"""The allocation-free scan entry point (skel_scan_noalloc), for callers that
cannot allocate device memory (a fixed budget owned by the host, or a
latency-critical path that must avoid allocator locks and the synchronisation
cudaMalloc/cudaFree can cause).  Its scratch is a static device array inside
libskel.so, so this test checks it against the regular skel_scan on two calls
in a row (the second call reuses what the first left in the array), and that
sizes beyond the array's capacity are refused.  It is collected last so that
it also runs after every other test in the same process."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import SUM_REL, dev_empty, dev_tensor, skel, to_np, wrap

pytestmark = pytest.mark.gpu


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
        stream = torch.cuda.current_stream().cuda_stream
        rc = sk.lib.skel_scan_noalloc(0, int(inclusive), dt_code, C.c_void_p(dx.data_ptr()),
                                      C.c_void_p(out.data_ptr()), n, C.c_void_p(stream))
        assert rc == 0, sk.lib.skel_last_error().decode()
        got = to_np(out)
        if dtype == "int32":
            assert np.array_equal(got, ref_h), f"call {call}"
        else:
            _, ab = oracle.scan_f32(x, inclusive)
            err = np.abs(got.astype(np.float64) - ref_h.astype(np.float64))
            assert np.all(err <= SUM_REL * ab), f"call {call}: max excess {float(np.max(err - SUM_REL * ab))}"


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
