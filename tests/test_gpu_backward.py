"""Parity of the hand-written backward kernels (Map, Reduce, MapReduce,
Scan; MapOverlap's adjoint is in test_gpu_mapoverlap.py) and of the
differentiable composed pipeline behind torch.autograd.Function, against the
oracle gradient and central finite differences."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import (SUM_REL, assert_elem_close, assert_prefix_close, dev_empty, dev_tensor, skel, to_np,
                     wrap)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fn", ["axpy", "add", "sub", "mul", "tanh", "sq", "scale", "copy"])
@pytest.mark.parametrize("n,pad", [(1, 0), (5, 0), (100_003, 0), (100_003, 1)])
def test_map_bwd(fn, n, pad):
    import torch
    sk = skel()
    two = fn in ("axpy", "add", "sub", "mul")
    x, y, g = syn.uniform_f32(1, n), syn.uniform_f32(2, n), syn.uniform_f32(3, n)
    ins = [wrap(dev_tensor(x, pad))] + ([wrap(dev_tensor(y, pad))] if two else [])
    gx = dev_empty((n,), torch.float32, pad)
    gy = dev_empty((n,), torch.float32, pad) if two else None
    sk.skel_map_bwd(fn, ins, wrap(dev_tensor(g, pad)), [wrap(gx)] + ([wrap(gy)] if two else []),
                    params=[2.5] if fn in ("axpy", "scale") else [])
    rx, ry = oracle.map_bwd_f32(fn if fn != "copy" else "copy", g, x, y if two else None, a=2.5)
    assert_elem_close(to_np(gx), rx, f"{fn} dx")
    if two:
        assert_elem_close(to_np(gy), ry, f"{fn} dy")


@pytest.mark.parametrize("fn", ["axpy", "mul", "tanh", "sq"])
@pytest.mark.parametrize("n,pad", [(5, 0), (100_003, 0), (100_003, 1)])
def test_map_bwd_sum_of_two_upstream_gradients(fn, n, pad):
    """The adjoint of a map whose output fed two calls: the two upstream
    gradients are added (float32, one rounding, as a separate Map ADD would)
    inside the adjoint's pass; compared with the oracle adjoint of that sum.
    A second gradient of another length is refused."""
    import torch
    sk = skel()
    two = fn in ("axpy", "mul")
    x, y = syn.uniform_f32(11, n), syn.uniform_f32(12, n)
    g1, g2 = syn.uniform_f32(13, n), syn.uniform_f32(14, n)
    ins = [wrap(dev_tensor(x, pad))] + ([wrap(dev_tensor(y, pad))] if two else [])
    gx = dev_empty((n,), torch.float32, pad)
    gy = dev_empty((n,), torch.float32, pad) if two else None
    params = [2.5] if fn == "axpy" else []
    sk.skel_map_bwd_sum(fn, ins, [wrap(dev_tensor(g1, pad)), wrap(dev_tensor(g2, pad))],
                        [wrap(gx)] + ([wrap(gy)] if two else []), params=params)
    g = (g1 + g2).astype(np.float32)
    rx, ry = oracle.map_bwd_f32(fn, g, x, y if two else None, a=2.5)
    assert_elem_close(to_np(gx), rx, f"{fn} dx, summed upstream")
    if two:
        assert_elem_close(to_np(gy), ry, f"{fn} dy, summed upstream")
    with pytest.raises(sk.SkelError) as e:
        sk.skel_map_bwd_sum(fn, ins, [wrap(dev_tensor(g1)), wrap(dev_tensor(g2[:-1] if n > 1 else g2[:0]))],
                            [wrap(gx)] + ([wrap(gy)] if two else []), params=params)
    assert e.value.code == -2


def test_tanh_bwd_from_saved_output():
    """gx = g (1 - t^2) from the saved t = tanhf(x) against g (1 - tanh(x)^2)
    in float64, within the elementwise 1e-6: tanhf is within 2 ulp, so
    |dt| <= 2^-23 for |t| < 1 and |d(1 - t^2)| <= 2|t||dt| <= 2^-22; the
    float32 square, difference and product add at most 3 * 2^-24; with
    |g| < 1 the total stays below 2^-22 + 3 * 2^-24 < 4.2e-7."""
    import torch
    sk = skel()
    n = 50_001
    x, g = syn.uniform_f32(4, n, -3, 3), syn.uniform_f32(5, n)
    t = torch.tanh(dev_tensor(x)) * 0   # placeholder buffer, filled by the skeleton below
    sk.skel_map("tanh", [wrap(dev_tensor(x))], wrap(t))
    gx = dev_empty((n,), torch.float32)
    sk.skel_map_bwd("tanh", [wrap(t)], wrap(dev_tensor(g)), [wrap(gx)], params=[1.0])
    rx, _ = oracle.map_bwd_f32("tanh", g, x)
    assert_elem_close(to_np(gx), rx, "tanh from output")


@pytest.mark.parametrize("n", [1, 4097, 1_000_003])
def test_reduce_and_mapreduce_bwd(n):
    import torch
    sk = skel()
    x, y = syn.uniform_f32(6, n), syn.uniform_f32(7, n)
    gr = torch.tensor([0.375], device="cuda")
    gx = dev_empty((n,), torch.float32)
    sk.skel_reduce_bwd("add", wrap(gr), wrap(gx))
    assert np.all(to_np(gx) == np.float32(0.375))
    sk.skel_reduce_bwd("add", None, wrap(gx), gr_host=-2.0)
    assert np.all(to_np(gx) == -2.0)
    gy = dev_empty((n,), torch.float32)
    sk.skel_mapreduce_bwd("mul", "add", [wrap(dev_tensor(x)), wrap(dev_tensor(y))], wrap(gr), [wrap(gx), wrap(gy)])
    assert_elem_close(to_np(gx), 0.375 * y.astype(np.float64), "dot dx")
    assert_elem_close(to_np(gy), 0.375 * x.astype(np.float64), "dot dy")
    sk.skel_mapreduce_bwd("sq", "add", [wrap(dev_tensor(x))], wrap(gr), [wrap(gx)])
    assert_elem_close(to_np(gx), oracle.map_bwd_f32("sq", np.full(n, 0.375, np.float32), x)[0], "sumsq dx")


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 3, 4095, 4097, 1_000_003, 1 << 22])
@pytest.mark.parametrize("inclusive", [True, False])
def test_scan_bwd(variant, n, inclusive):
    import torch
    from helpers import forced
    sk = skel()
    g = syn.uniform_f32(8, n)
    out = dev_empty((n,), torch.float32)
    with forced("scan", variant):
        sk.skel_scan_bwd("add", inclusive, wrap(dev_tensor(g)), wrap(out))
    ref, ab = oracle.scan_bwd_f32(g, inclusive)
    assert_prefix_close(to_np(out), ref, ab, f"reverse scan n={n}")


@pytest.mark.parametrize("rows,cols", [(3, 4096), (5, 1001), (2, 8192)])
def test_scan_bwd_rows(rows, cols):
    import torch
    sk = skel()
    g = syn.uniform_f32(9, rows * cols).reshape(rows, cols)
    out = dev_empty((rows, cols), torch.float32)
    sk.skel_scan_bwd("add", True, wrap(dev_tensor(g)), wrap(out))
    o = to_np(out)
    for r in range(rows):
        ref, ab = oracle.scan_bwd_f32(g[r], True)
        assert_prefix_close(o[r], ref, ab, f"row {r}")


def grad_tolerance(x, g_ref):
    """Per-element bound of the composed gradient.  Elementwise and stencil
    paths: 1e-6 * max(1, |g|).  Scan path: gt2[c] = sum_{c' >= c} 2 s[c'] g / N
    is a reverse scan of gs = 2 s g / N, so it carries (1) the reverse scan's
    own rounding, 2^-20 * sum_{c' >= c} |gs[c']|, and (2) the forward row
    scan's error |ds[c']| <= 2^-20 * P[c'] (P the prefix sum of |t|), which
    the linear map and the reverse scan carry into gt2 as
    2^-20 * sum_{c' >= c} 2 P[c'] / N -- the same sum, because |gs| is bounded
    by 2 P / N.  Hence 2 * 2^-20 times that suffix sum."""
    rows, cols = x.shape
    t = np.tanh(x.astype(np.float64))
    s_abs = np.cumsum(np.abs(t), axis=1)                  # |prefix| bound of the forward row scan
    gs_abs = 2.0 * s_abs / x.size                         # |upstream| of the reverse scan
    suffix = np.cumsum(gs_abs[:, ::-1], axis=1)[:, ::-1]
    return 1e-6 * np.maximum(1.0, np.abs(g_ref)) + 2 * SUM_REL * suffix


def loss_value_bound(x, L_ref):
    """Bound of |L_gpu - L| for L = sum u^2 + C, u = S9 t, t = tanh x,
    C = sum s^2 / N, s the row scans of t (e = 2^-24, float64 quantities):
      sum u^2 as a reduction:  2^-20 * sum u^2;
      rounding upstream of it: tanhf within 2 ulp (4e relative), the 9-tap
        stencil within 9e relative to A = sum_taps |w||t|, so |du| <= 13 e A;
        the square doubles it and rounds once: 27 e * sum |u| A;
      C: the reduction 2^-20 sum s^2, the row scan's error 2^-20 P plus the
        tanh error 4e P (P = prefix sums of |t|) doubled by the square, and
        the square's rounding e s^2, all divided by N;
      the combining axpy (1/N rounded, a product, a sum): 3e |L|.
    The whole comes to about 4.7 * 2^-20 * L on U[-1, 1] inputs."""
    from scipy import ndimage
    e = 2.0 ** -24
    t = np.tanh(x.astype(np.float64))
    w = oracle.stencil_weights("9pt").astype(np.float64)
    u = ndimage.correlate(t, w, mode="nearest")
    A = ndimage.correlate(np.abs(t), np.abs(w), mode="nearest")
    s = np.cumsum(t, axis=1)
    P = np.cumsum(np.abs(t), axis=1)
    E1 = SUM_REL * float((u * u).sum())
    E2 = 27 * e * float((np.abs(u) * A).sum())
    E3 = (SUM_REL * float((s * s).sum()) + float((2 * np.abs(s) * (SUM_REL + 4 * e) * P).sum())
          + e * float((s * s).sum())) / x.size
    return E1 + E2 + E3 + 3 * e * abs(L_ref)


@pytest.mark.parametrize("shape", [(16, 16), (64, 100), (257, 300)])
def test_composed_loss_small(shape):
    import torch
    from paper_1405_2915_gb300.autograd import composed_loss
    x = syn.uniform_f32(syn.SEED_GRAD, shape[0] * shape[1]).reshape(shape)
    xt = dev_tensor(x).requires_grad_(True)
    L = composed_loss(xt)
    L.backward()
    Lr, gr = oracle.composed_loss_f32(x, 1, oracle.stencil_weights("9pt"), "clamp")
    assert abs(float(L.item()) - Lr) <= loss_value_bound(x, Lr)
    g = to_np(xt.grad)
    assert np.all(np.abs(g - gr) <= grad_tolerance(x, gr))


def test_composed_loss_8192_fd_and_oracle_gradient():
    """The differentiable workload: 8192 x 8192 grid, U[-1,1]; GPU gradient vs
    the float64 oracle gradient at every point, and vs central finite
    differences (h = 1e-3) of the float64 oracle at 64 seeded probes."""
    import torch
    from paper_1405_2915_gb300.autograd import composed_loss
    W = 8192
    x = syn.uniform_f32(syn.SEED_GRAD, W * W).reshape(W, W)
    xt = dev_tensor(x).requires_grad_(True)
    L = composed_loss(xt)
    L.backward()
    g = to_np(xt.grad)
    w9 = oracle.stencil_weights("9pt")
    Lr, gr = oracle.composed_loss_f32(x, 1, w9, "clamp")
    assert abs(float(L.item()) - Lr) <= loss_value_bound(x, Lr)
    assert np.all(np.abs(g - gr) <= grad_tolerance(x, gr))
    probes = syn.splitmix64(syn.SEED_GRAD + 1, 64) % np.uint64(W * W)
    h = 1e-3
    for p in probes:
        i, j = divmod(int(p), W)
        fd = (oracle.composed_loss_delta_f32(x, 1, w9, i, j, h) -
              oracle.composed_loss_delta_f32(x, 1, w9, i, j, -h)) / (2 * h)
        assert abs(g[i, j] - fd) <= 1e-4 * abs(fd) + 1e-7, (i, j, g[i, j], fd)


@pytest.mark.parametrize("n", [4, 4096, 12288, 12292, 16384, 16388, 28672, 40964, 1_000_000, 1 << 22])
@pytest.mark.parametrize("inclusive", [True, False])
@pytest.mark.parametrize("variant,tile", [(5, 0), (5, 1), (5, 3), (6, 0), (6, 1), (7, 0), (7, 1), (7, 2), (7, 3), (8, 0),
                                          (8, 1), (8, 2), (8, 3)])
def test_scan_bwd_big_tiles(n, inclusive, variant, tile):
    """Reverse scans through the staged big-tile and warp-specialised
    variants (n % 4 == 0)."""
    import torch
    from helpers import forced
    sk = skel()
    g = syn.uniform_f32(10, n)
    out = dev_empty((n,), torch.float32)
    with forced("scan", variant, 0, 0, tile):
        sk.skel_scan_bwd("add", inclusive, wrap(dev_tensor(g)), wrap(out))
    ref, ab = oracle.scan_bwd_f32(g, inclusive)
    assert_prefix_close(to_np(out), ref, ab, f"reverse big n={n}")


@pytest.mark.parametrize("variant", [5, 6, 7, 8])
def test_scan_bwd_big_tiles_rows_and_refusal(variant):
    import torch
    from helpers import forced
    sk = skel()
    rows, cols = 3, 40000
    g = syn.uniform_f32(11, rows * cols).reshape(rows, cols)
    out = dev_empty((rows, cols), torch.float32)
    with forced("scan", variant):
        sk.skel_scan_bwd("add", True, wrap(dev_tensor(g)), wrap(out))
        o = to_np(out)
        for r in range(rows):
            ref, ab = oracle.scan_bwd_f32(g[r], True)
            assert_prefix_close(o[r], ref, ab, f"row {r}")
        bad = dev_empty((4099,), torch.float32)
        with pytest.raises(sk.SkelError) as e:   # reverse 1D scans need n % 4 == 0 here
            sk.skel_scan_bwd("add", True, wrap(dev_tensor(syn.uniform_f32(12, 4099))), wrap(bad))
        assert e.value.code == -4


def test_scan_bwd_reread_refusals():
    """The re-reading variant refuses reverse 1D scans with n % 4 != 0 before
    any launch."""
    import torch
    from helpers import forced
    sk = skel()
    with forced("scan", 8):
        for n in (4099, 2):
            bad = dev_empty((n,), torch.float32)
            with pytest.raises(sk.SkelError) as e:
                sk.skel_scan_bwd("add", True, wrap(dev_tensor(syn.uniform_f32(12, n))), wrap(bad))
            assert e.value.code == -4
