"""Shared helpers of the GPU tests: device containers over torch tensors,
tolerance checks that state the bound they apply."""
from __future__ import annotations

import contextlib

import numpy as np

# float32 tolerance of sums and scans: |gpu - oracle| <= 2^-20 * sum |terms|
SUM_REL = 2.0 ** -20
# elementwise tolerance of map / mapoverlap outputs (absolute)
ELEM_ABS = 1e-6


def skel():
    import paper_1405_2915_gb300 as sk
    return sk


def dev_tensor(a: np.ndarray, pad_front: int = 0):
    """Copies a host array to a CUDA tensor; with pad_front > 0 the returned
    tensor is a view starting pad_front elements into a larger allocation
    (so its address is not 16-byte aligned when pad_front % 4 != 0)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a).ravel())
    if pad_front:
        big = torch.zeros(t.numel() + pad_front, dtype=t.dtype)
        big[pad_front:] = t
        d = big.cuda()[pad_front:]
    else:
        d = t.cuda()
    return d.view(a.shape) if a.ndim == 2 else d


def dev_empty(shape, dtype, pad_front: int = 0):
    import torch
    n = int(np.prod(shape))
    t = torch.empty(n + pad_front, dtype=dtype, device="cuda")[pad_front:]
    return t.view(*shape) if len(shape) == 2 else t


def wrap(t):
    return skel().Container.from_tensor(t)


def to_np(t) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@contextlib.contextmanager
def forced(skeleton: str, variant: int, block: int = 0, ept: int = 0, tile: int = 0):
    sk = skel()
    sk.skel_force_variant(skeleton, variant, block, ept, tile)
    try:
        yield
    finally:
        sk.skel_force_variant(skeleton, -1)


def assert_sum_close(gpu: float, ref: float, abs_sum: float, what: str = ""):
    tol = SUM_REL * abs_sum
    err = abs(float(gpu) - ref)
    assert err <= tol, f"{what}: |gpu-oracle| = {err:.3e} > 2^-20 * sum|terms| = {tol:.3e}"


def assert_prefix_close(gpu: np.ndarray, ref: np.ndarray, abs_prefix: np.ndarray, what: str = ""):
    err = np.abs(gpu.astype(np.float64) - ref)
    tol = SUM_REL * abs_prefix
    bad = err > tol
    if bad.any():
        i = int(np.argmax(bad))
        raise AssertionError(f"{what}: element {i}: |gpu-oracle| = {err[i]:.3e} > {tol[i]:.3e} "
                             f"({int(bad.sum())} elements out of bound)")


def assert_elem_close(gpu: np.ndarray, ref: np.ndarray, what: str = "", atol: float = ELEM_ABS):
    err = np.abs(gpu.astype(np.float64) - ref)
    if err.size and err.max() > atol:
        i = int(np.argmax(err))
        raise AssertionError(f"{what}: element {i}: |gpu-oracle| = {err.flat[i]:.3e} > {atol:.1e}")
