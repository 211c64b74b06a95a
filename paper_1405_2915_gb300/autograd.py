"""torch.autograd.Function wrappers of the skeletons and their hand-written
adjoints.  Forward and backward both run in libskel.so: the adjoint of Map is
an elementwise map, of MapReduce and Reduce a scaled broadcast, of Scan a
reverse scan, of MapOverlap the transposed stencil.  torch only supplies the
tensors (device memory) and the current stream; each Function wraps its
tensors as containers and calls the C ABI.
"""
from __future__ import annotations

import torch

from . import (Container, skel_map, skel_map_bwd, skel_mapoverlap, skel_mapoverlap_bwd, skel_mapreduce,
               skel_mapreduce_bwd, skel_reduce, skel_reduce_bwd, skel_scan, skel_scan_bwd)


def _c(t: torch.Tensor) -> Container:
    return Container.from_tensor(t)


def _prep(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError("skeleton autograd functions take float32 CUDA tensors")
    return t.contiguous()


class MapFn(torch.autograd.Function):
    """out = f(x[, y]; a) elementwise (skel_map); backward: skel_map_bwd."""

    @staticmethod
    def forward(ctx, fn: str, a: float, x, y=None):
        x = _prep(x)
        ins = [x] if y is None else [x, _prep(y)]
        out = torch.empty_like(x)
        params = [a] if fn in ("axpy", "scale") else []
        skel_map(fn, [_c(t) for t in ins], _c(out), params)
        ctx.fn, ctx.a = fn, a
        # tanh's derivative is taken from the saved output (1 - out^2)
        ctx.save_for_backward(*([out] if fn == "tanh" else ins))
        ctx.nin = len(ins)
        return out

    @staticmethod
    def backward(ctx, g):
        g = _prep(g)
        saved = ctx.saved_tensors
        gins = [torch.empty_like(g) if ctx.needs_input_grad[2 + k] else None for k in range(ctx.nin)]
        if any(t is not None for t in gins):
            if ctx.fn == "tanh":
                skel_map_bwd("tanh", [_c(saved[0])], _c(g), [None if t is None else _c(t) for t in gins], [1.0])
            else:
                params = [ctx.a] if ctx.fn in ("axpy", "scale") else []
                skel_map_bwd(ctx.fn, [_c(t) for t in saved], _c(g),
                             [None if t is None else _c(t) for t in gins], params)
        return (None, None, *gins) if ctx.nin == 2 else (None, None, gins[0], None)


class MapOverlapFn(torch.autograd.Function):
    """Stencil (skel_mapoverlap); backward: transposed stencil."""

    @staticmethod
    def forward(ctx, x, fn: str, radius: int, weights, boundary: str):
        x = _prep(x)
        out = torch.empty_like(x)
        skel_mapoverlap(fn, radius, weights, boundary, _c(x), _c(out))
        ctx.args = (fn, radius, weights, boundary)
        return out

    @staticmethod
    def backward(ctx, g):
        g = _prep(g)
        gin = torch.empty_like(g)
        skel_mapoverlap_bwd(*ctx.args, _c(g), _c(gin))
        return gin, None, None, None, None


class SumSqFn(torch.autograd.Function):
    """sum_i x_i^2 (skel_mapreduce with SQ, ADD) as a 1-element tensor;
    backward: gx = 2 x g (skel_mapreduce_bwd)."""

    @staticmethod
    def forward(ctx, x):
        x = _prep(x)
        r = torch.empty(1, device=x.device, dtype=torch.float32)
        skel_mapreduce("sq", "add", [_c(x)], result_dev=_c(r), host=False)
        ctx.save_for_backward(x)
        return r

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        gx = torch.empty_like(x)
        skel_mapreduce_bwd("sq", "add", [_c(x)], _c(_prep(g.reshape(1))), [_c(gx)])
        return gx


class SumFn(torch.autograd.Function):
    """sum_i x_i (skel_reduce ADD) as a 1-element tensor; backward: broadcast."""

    @staticmethod
    def forward(ctx, x):
        x = _prep(x)
        r = torch.empty(1, device=x.device, dtype=torch.float32)
        skel_reduce("add", _c(x), result_dev=_c(r), host=False)
        ctx.shape = x.shape
        return r

    @staticmethod
    def backward(ctx, g):
        gx = torch.empty(ctx.shape, device=g.device, dtype=torch.float32)
        skel_reduce_bwd("add", _c(_prep(g.reshape(1))), _c(gx))
        return gx


class ScanFn(torch.autograd.Function):
    """Scan (+) of a 1D tensor, or of every row of a 2D tensor (skel_scan);
    backward: the reverse scan (skel_scan_bwd)."""

    @staticmethod
    def forward(ctx, x, inclusive: bool = True):
        x = _prep(x)
        out = torch.empty_like(x)
        skel_scan("add", inclusive, _c(x), _c(out))
        ctx.inclusive = inclusive
        return out

    @staticmethod
    def backward(ctx, g):
        g = _prep(g)
        gin = torch.empty_like(g)
        skel_scan_bwd("add", ctx.inclusive, _c(g), _c(gin))
        return gin, None


def composed_loss(x: torch.Tensor, weights=None, boundary: str = "clamp") -> torch.Tensor:
    """The differentiable composed pipeline on a rows x cols grid:
        t = tanh(x)                         Map
        L1 = sum (S9 t)^2                   MapOverlap, MapReduce
        C  = sum (rowscan t)^2              Scan (per row), MapReduce
        L  = C / (rows * cols) + L1         Map (axpy on the two scalars)
    Every step, forward and backward, is a skeleton call."""
    t = MapFn.apply("tanh", 0.0, x)
    l1 = SumSqFn.apply(MapOverlapFn.apply(t, "stencil9", 1, weights, boundary))
    c = SumSqFn.apply(ScanFn.apply(t, True))
    return MapFn.apply("axpy", 1.0 / x.numel(), c, l1)
