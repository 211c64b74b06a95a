"""torch.autograd.Function wrappers of the skeletons and their hand-written
adjoints.  Forward and backward both run in libskel.so: the adjoint of Map is
an elementwise map, of MapReduce and Reduce a scaled broadcast, of Scan a
reverse scan, of MapOverlap the transposed stencil.  torch only supplies the
tensors (device memory) and the current stream; each Function wraps its
tensors as containers and calls the C ABI.
"""
from __future__ import annotations

import torch

from . import (Container, skel_map, skel_map_bwd, skel_map_bwd_sum, skel_mapoverlap, skel_mapoverlap_bwd,
               skel_mapreduce, skel_mapreduce_bwd, skel_reduce, skel_reduce_bwd, skel_scan, skel_scan_bwd)


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


def _call(step, name: str, fn) -> None:
    if step is None:
        fn()
    else:
        step(name, fn)


class ComposedLossFn(torch.autograd.Function):
    """The differentiable composed pipeline as one Function, so that the
    gradients of its two branches (t feeds both the stencil and the row scan)
    are added by a skeleton call instead of by torch's autograd engine (the
    tanh adjoint takes both and adds them in its own pass).

    Forward (skeleton calls):
        t = tanh(x)                              Map
        u = S t, l1 = sum u^2                    MapOverlap, MapReduce(sq, +)
        s = rowscan t, c = sum s^2               Scan (per row), MapReduce(sq, +)
        L = c / (rows * cols) + l1               Map (axpy on the two scalars)
    Backward, with g = dL (a device scalar):
        gc = g / (rows * cols)                   Map (scale on the scalar)
        gt = S^T (2 u g)                         MapReduce adjoint, transposed stencil
        gt2 = rscan(2 s gc)                      MapReduce adjoint, reverse scan
        gx = (gt + gt2) (1 - t^2)                Map adjoint of tanh (from the saved t) over the
                                                 sum of the two branches' gradients, one pass
    `step(name, thunk)`, when given, runs each call (the benchmark times
    them one by one); the calls and their order are the same either way."""

    @staticmethod
    def forward(ctx, x, weights, boundary: str, step=None):
        x = _prep(x)
        t, u, s = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        r = torch.empty(2, device=x.device, dtype=torch.float32)     # l1, c
        L = torch.empty(1, device=x.device, dtype=torch.float32)
        ct, cu, cs = _c(t), _c(u), _c(s)
        cl1, cc, cL = _c(r[0:1]), _c(r[1:2]), _c(L)
        _call(step, "fwd_map_tanh", lambda: skel_map("tanh", [_c(x)], ct))
        _call(step, "fwd_mapoverlap_9pt", lambda: skel_mapoverlap("stencil9", 1, weights, boundary, ct, cu))
        _call(step, "fwd_sumsq_stencil", lambda: skel_mapreduce("sq", "add", [cu], result_dev=cl1, host=False))
        _call(step, "fwd_row_scan", lambda: skel_scan("add", True, ct, cs))
        _call(step, "fwd_sumsq_scan", lambda: skel_mapreduce("sq", "add", [cs], result_dev=cc, host=False))
        _call(step, "fwd_combine", lambda: skel_map("axpy", [cc, cl1], cL, [1.0 / x.numel()]))
        ctx.save_for_backward(t, u, s)
        ctx.args = (weights, boundary, step, x.numel())
        return L

    @staticmethod
    def backward(ctx, g):
        t, u, s = ctx.saved_tensors
        weights, boundary, step, n = ctx.args
        g = _prep(g.reshape(1))
        gc = torch.empty(1, device=g.device, dtype=torch.float32)
        gu, gt, gs, gt2, gx = (torch.empty_like(t) for _ in range(5))
        cg, cgc, cgt = _c(g), _c(gc), _c(gt)
        _call(step, "bwd_scale", lambda: skel_map("scale", [cg], cgc, [1.0 / n]))
        _call(step, "bwd_sumsq_stencil", lambda: skel_mapreduce_bwd("sq", "add", [_c(u)], cg, [_c(gu)]))
        _call(step, "bwd_mapoverlap_9pt", lambda: skel_mapoverlap_bwd("stencil9", 1, weights, boundary, _c(gu), cgt))
        _call(step, "bwd_sumsq_scan", lambda: skel_mapreduce_bwd("sq", "add", [_c(s)], cgc, [_c(gs)]))
        _call(step, "bwd_reverse_scan", lambda: skel_scan_bwd("add", True, _c(gs), _c(gt2)))
        _call(step, "bwd_map_tanh_sum", lambda: skel_map_bwd_sum("tanh", [_c(t)], [cgt, _c(gt2)], [_c(gx)], [1.0]))
        return gx, None, None, None


def composed_loss(x: torch.Tensor, weights=None, boundary: str = "clamp", step=None) -> torch.Tensor:
    """L = sum (S9 tanh x)^2 + sum (rowscan tanh x)^2 / (rows * cols) on a
    rows x cols grid (ComposedLossFn); every step, forward and backward, is a
    skeleton call of libskel.so."""
    return ComposedLossFn.apply(x, weights, boundary, step)
