"""Off-line autotuner: builds the execution-plan table (Sec. II off-line
tuning into a dispatch structure for fast run-time lookup; Sec. III execution
plans recomputed once per target system) by timing every variant and launch
shape of each skeleton instance at one representative size per bucket
(n = 4^k, bucket k = floor(log2(n) / 2)).

Rules:
  * the built-in default variant is always a candidate, and another candidate
    replaces it only when it is faster by more than `--margin` (3 %);
  * each candidate is timed on the device (CUDA events on the launching
    stream) as the median of `--reps` runs, with L2 flushed before every run
    when the operands fit in L2;
  * after tuning, sizes between the buckets (n = 2 * 4^k) are timed with the
    table and with the defaults; a bucket whose choice is slower there than
    the default by more than the margin is re-timed and, unless it holds up,
    set back to the default, so that the table is never slower.

    python -m paper_1405_2915_gb300.tune --out paper_1405_2915_gb300/dispatch_gb300.tbl \
        --report paper_1405_2915_gb300/dispatch_gb300_report.md
"""
from __future__ import annotations

import argparse
import itertools
import os
import statistics
import sys
import time

import numpy as np
import torch

from . import (F32, I32, SK, UNIT_HOST, Container, SkelError, skel_batched, skel_force_variant, skel_load_dispatch_table,
               skel_map, skel_mapoverlap, skel_mapoverlap_chain, skel_maparray, skel_maparray_grid, skel_mapreduce,
               skel_reduce, skel_scan, skel_scan_bwd, skel_compose_map_stencil_sumsq)
from ._lib import FN

L2_FLUSH_BYTES = 512 << 20


class Timer:
    def __init__(self):
        self.flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.stream = torch.cuda.current_stream()

    def time(self, fn, nbytes: int, reps: int) -> float:
        """Median device time in ms of fn()."""
        fn()   # warm-up (also surfaces an unsupported configuration)
        flush = nbytes < 2 * 129 * (1 << 20)
        ts = []
        for _ in range(reps):
            if flush:
                # read (not write) a buffer larger than L2: L2 ends up full of
                # clean lines, so no write-back of flush data is charged to fn
                self.flush.sum()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            fn()
            b.record(self.stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)


def grid_of(**axes):
    keys = list(axes)
    for vals in itertools.product(*(axes[k] for k in keys)):
        yield dict(zip(keys, vals))


# candidates per skeleton: (variant, block, ept, tile)
def candidates(sk_name: str):
    if sk_name == "map":
        yield (0, 256, 0, 0)
        for v in (1, 2, 3):
            for blk in (128, 256, 512):
                for e in (1, 2, 4):
                    yield (v, blk, e, 0)
    elif sk_name in ("reduce", "mapreduce"):
        for v in (0, 1, 2):
            for blk in (128, 256, 512):
                for e in (1, 2, 4, 8):
                    yield (v, blk, e, 0)
    elif sk_name == "scan":
        for v in (0, 1, 2, 3):
            for e in (2, 4, 8):
                yield (v, 256, e, 0)
        yield (4, 256, 4, 0)
        for t in (0, 1, 2, 3):   # early aggregate (bit 0), 48 KiB tiles (bit 1)
            yield (5, 256, 4, t)
        for t in (0, 1):         # warp-specialised stages: 4 x 48 KiB, 6 x 32 KiB
            yield (6, 256, 4, t)
        for t in (0, 1, 2, 3):   # hybrid-staged tiles: 96 + 64, 64 + 32, 64 + 48, 96 + 80 KiB
            yield (7, 256, 4, t)
        for t in (0, 1, 2, 3):   # aggregators and re-reading scanners: ring tiles + scanners 6 + 6, 4 + 8, 6 + 8, 5 + 8
            yield (8, 256, 4, t)
    elif sk_name == "mapoverlap2d":
        yield (0, 256, 0, 0)
        yield (1, 256, 0, 0)
        yield (2, 256, 0, 0)
        for t in (16, 32, 64, 128):
            yield (3, 128, 0, t)
    elif sk_name == "mapoverlap1d":
        yield (0, 256, 0, 0)
        yield (1, 256, 8, 0)
        yield (2, 256, 0, 0)
    elif sk_name == "maparray":
        for v in (0, 1, 2, 3):
            yield (v, 256, 0, 0)
        for e in (4, 8):         # gather: more groups of four in flight per thread (rowdot ignores ept)
            yield (2, 256, e, 0)
    elif sk_name == "chain2d":
        yield (0, 0, 0, 0)
        for k in (1, 2, 3, 4, 5, 6, 8):
            yield (1, 256, 0, k)
    elif sk_name == "compose":
        yield (0, 0, 0, 0)
        for t in (0, 1, 2):      # fused: 32, 64, 128 rows per block
            yield (1, 0, 0, t)
    elif sk_name == "edge":
        yield (0, 0, 0, 0)
        for t in (0, 1, 2):      # chunks of 8, 32, 128 MiB
            yield (1, 0, 0, t)
        yield (2, 0, 0, 0)
    elif sk_name == "batched":
        for v in (0, 1, 2, 4):
            for e in (2, 4, 8):
                yield (v, 256, e, 0)
        yield (3, 256, 4, 0)
        yield (5, 256, 4, 0)
        yield (5, 256, 8, 0)
        for t in (0, 1):         # the instances as one flat segmented scan, two tile shapes
            yield (6, 256, 4, t)
        for t in (0, 1):         # flat, aggregators and re-reading scanners: ring tiles + scanners 6 + 6, 4 + 8
            yield (7, 256, 4, t)


def grid_side(n: int) -> int:
    """The side of the square grid that stands for n points: sqrt(n) rounded
    to a multiple of 4, so that a grid of about 2n points (the second timing
    point of a bucket) keeps 16-byte aligned rows like the bucket's own
    4^k-point grid, and no variant that needs them is ruled out there."""
    return max(4, 4 * int(round(n ** 0.5 / 4)))


class Instance:
    """One skeleton instance (skeleton + user function + dtype) with buffers
    for its largest size; call(n) runs it on the first n elements."""

    def __init__(self, name, sk_name, fn_key, dtype, radius, nmax, make, nbytes, sizes, residency=0):
        self.name, self.sk_name, self.fn_key, self.dtype, self.radius = name, sk_name, fn_key, dtype, radius
        self.nmax, self.make, self.nbytes, self.sizes = nmax, make, nbytes, sizes
        self.residency = residency


def instances(nmax_log2: int):
    nmax = 1 << nmax_log2
    sizes = [1 << (2 * k) for k in range(5, nmax_log2 // 2 + 1)]
    dev = torch.device("cuda")
    out = []

    def vec(n, lo=-1.0, hi=1.0):
        return (torch.rand(n, device=dev) * (hi - lo) + lo).contiguous()

    def mk_map(fn, nin):
        bufs = {}

        def make(n):
            if "x" not in bufs:
                bufs["x"], bufs["y"], bufs["o"] = vec(nmax), vec(nmax), vec(nmax)
            ins = [Container.from_tensor(bufs["x"][:n])] + ([Container.from_tensor(bufs["y"][:n])] if nin == 2 else [])
            o = Container.from_tensor(bufs["o"][:n])
            return lambda: skel_map(fn, ins, o, [2.5] if fn == "axpy" else [])
        return make

    out.append(Instance("map axpy f32", "map", FN["axpy"], F32, 0, nmax, mk_map("axpy", 2), lambda n: 12 * n, sizes))
    out.append(Instance("map tanh f32", "map", FN["tanh"], F32, 0, nmax, mk_map("tanh", 1), lambda n: 8 * n, sizes))

    def mk_red(op, dt):
        bufs = {}

        def make(n):
            if "x" not in bufs:
                bufs["x"] = vec(nmax) if dt == F32 else torch.randint(0, 101, (nmax,), device=dev, dtype=torch.int32)
                bufs["r"] = torch.zeros(1, device=dev, dtype=bufs["x"].dtype)
            x, r = Container.from_tensor(bufs["x"][:n]), Container.from_tensor(bufs["r"])
            return lambda: skel_reduce(op, x, r, host=False)
        return make

    for op in ("add", "max"):
        for dt, dn in ((F32, "f32"), (I32, "i32")):
            out.append(Instance(f"reduce {op} {dn}", "reduce", FN[op], dt, 0, nmax, mk_red(op, dt), lambda n: 4 * n, sizes))

    def mk_mr(fn):
        bufs = {}

        def make(n):
            if "x" not in bufs:
                bufs["x"], bufs["y"], bufs["r"] = vec(nmax), vec(nmax), torch.zeros(1, device=dev)
            ins = [Container.from_tensor(bufs["x"][:n])] + ([Container.from_tensor(bufs["y"][:n])] if fn == "mul" else [])
            r = Container.from_tensor(bufs["r"])
            return lambda: skel_mapreduce(fn, "add", ins, r, host=False)
        return make

    out.append(Instance("mapreduce dot f32", "mapreduce", FN["mul"], F32, 0, nmax, mk_mr("mul"), lambda n: 8 * n, sizes))
    out.append(Instance("mapreduce sumsq f32", "mapreduce", FN["sq"], F32, 0, nmax, mk_mr("sq"), lambda n: 4 * n, sizes))

    def mk_scan(dt, incl):
        bufs = {}

        def make(n):
            if "x" not in bufs:
                if dt == F32:
                    bufs["x"], bufs["o"] = vec(nmax), vec(nmax)
                else:
                    bufs["x"] = torch.randint(0, 101, (nmax,), device=dev, dtype=torch.int32)
                    bufs["o"] = torch.empty(nmax, device=dev, dtype=torch.int32)
            x, o = Container.from_tensor(bufs["x"][:n]), Container.from_tensor(bufs["o"][:n])
            return lambda: skel_scan("add", incl, x, o)
        return make

    for dt, dn in ((I32, "i32"), (F32, "f32")):
        for incl in (True, False):
            out.append(Instance(f"scan {'incl' if incl else 'excl'} {dn}", "scan", 1 if incl else 0, dt, 0, nmax,
                                mk_scan(dt, incl), lambda n: 8 * n, sizes))

    def mk_rscan(incl):   # the reverse scan of the adjoint (its own keys: fn 3 inclusive, 2 exclusive)
        bufs = {}

        def make(n):
            if "x" not in bufs:
                bufs["x"], bufs["o"] = vec(nmax), vec(nmax)
            x, o = Container.from_tensor(bufs["x"][:n]), Container.from_tensor(bufs["o"][:n])
            return lambda: skel_scan_bwd("add", incl, x, o)
        return make

    for incl in (True, False):
        out.append(Instance(f"reverse scan {'incl' if incl else 'excl'} f32", "scan", 3 if incl else 2, F32, 0, nmax,
                            mk_rscan(incl), lambda n: 8 * n, sizes))

    def mk_st2(fn):
        bufs = {}

        def make(n):
            side = grid_side(n)
            if "x" not in bufs:
                bufs["x"], bufs["o"] = vec(nmax, 0.0, 1.0), vec(nmax)
            x = Container.from_tensor(bufs["x"][:side * side].view(side, side))
            o = Container.from_tensor(bufs["o"][:side * side].view(side, side))
            return lambda: skel_mapoverlap(fn, 1, None, "clamp", x, o)
        return make

    for fn in ("stencil9", "stencil5"):
        out.append(Instance(f"mapoverlap2d {fn} clamp", "mapoverlap2d", FN[fn], F32, 1, nmax, mk_st2(fn),
                            lambda n: 8 * n, sizes))

    def mk_chain(fn, steps):   # key: radius field = number of steps
        bufs = {}

        def make(n):
            side = grid_side(n)
            if "x" not in bufs:
                bufs["x"], bufs["o"], bufs["t"] = vec(nmax, 0.0, 1.0), vec(nmax), vec(nmax)
            x, o, t = (Container.from_tensor(bufs[k][:side * side].view(side, side)) for k in ("x", "o", "t"))
            return lambda: skel_mapoverlap_chain(fn, None, "clamp", steps, x, t, o)
        return make

    for fn in ("stencil9", "stencil5"):
        out.append(Instance(f"mapoverlap2d chain {fn} clamp x10", "chain2d", FN[fn], F32, 10, nmax, mk_chain(fn, 10),
                            lambda n: 80 * n, sizes))

    def mk_compose(fn, map_fn):   # Map -> MapOverlap -> MapReduce(sq, +), one call
        bufs = {}

        def make(n):
            side = grid_side(n)
            if "x" not in bufs:
                bufs["x"], bufs["r"] = vec(nmax), torch.zeros(1, device=dev)
            x = Container.from_tensor(bufs["x"][:side * side].view(side, side))
            r = Container.from_tensor(bufs["r"])
            return lambda: skel_compose_map_stencil_sumsq(map_fn, fn, x, result_dev=r, host=False)
        return make

    out.append(Instance("compose tanh -> stencil9 -> sumsq", "compose", FN["stencil9"], F32, 1, nmax,
                        mk_compose("stencil9", "tanh"), lambda n: 4 * n, sizes))

    def mk_st1(r):
        bufs = {}

        def make(n):
            if "x" not in bufs:
                bufs["x"], bufs["o"] = vec(nmax), vec(nmax)
            x, o = Container.from_tensor(bufs["x"][:n]), Container.from_tensor(bufs["o"][:n])
            return lambda: skel_mapoverlap("stencil1d", r, None, "clamp", x, o)
        return make

    for r in (1, 4, 8, 16):
        out.append(Instance(f"mapoverlap1d r={r} clamp", "mapoverlap1d", FN["stencil1d"], F32, r, nmax, mk_st1(r),
                            lambda n: 8 * n, sizes))

    def mk_rowdot():
        bufs = {}

        def make(m):   # key = row length m; rows so that the matrix holds min(nmax, 64 m) elements... at most nmax
            rows = max(1, min(nmax // m, 1 << 14))
            if "M" not in bufs:
                bufs["M"], bufs["A"], bufs["o"] = vec(nmax), vec(nmax), vec(1 << 20)
            A = Container.from_tensor(bufs["A"][:m])
            M = Container.from_tensor(bufs["M"][:rows * m].view(rows, m))
            o = Container.from_tensor(bufs["o"][:rows])
            make.rows = rows
            return lambda: skel_maparray("rowdot", A, M, o)
        return make

    rd = mk_rowdot()
    out.append(Instance("maparray rowdot f32", "maparray", FN["rowdot"], F32, 0, nmax, rd,
                        lambda m: 4 * m * max(1, min(nmax // m, 1 << 14)), sizes))

    def mk_gather():
        bufs = {}

        def make(n):
            if "i" not in bufs:
                bufs["A"] = vec(1 << 20)
                bufs["i"] = torch.randint(0, 1 << 20, (nmax,), device=dev, dtype=torch.int32)
                bufs["o"] = vec(nmax)
            A, i, o = (Container.from_tensor(bufs["A"]), Container.from_tensor(bufs["i"][:n]),
                       Container.from_tensor(bufs["o"][:n]))
            return lambda: skel_maparray("gather", A, i, o)
        return make

    out.append(Instance("maparray gather f32", "maparray", FN["gather"], F32, 0, nmax, mk_gather(), lambda n: 8 * n, sizes))

    def mk_coulomb():   # n grid points (a square-ish slab, 256 columns) against 1024 atoms
        bufs = {}

        def make(n):
            if "a" not in bufs:
                a = torch.rand((1024, 4), device=dev) * 32.0
                a[:, 2] += 0.5
                a[:, 3] = a[:, 3] / 16.0 - 1.0
                bufs["a"], bufs["o"] = a, vec(min(nmax, 1 << 22))
            cols = 256 if n >= 256 else n
            o = bufs["o"][:n].view(n // cols, cols)
            A, O = Container.from_tensor(bufs["a"]), Container.from_tensor(o)
            return lambda: skel_maparray_grid("coulomb", A, O, (0.125, 0.0))
        return make

    csizes = [q for q in sizes if q <= (1 << 20)]
    out.append(Instance("maparray coulomb f32 (1024 atoms)", "maparray", FN["coulomb"], F32, 0, 1 << 21, mk_coulomb(),
                        lambda n: 4 * n, csizes))

    # the host edge: inputs valid only in pinned host memory at every call
    # (residency 1); the bytes counted are the call's own, so the rates are
    # bounded by the host link, not by HBM
    emax = min(nmax, 1 << 26)
    esizes = [s for s in sizes if (1 << 16) <= s <= emax]

    def mk_edge(kind):
        bufs = {}

        def make(n):
            if "x" not in bufs:
                bufs["x"] = torch.rand(emax).pin_memory()
                bufs["y"] = torch.rand(emax).pin_memory()
                bufs["o"], bufs["r"] = vec(emax), torch.zeros(1, device=dev)
            cx = Container.from_host(bufs["x"].numpy()[:n])
            cy = Container.from_host(bufs["y"].numpy()[:n])
            co, cr = Container.from_tensor(bufs["o"][:n]), Container.from_tensor(bufs["r"])

            def call():
                cx.mark(UNIT_HOST)
                cy.mark(UNIT_HOST)
                if kind == "map":
                    skel_map("axpy", [cx, cy], co, [2.5])
                elif kind == "reduce":
                    skel_reduce("add", cx, cr, host=False)
                else:
                    skel_mapreduce("mul", "add", [cx, cy], cr, host=False)
            return call
        return make

    out.append(Instance("host edge: map axpy f32", "edge", SK["map"], F32, 0, emax, mk_edge("map"),
                        lambda n: 12 * n, esizes, residency=1))
    out.append(Instance("host edge: reduce add f32", "edge", SK["reduce"], F32, 0, emax, mk_edge("reduce"),
                        lambda n: 4 * n, esizes, residency=1))
    out.append(Instance("host edge: mapreduce dot f32", "edge", SK["mapreduce"], F32, 0, emax, mk_edge("mapreduce"),
                        lambda n: 8 * n, esizes, residency=1))
    return out


def batched_instance():
    """The batched workload: 4096 log-uniform instances in [64, 2^20] (one
    bucket; smaller and larger totals extrapolate from it)."""
    import synthetic as syn
    lens = syn.loguniform_lengths(syn.SEED_BATCH_LEN, 4096)
    off = syn.csr_offsets(lens)
    total = int(off[-1])
    dev = torch.device("cuda")
    v = torch.rand(total, device=dev) * 2 - 1
    o = torch.from_numpy(off).to(dev)
    res = torch.empty(4096, device=dev)
    sc = torch.empty(total, device=dev)
    cv, co, cr, cs = (Container.from_tensor(t) for t in (v, o, res, sc))
    return total, (lambda: skel_batched(cv, co, cr, cs, True)), 8 * total


def bucket(n: int) -> int:
    return min(15, (int(n).bit_length() - 1) // 2)


def adaptive_sizes(sizes, decide, key, stride: int = 3):
    """Adaptive sampling over the size buckets: decide() every stride-th size
    and the last one; between two sampled sizes whose decisions (compared by
    key) differ, decide the middle one and recurse on both halves.  A run of
    buckets bounded by two equal decisions is left unsampled (None) and takes
    that decision (a change and its undoing within one stride go unseen; the
    validation between buckets still checks every bucket against the
    default).  Returns {size: decide(size) or None}."""
    got = {}

    def d(i):
        if i not in got:
            got[i] = decide(sizes[i])
        return got[i]

    def rec(lo, hi):
        if hi - lo <= 1 or key(d(lo)) == key(d(hi)):
            return
        mid = (lo + hi) // 2
        d(mid)
        rec(lo, mid)
        rec(mid, hi)

    if sizes:
        coarse = sorted(set(list(range(0, len(sizes), stride)) + [len(sizes) - 1]))
        for i in coarse:
            d(i)
        for lo, hi in zip(coarse, coarse[1:]):
            rec(lo, hi)
    return {n: got.get(i) for i, n in enumerate(sizes)}


def tune(args):
    timer = Timer()
    lines = ["# execution-plan table of libskel.so, written by paper_1405_2915_gb300.tune on "
             + torch.cuda.get_device_name(),
             "# skeleton fn dtype bucket radius residency variant block ept tile"]
    report = ["| skeleton instance | n | default GB/s | tuned GB/s | speedup | chosen |", "|---|---|---|---|---|---|"]
    chosen_all = []
    samples_taken = samples_full = 0
    skel_load_dispatch_table(None)
    for inst in instances(args.nmax_log2):
        if args.only and not any(s in inst.name for s in args.only):
            continue
        sk_id = SK[inst.sk_name]

        def decide(n):
            """Times the default and every candidate at n (and 2n); returns
            (choice or None, default ms, chosen ms, bytes)."""
            # a bucket spans [n, 4n): a candidate must beat the default both
            # at its lower edge and in its middle (2n) to be chosen
            pts = [n] + ([2 * n] if 2 * n <= inst.nmax else [])
            fns = [inst.make(q) for q in pts]
            nbs = [inst.nbytes(q) for q in pts]
            skel_force_variant(sk_id, -1)
            t_def = [timer.time(f, b_, args.reps) for f, b_ in zip(fns, nbs)]

            def time_cand(cand):
                skel_force_variant(sk_id, *cand)
                try:
                    return [timer.time(f, b_, args.reps) for f, b_ in zip(fns, nbs)]
                finally:
                    skel_force_variant(sk_id, -1)

            best, best_ratio, t_best = None, 1.0 - args.margin, t_def
            for cand in candidates(inst.sk_name):
                try:
                    ts = time_cand(cand)
                except SkelError as e:
                    if args.verbose:
                        print(f"    {inst.name} n={n} {cand}: not applicable ({e})", flush=True)
                    continue
                ratio = max(t / td for t, td in zip(ts, t_def))   # the worse of the two points
                if args.verbose:
                    print(f"    {inst.name} n={n} {cand}: {nbs[0] / ts[0] / 1e6:.1f} GB/s (worst ratio {ratio:.3f})",
                          flush=True)
                if ratio < best_ratio:
                    best, best_ratio, t_best = cand, ratio, ts
            if best is not None:
                # confirm against noise (tiny calls last a few microseconds):
                # time both again and keep the candidate only if it still wins
                skel_force_variant(sk_id, -1)
                t_def2 = [timer.time(f, b_, args.reps) for f, b_ in zip(fns, nbs)]
                t_best2 = time_cand(best)
                if not max(t / td for t, td in zip(t_best2, t_def2)) < 1.0 - args.margin:
                    best = None
            return best, t_def[0], (t_best[0] if best is not None else t_def[0]), nbs[0]

        if args.adaptive:
            measured = adaptive_sizes(inst.sizes, lambda n: decide(n), key=lambda r: r[0])
        else:
            measured = {n: decide(n) for n in inst.sizes}
        samples_taken += sum(1 for v in measured.values() if v is not None)
        samples_full += len(inst.sizes)
        last = None
        for n in inst.sizes:
            r = measured.get(n)
            sampled = r is not None
            r = r if sampled else last          # unsampled: its sampled neighbours agree
            last = r
            best, t_def, t_tuned, nb = r
            if best is not None:
                lines.append(f"{sk_id} {inst.fn_key} {inst.dtype} {bucket(n)} {inst.radius} {inst.residency} "
                             f"{best[0]} {best[1]} {best[2]} {best[3]}")
                chosen = best
            else:
                # record that the default won here, so this bucket never
                # inherits a neighbouring bucket's choice by extrapolation
                lines.append(f"{sk_id} {inst.fn_key} {inst.dtype} {bucket(n)} {inst.radius} {inst.residency} -1 0 0 0")
                chosen = "default"
            chosen_all.append((inst.name, n, chosen))
            if sampled:
                report.append(f"| {inst.name} | {n} | {nb / t_def / 1e6:.1f} | {nb / t_tuned / 1e6:.1f} | "
                              f"{t_def / t_tuned:.3f} | {chosen} |")
            else:
                report.append(f"| {inst.name} | {n} | - | - | - | {chosen} (not sampled: neighbours agree) |")
            print(report[-1], flush=True)
    if not args.only or "batched" in args.only:
        total, fn, nb = batched_instance()
        sk_id = SK["batched"]
        t_def = timer.time(fn, nb, args.reps)
        best, t_best = None, t_def
        for cand in candidates("batched"):
            skel_force_variant(sk_id, *cand)
            try:
                t = timer.time(fn, nb, args.reps)
            except SkelError:
                continue
            finally:
                skel_force_variant(sk_id, -1)
            if t < t_best:
                best, t_best = cand, t
        if best is not None and t_best < t_def * (1.0 - args.margin):
            lines.append(f"{sk_id} 0 {F32} {bucket(total)} 0 0 {best[0]} {best[1]} {best[2]} {best[3]}")
        else:
            lines.append(f"{sk_id} 0 {F32} {bucket(total)} 0 0 -1 0 0 0")
        report.append(f"| batched sumsq+scan f32 | {total} | {nb / t_def / 1e6:.1f} | {nb / t_best / 1e6:.1f} | "
                      f"{t_def / t_best:.3f} | {best if best and t_best < t_def * (1 - args.margin) else 'default'} |")
        print(report[-1], flush=True)
    with open(args.out, "w") as f:
        f.write("\n".join(lines) + "\n")
    report.append(f"\nsize buckets sampled: {samples_taken} of {samples_full}"
                  + (" (adaptive)" if args.adaptive else ""))
    return report


def table_key(inst, n) -> tuple:
    return (SK[inst.sk_name], inst.fn_key, inst.dtype, bucket(n), inst.radius, inst.residency)


def set_table_entry(path: str, key: tuple, choice) -> None:
    """Rewrites the table line of `key` (adding one if the bucket had none)
    with `choice` = (variant, block, ept, tile), variant -1 = the default."""
    lines = open(path).read().splitlines()
    new = " ".join(str(v) for v in (*key, *choice))
    for i, ln in enumerate(lines):
        f = ln.split()
        if ln.startswith("#") or len(f) != 10:
            continue
        if tuple(int(v) for v in f[:6]) == key:
            lines[i] = new
            break
    else:
        lines.append(new)
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def validate(args):
    """Tuned table vs defaults at sizes between the buckets (n = 2 * 4^k).

    Each point times the default twice around the table (the two default
    timings give the point's noise ratio).  A point where the table is slower
    than the default by more than the margin re-decides its bucket: the
    table's choice and the default are timed again with three times the
    repetitions at the bucket's own size and at the failing size, and unless
    the choice is within the margin of the default at both, the bucket is set
    to the default in the table.  The point is then timed again with the
    corrected table."""
    timer = Timer()
    rows = ["| skeleton instance | n (between buckets) | default GB/s | table GB/s | table / default | "
            "default / default | re-decided |", "|---|---|---|---|---|---|---|"]
    worst, noise = 10.0, 10.0
    redecided = []
    for inst in instances(args.nmax_log2):
        if args.only and not any(s in inst.name for s in args.only):
            continue
        for n in [2 * s for s in inst.sizes if 2 * s <= inst.nmax]:
            if inst.sk_name == "mapoverlap2d":
                continue   # square grids only: between-bucket sizes are not squares
            fn = inst.make(n)
            nb = inst.nbytes(n)
            skel_load_dispatch_table(None)
            t_def = timer.time(fn, nb, args.reps)
            skel_load_dispatch_table(args.out)
            t_tab = timer.time(fn, nb, args.reps)
            skel_load_dispatch_table(None)
            t_def2 = timer.time(fn, nb, args.reps)
            point_noise = min(t_def, t_def2) / max(t_def, t_def2)
            t_def = min(t_def, t_def2)
            note = ""
            if t_def / t_tab < 1.0 - args.margin:
                pts = [n // 2, n]
                fns = [inst.make(q) for q in pts]
                nbs = [inst.nbytes(q) for q in pts]
                reps3 = 3 * args.reps
                td = [timer.time(f, b_, reps3) for f, b_ in zip(fns, nbs)]
                skel_load_dispatch_table(args.out)
                tt = [timer.time(f, b_, reps3) for f, b_ in zip(fns, nbs)]
                if max(a / b for a, b in zip(tt, td)) > 1.0 + args.margin:
                    set_table_entry(args.out, table_key(inst, n), (-1, 0, 0, 0))
                    redecided.append((inst.name, n))
                    note = "bucket set to the default"
                    skel_load_dispatch_table(args.out)
                    t_tab = timer.time(fn, nb, args.reps)
                    skel_load_dispatch_table(None)
                    t_def = min(t_def, timer.time(fn, nb, args.reps))
                else:
                    note = "choice kept (within the margin on re-timing)"
                    skel_load_dispatch_table(args.out)
                    t_tab = min(t_tab, timer.time(fn, nb, reps3))
            worst = min(worst, t_def / t_tab)
            noise = min(noise, point_noise)
            rows.append(f"| {inst.name} | {n} | {nb / t_def / 1e6:.1f} | {nb / t_tab / 1e6:.1f} | {t_def / t_tab:.3f} | "
                        f"{point_noise:.3f} | {note} |")
            print(rows[-1], flush=True)
    skel_load_dispatch_table(args.out)
    rows.append(f"\nworst table/default speed ratio between buckets: {worst:.3f}; noise floor (worst ratio of two "
                f"timings of the default at one point): {noise:.3f}; buckets re-decided: {len(redecided)}"
                + ("" if not redecided else " (" + ", ".join(f"{a} at {b}" for a, b in redecided) + ")"))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "dispatch_gb300.tbl"))
    ap.add_argument("--report", default=None)
    ap.add_argument("--reps", type=int, default=15)
    ap.add_argument("--margin", type=float, default=0.03)
    ap.add_argument("--nmax-log2", type=int, default=28)
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--no-validate", action="store_true")
    ap.add_argument("--verbose", action="store_true", help="log every candidate's time")
    ap.add_argument("--adaptive", action="store_true",
                    help="sample size buckets adaptively (refine only where the choice changes)")
    args = ap.parse_args()
    t0 = time.time()
    report = tune(args)
    val = [] if args.no_validate else validate(args)
    if args.report:
        with open(args.report, "w") as f:
            f.write(f"# Tuned vs default variants on {torch.cuda.get_device_name()}\n\n")
            f.write("Command: `python -m paper_1405_2915_gb300.tune " + " ".join(sys.argv[1:]) + "`\n\n")
            f.write("Device time per call, median of %d runs (CUDA events), L2 flushed before each run when the "
                    "operands fit in L2.  GB/s = algorithmic bytes / time.\n\n" % args.reps)
            f.write("\n".join(report) + "\n\n## Sizes between the tuned buckets\n\n" + "\n".join(val) + "\n")
    print(f"tuned in {time.time() - t0:.0f} s -> {args.out}", file=sys.stderr)


if __name__ == "__main__":
    main()
