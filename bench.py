"""Benchmark of the skeleton hot path on GB300.

One step = one pass of every skeleton of the hot path over one batch of
synthetic input at the size sweep's largest point, n = 2^28 elements
(float32 / int32, seeded, inputs resident in HBM and each larger than L2):

    map axpy (a = 2.5)            12 B/elem     reduce sum, reduce max   4 B/elem each
    mapreduce dot                  8 B/elem     scan incl int32, excl f32 8 B/elem each
    mapoverlap 2D 9pt, 5pt clamp   8 B/point (16384 x 16384 grid, U[0,1])
    mapoverlap 1D r=8 clamp        8 B/elem     maparray rowdot (16384 x 16384)  4 B/elem
    maparray gather (A = 2^20)     8 B/elem     batched sumsq + scan (4096 uneven instances) 8 B/elem
    backward: map tanh 12 B/elem, reverse scan 8 B/elem, transposed 9pt stencil 8 B/point

value = algorithmic bytes of the step / step time (GB/s, whole job over all
ranks).  Per-skeleton GB/s, the tuned-vs-default speedup, the roofline of
the dominant kernel, the end-to-end number through host buffers and the
oracle's CPU throughput are added to the one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

METRIC = "achieved HBM GB/s and fraction of GB300 peak per skeleton; tuned-vs-default-variant speedup"
N = 1 << 28
SIDE = 1 << 14
ROWDOT_M = 1 << 14
GATHER_M = 1 << 20
BATCH_B = 4096
R1D = 8
TABLE = os.path.join(ROOT, "paper_1405_2915_gb300", "dispatch_gb300.tbl")


def workload_config():
    return {"workload": "skeleton hot path, n = 2^28 per skeleton (grids 16384^2, rowdot 16384x16384, "
                        "4096 uneven instances in [64, 2^20])",
            "n": N, "grid": [SIDE, SIDE], "batched_instances": BATCH_B,
            "l2": "no flush: every input is >= 1 GiB, larger than the 129 MB L2",
            "parallelism": "replicas (one independent workload per GPU)"}


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                mhz.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


# ---------------------------------------------------------------- workload --
class Workload:
    """Inputs (device tensors wrapped as containers) and the step's calls."""

    def __init__(self, sk, torch, rank: int):
        self.sk, self.torch = sk, torch
        dev = torch.device("cuda")
        s = 1000 * rank
        t0 = time.time()
        f32 = lambda a: torch.from_numpy(a).to(dev)
        self.x = f32(syn.uniform_f32(syn.SEED_X + s, N))
        self.y = f32(syn.uniform_f32(syn.SEED_Y + s, N))
        self.xi = f32(syn.uniform_int(syn.SEED_INT + s, N, 0, 100))
        self.grid = f32(syn.uniform_f32(syn.SEED_GRID + s, N, 0.0, 1.0)).view(SIDE, SIDE)
        self.M = f32(syn.uniform_f32(syn.SEED_MAT + s, N)).view(N // ROWDOT_M, ROWDOT_M)
        self.A = f32(syn.uniform_f32(syn.SEED_X + s + 7, ROWDOT_M))
        self.Ag = f32(syn.uniform_f32(syn.SEED_X + s + 8, GATHER_M))
        self.idx = f32(syn.uniform_int(syn.SEED_IDX + s, N, 0, GATHER_M - 1))
        lens = syn.loguniform_lengths(syn.SEED_BATCH_LEN + s, BATCH_B)
        off = syn.csr_offsets(lens)
        self.total = int(off[-1])
        self.bv = f32(syn.uniform_f32(syn.SEED_BATCH_VAL + s, self.total))
        self.boff = f32(off)
        self.gen_s = time.time() - t0
        e = lambda shape, dt=torch.float32: torch.empty(shape, dtype=dt, device=dev)
        self.oA, self.oB = e(N), e(N)
        self.oI = e(N, torch.int32)
        self.oG, self.oG2 = e((SIDE, SIDE)), e((SIDE, SIDE))
        self.rd = e(N // ROWDOT_M)
        self.bres, self.bsc = e(BATCH_B), e(self.total)
        self.r1 = e(1)
        C = sk.Container.from_tensor
        self.c = {k: C(getattr(self, k)) for k in
                  ("x", "y", "xi", "grid", "M", "A", "Ag", "idx", "bv", "boff", "oA", "oB", "oI", "oG", "oG2",
                   "rd", "bres", "bsc", "r1")}

    def calls(self):
        """(name, algorithmic bytes, thunk) for every call of one step."""
        sk, c, n = self.sk, self.c, N
        return [
            ("map_axpy", 12 * n, lambda: sk.skel_map("axpy", [c["x"], c["y"]], c["oA"], [2.5])),
            ("reduce_sum", 4 * n, lambda: sk.skel_reduce("add", c["x"], c["r1"], host=False)),
            ("reduce_max", 4 * n, lambda: sk.skel_reduce("max", c["x"], c["r1"], host=False)),
            ("mapreduce_dot", 8 * n, lambda: sk.skel_mapreduce("mul", "add", [c["x"], c["y"]], c["r1"], host=False)),
            ("scan_incl_i32", 8 * n, lambda: sk.skel_scan("add", True, c["xi"], c["oI"])),
            ("scan_excl_f32", 8 * n, lambda: sk.skel_scan("add", False, c["x"], c["oB"])),
            ("mapoverlap2d_9pt", 8 * n, lambda: sk.skel_mapoverlap("stencil9", 1, None, "clamp", c["grid"], c["oG"])),
            ("mapoverlap2d_5pt", 8 * n, lambda: sk.skel_mapoverlap("stencil5", 1, None, "clamp", c["grid"], c["oG2"])),
            ("mapoverlap1d_r8", 8 * n, lambda: sk.skel_mapoverlap("stencil1d", R1D, None, "clamp", c["x"], c["oA"])),
            ("maparray_rowdot", 4 * n + 4 * ROWDOT_M + 4 * (n // ROWDOT_M),
             lambda: sk.skel_maparray("rowdot", c["A"], c["M"], c["rd"])),
            ("maparray_gather", 8 * n, lambda: sk.skel_maparray("gather", c["Ag"], c["idx"], c["oB"])),
            ("batched_sumsq_scan", 8 * self.total + 8 * (BATCH_B + 1) + 4 * BATCH_B,
             lambda: sk.skel_batched(c["bv"], c["boff"], c["bres"], c["bsc"], True)),
            ("map_tanh_bwd", 12 * n, lambda: sk.skel_map_bwd("tanh", [c["y"]], c["x"], [c["oA"]], [1.0])),
            ("scan_bwd_f32", 8 * n, lambda: sk.skel_scan_bwd("add", True, c["x"], c["oB"])),
            ("mapoverlap2d_9pt_bwd", 8 * n, lambda: sk.skel_mapoverlap_bwd("stencil9", 1, None, "clamp", c["grid"], c["oG"])),
        ]


    def extra_calls(self):
        """Calls outside the step that profiling runs may name with --only:
        the ten-step 9-point chain (composed, as the table chooses it) and
        the fused Map -> MapOverlap -> MapReduce chain, on the step's grid."""
        sk, c, n = self.sk, self.c, N
        return [
            ("chain_9pt_x10", 8 * n * 10,
             lambda: sk.skel_mapoverlap_chain("stencil9", None, "clamp", 10, c["grid"], c["oG2"], c["oG"])),
            ("compose_tanh_9pt", 4 * n,
             lambda: sk.skel_compose_map_stencil_sumsq("tanh", "stencil9", c["grid"], result_dev=c["r1"], host=False)),
        ]


def run_steps(torch, calls, steps, stream, per_call=True):
    """Runs `steps` steps; returns (total ms, {name: summed ms})."""
    E = torch.cuda.Event
    if per_call:
        evs = [[E(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(steps)]
    start, end = E(enable_timing=True), E(enable_timing=True)
    start.record(stream)
    for s in range(steps):
        if per_call:
            evs[s][0].record(stream)
        for k, (_, _, fn) in enumerate(calls):
            fn()
            if per_call:
                evs[s][k + 1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    per = {}
    if per_call:
        for k, (name, _, _) in enumerate(calls):
            per[name] = sum(evs[s][k].elapsed_time(evs[s][k + 1]) for s in range(steps))
    return start.elapsed_time(end), per


def max_over_ranks(ms: float, device: str = "cuda") -> float:
    """The slowest rank's time (the whole job is done when the last rank
    is); a single process returns its own time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(step_bytes: int, world: int, steps: int, ms_max: float) -> float:
    """Aggregate GB/s over all ranks: every rank moves step_bytes per step
    (weak scaling), and the job takes the slowest rank's time."""
    return world * step_bytes * steps / (ms_max * 1e-3) / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def committed_traffic(kernel_key: str):
    """dram bytes per launch of a kernel from the committed ncu summary, if any."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = line.split()
        if len(parts) >= 2 and not line.startswith("#") and parts[0] == kernel_key:
            return float(parts[1])
    return None


# ------------------------------------------------------------- CPU oracle --
def oracle_sample_step(sample: int):
    """One bounded sample of the step on the host: every skeleton of the step
    run by the float64 oracle on `sample` elements.  Returns (seconds, bytes),
    the bytes counted with the same per-element figures as the GPU step."""
    import oracle
    n = sample
    side = int(np.sqrt(n))
    x, y = syn.uniform_f32(syn.SEED_X, n), syn.uniform_f32(syn.SEED_Y, n)
    xi = syn.uniform_int(syn.SEED_INT, n, 0, 100)
    g = syn.uniform_f32(syn.SEED_GRID, side * side, 0.0, 1.0).reshape(side, side)
    m = 1 << 10
    M = syn.uniform_f32(syn.SEED_MAT, (n // m) * m).reshape(n // m, m)
    A = syn.uniform_f32(syn.SEED_X + 7, m)
    Ag = syn.uniform_f32(syn.SEED_X + 8, GATHER_M)
    idx = syn.uniform_int(syn.SEED_IDX, n, 0, GATHER_M - 1)
    lens = syn.loguniform_lengths(syn.SEED_BATCH_LEN, 64, 64, 1 << 16)
    off = syn.csr_offsets(lens)
    bv = syn.uniform_f32(syn.SEED_BATCH_VAL, int(off[-1]))
    w9, w5 = oracle.stencil_weights("9pt"), oracle.stencil_weights("5pt")
    # the library's default 1D weights: binomial C(2r, k) / 4^r
    w1 = (np.array([math.comb(2 * R1D, k) for k in range(2 * R1D + 1)], np.float64) / 4 ** R1D).astype(np.float32)
    t0 = time.perf_counter()
    oracle.map_f32("axpy", x, y, a=2.5)
    oracle.reduce_f32("add", x)
    oracle.reduce_f32("max", x)
    oracle.mapreduce_f32("mul", x, y)
    oracle.scan_i32(xi, True)
    oracle.scan_f32(x, False)
    oracle.mapoverlap2d_f32(g, 1, w9, "clamp")
    oracle.mapoverlap2d_f32(g, 1, w5, "clamp")
    oracle.mapoverlap1d_f32(x, R1D, w1, "clamp")
    oracle.rowdot_f32(A, M)
    oracle.gather_f32(Ag, idx)
    oracle.batched_f32(bv, off, True)
    oracle.map_bwd_f32("tanh", x, y)
    oracle.scan_bwd_f32(x, True)
    oracle.mapoverlap2d_bwd_f32(g, 1, w9, "clamp")
    dt = time.perf_counter() - t0
    nb = (12 + 4 + 4 + 8 + 8 + 8 + 8 + 8 + 8 + 4 + 8 + 12 + 8 + 8) * n + 8 * int(off[-1])
    return dt, nb


def reference_sample(n_steps: int, budget_s: float = 150.0, cap_s: float = 8.0) -> int:
    """Elements per sampled step so that n_steps oracle steps take about
    min(cap_s, budget_s / n_steps) seconds each (a power of two in [2^16, 2^26])."""
    t1, _ = oracle_sample_step(1 << 18)
    target = min(cap_s, budget_s / max(1, n_steps))
    k = int(np.clip(np.floor(np.log2(max(target / max(t1, 1e-6), 1e-3))) + 18, 16, 26))
    return 1 << k


def cpu_baseline(sample: int = 1 << 25):
    dt, nb = oracle_sample_step(sample)
    return {"value": nb / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "cpu_model": host_model(),
            "sample": f"every skeleton of the step on n = {sample} elements (float64 oracle, one thread), "
                      f"{dt:.1f} s"}


# ------------------------------------------------ parallel CPU baseline --
def cpu_parallel_leg(sample_log2: int = 26, reps: int = 3):
    """The step's calls by the parallel float32 CPU baseline (std::thread over
    the cores of this process's affinity mask) on n = 2^sample_log2 elements
    per call (grids 2^(k/2) square, rowdot rows of 2^(k/2), the batched
    instances of the workload with lengths scaled by the same factor), each
    call the median of `reps` runs; GB/s of the same algorithmic bytes as the
    GPU step."""
    import cpu_baseline as cb
    n = 1 << sample_log2
    side = 1 << (sample_log2 // 2)
    x, y = syn.uniform_f32(syn.SEED_X, n), syn.uniform_f32(syn.SEED_Y, n)
    xi = syn.uniform_int(syn.SEED_INT, n, 0, 100)
    g = syn.uniform_f32(syn.SEED_GRID, n, 0.0, 1.0).reshape(side, side)
    M = syn.uniform_f32(syn.SEED_MAT, n).reshape(n // side, side)
    A = syn.uniform_f32(syn.SEED_X + 7, side)
    Ag = syn.uniform_f32(syn.SEED_X + 8, GATHER_M)
    idx = syn.uniform_int(syn.SEED_IDX, n, 0, GATHER_M - 1)
    scale = n / N
    lens = np.maximum(1, (syn.loguniform_lengths(syn.SEED_BATCH_LEN, BATCH_B) * scale).astype(np.int64))
    off = syn.csr_offsets(lens)
    bv = syn.uniform_f32(syn.SEED_BATCH_VAL, int(off[-1]))
    w9 = np.outer([1, 2, 1], [1, 2, 1]).astype(np.float32) / np.float32(16)
    w5 = np.array([[0, 1, 0], [1, 4, 1], [0, 1, 0]], np.float32) / np.float32(8)
    w1 = (np.array([math.comb(2 * R1D, k) for k in range(2 * R1D + 1)], np.float64) / 4 ** R1D).astype(np.float32)
    oA, oB, oI = np.empty_like(x), np.empty_like(x), np.empty_like(xi)
    oG, rd = np.empty_like(g), np.empty(n // side, np.float32)
    bres, bsc = np.empty(BATCH_B, np.float32), np.empty_like(bv)
    tb = int(off[-1])
    calls = [
        ("map_axpy", 12 * n, lambda: cb.map_axpy(x, y, 2.5, oA)),
        ("reduce_sum", 4 * n, lambda: cb.reduce_sum(x)),
        ("reduce_max", 4 * n, lambda: cb.reduce_max(x)),
        ("mapreduce_dot", 8 * n, lambda: cb.dot(x, y)),
        ("scan_incl_i32", 8 * n, lambda: cb.scan_i32(xi, True, oI)),
        ("scan_excl_f32", 8 * n, lambda: cb.scan_f32(x, False, oB)),
        ("mapoverlap2d_9pt", 8 * n, lambda: cb.stencil2d(g, w9, oG)),
        ("mapoverlap2d_5pt", 8 * n, lambda: cb.stencil2d(g, w5, oG)),
        ("mapoverlap1d_r8", 8 * n, lambda: cb.stencil1d(x, R1D, w1, oA)),
        ("maparray_rowdot", 4 * n + 4 * side + 4 * (n // side), lambda: cb.rowdot(A, M, rd)),
        ("maparray_gather", 8 * n, lambda: cb.gather(Ag, idx, oB)),
        ("batched_sumsq_scan", 8 * tb + 8 * (BATCH_B + 1) + 4 * BATCH_B, lambda: cb.batched(bv, off, bres, bsc)),
        ("map_tanh_bwd", 12 * n, lambda: cb.map_tanh_bwd(x, y, oA)),
        ("scan_bwd_f32", 8 * n, lambda: cb.scan_bwd_f32(x, oB)),
        ("mapoverlap2d_9pt_bwd", 8 * n, lambda: cb.stencil2d_bwd(g, w9, oG)),
    ]
    per, tot_t, tot_b = {}, 0.0, 0
    for name, nb, fn in calls:
        fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        t = statistics.median(ts)
        per[name] = round(nb / t / 1e9, 2)
        tot_t += t
        tot_b += nb
    host = cb.host_cpu()
    return {"value": round(tot_b / tot_t / 1e9, 2), "unit": "GB/s", "cores": cb.cores(), "cpu_model": host["model"],
            "kind": "parallel float32 CPU baseline (std::thread, cpu_baseline/cpu_parallel.cpp)",
            "sample": f"every call of the step on n = 2^{sample_log2} elements (grids {side}^2), median of {reps} "
                      f"runs per call, {tot_t:.2f} s per step", "per_call_GB/s": per}


def host_model() -> str:
    import cpu_baseline as cb
    return cb.host_cpu()["model"]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample = reference_sample(args.steps + args.warmup)
    for _ in range(args.warmup):
        oracle_sample_step(sample)
    tot_t = tot_b = 0.0
    for _ in range(args.steps):
        dt, nb = oracle_sample_step(sample)
        tot_t += dt
        tot_b += nb
    value = tot_b / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "cpu_model": host_model(),
                             "sample": f"each step: every skeleton of the step on n = {sample} elements "
                                       "(float64 oracle, one thread)"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- e2e ----
def parse_cpulist(text: str) -> set:
    """'0-3,8,10-11' -> {0, 1, 2, 3, 8, 10, 11}."""
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_to_gpu_local_cpus(torch, device_index: int):
    """Run this process on the CPUs next to the GPU, so that pinned host
    buffers (placed on first touch) sit in the memory attached to the CPU
    that links to this GPU. Returns the CPUs kept, or None if unchanged."""
    p = torch.cuda.get_device_properties(device_index)
    try:
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bdf}/local_cpulist") as f:
            local = parse_cpulist(f.read())
    except (AttributeError, OSError, ValueError):
        return None
    keep = local & os.sched_getaffinity(0)
    if not keep or keep == os.sched_getaffinity(0):
        return None
    os.sched_setaffinity(0, keep)
    return sorted(keep)


def e2e_run(sk, torch, steps, stream):
    """The same step through the public API with host buffers: inputs live in
    pinned host memory and reach the device through the containers (H2D
    inside the timed region: prefetched on a copy stream in order of first
    use, so that copies overlap the calls), and every result is copied back
    to the host (D2H on a second copy stream as soon as it is final)."""
    cpus = bind_to_gpu_local_cpus(torch, torch.cuda.current_device())
    dev = torch.device("cuda")
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h = {}
    h["x"] = pin(syn.uniform_f32(syn.SEED_X, N))
    h["y"] = pin(syn.uniform_f32(syn.SEED_Y, N))
    h["xi"] = pin(syn.uniform_int(syn.SEED_INT, N, 0, 100))
    h["grid"] = pin(syn.uniform_f32(syn.SEED_GRID, N, 0.0, 1.0).reshape(SIDE, SIDE))
    h["M"] = pin(syn.uniform_f32(syn.SEED_MAT, N).reshape(N // ROWDOT_M, ROWDOT_M))
    h["A"] = pin(syn.uniform_f32(syn.SEED_X + 7, ROWDOT_M))
    h["Ag"] = pin(syn.uniform_f32(syn.SEED_X + 8, GATHER_M))
    h["idx"] = pin(syn.uniform_int(syn.SEED_IDX, N, 0, GATHER_M - 1))
    lens = syn.loguniform_lengths(syn.SEED_BATCH_LEN, BATCH_B)
    off = syn.csr_offsets(lens)
    total = int(off[-1])
    h["bv"] = pin(syn.uniform_f32(syn.SEED_BATCH_VAL, total))
    h["boff"] = pin(off)
    C = sk.Container
    ci = {k: C.from_host(v.numpy()) for k, v in h.items()}
    outs = {"oA": (N,), "oB": (N,), "oG": (SIDE, SIDE), "oG2": (SIDE, SIDE), "rd": (N // ROWDOT_M,),
            "bres": (BATCH_B,), "bsc": (total,), "r1": (1,)}
    co = {k: C.empty(s) for k, s in outs.items()}
    co["oI"] = C.empty((N,), np.int32)
    c = {**ci, **co}
    # (call, results final after it): each result starts its copy back to the
    # host as soon as no later call of the step writes it
    calls = [
        (lambda: sk.skel_map("axpy", [c["x"], c["y"]], c["oA"], [2.5]), []),
        (lambda: sk.skel_reduce("add", c["x"], c["r1"], host=False), []),
        (lambda: sk.skel_reduce("max", c["x"], c["r1"], host=False), []),
        (lambda: sk.skel_mapreduce("mul", "add", [c["x"], c["y"]], c["r1"], host=False), ["r1"]),
        (lambda: sk.skel_scan("add", True, c["xi"], c["oI"]), ["oI"]),
        (lambda: sk.skel_scan("add", False, c["x"], c["oB"]), []),
        (lambda: sk.skel_mapoverlap("stencil9", 1, None, "clamp", c["grid"], c["oG"]), []),
        (lambda: sk.skel_mapoverlap("stencil5", 1, None, "clamp", c["grid"], c["oG2"]), ["oG2"]),
        (lambda: sk.skel_mapoverlap("stencil1d", R1D, None, "clamp", c["x"], c["oA"]), []),
        (lambda: sk.skel_maparray("rowdot", c["A"], c["M"], c["rd"]), ["rd"]),
        (lambda: sk.skel_maparray("gather", c["Ag"], c["idx"], c["oB"]), []),
        (lambda: sk.skel_batched(c["bv"], c["boff"], c["bres"], c["bsc"], True), ["bres", "bsc"]),
        (lambda: sk.skel_map_bwd("tanh", [c["y"]], c["x"], [c["oA"]], [1.0]), ["oA"]),
        (lambda: sk.skel_scan_bwd("add", True, c["x"], c["oB"]), ["oB"]),
        (lambda: sk.skel_mapoverlap_bwd("stencil9", 1, None, "clamp", c["grid"], c["oG"]), ["oG"]),
    ]
    read_back = ["oA", "oB", "oI", "oG", "oG2", "rd", "bres", "bsc", "r1"]
    first_use = ["x", "y", "xi", "grid", "A", "M", "Ag", "idx", "bv", "boff"]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

    def one_step():
        for k in ci:                       # the host copies hold this step's inputs
            ci[k].mark(sk.UNIT_HOST)
        for k in first_use:                # inputs start moving in order of first use
            ci[k].prefetch(sk.UNIT_DEVICE, h2d)
        for fn, done in calls:
            fn()
            for k in done:                 # final results start moving back at once
                c[k].prefetch(sk.UNIT_HOST, d2h)
        for k in read_back:                # host reads wait for their copies
            c[k].host_ptr(sk.READ, stream)

    def stats():
        hs = [c[k].stats() for k in c]
        return sum(s["h2d_bytes"] for s in hs), sum(s["d2h_bytes"] for s in hs)

    for _ in range(2):                     # warm-up (allocates device and pinned copies)
        one_step()
    b0 = stats()
    torch.cuda.synchronize()
    per_step = []
    for _ in range(steps):
        t0 = time.perf_counter()
        one_step()
        torch.cuda.synchronize()
        per_step.append(time.perf_counter() - t0)
    dt = sum(per_step) / steps
    b1 = stats()
    for v in c.values():
        v.close()
    return dt, (b1[0] - b0[0]) / steps, (b1[1] - b0[1]) / steps, cpus, per_step


# ------------------------------------------------- Coulombic potential --
COUL_SIDE, COUL_ATOMS, COUL_H = 4096, 4096, 0.125
SFU_PER_SM_CLK = 16          # reciprocal square roots per SM per clock (4 per SM sub-partition)


def coulomb_leg(sk, torch, stream, clocks, reps: int = 5):
    """The Coulombic potential grid (MapArray over grid positions), a widening
    beyond the step: 4096 x 4096 points, 4096 atoms.  Bound by the SFU rate
    (one reciprocal square root per point-atom pair); reported apart from
    the step's GB/s."""
    dev = torch.device("cuda")
    m, side = COUL_ATOMS, COUL_SIDE
    a = np.empty((m, 4), np.float32)
    a[:, 0] = syn.uniform_f32(syn.SEED_X + 11, m, 0.0, 1.0) * np.float32(side * COUL_H)
    a[:, 1] = syn.uniform_f32(syn.SEED_X + 12, m, 0.0, 1.0) * np.float32(side * COUL_H)
    a[:, 2] = syn.uniform_f32(syn.SEED_X + 13, m, 0.5, 4.5)
    a[:, 3] = syn.uniform_f32(syn.SEED_X + 14, m)
    atoms = sk.Container.from_tensor(torch.from_numpy(a).to(dev))
    out_t = torch.empty((side, side), dtype=torch.float32, device=dev)
    out = sk.Container.from_tensor(out_t)
    call = lambda: sk.skel_maparray_grid("coulomb", atoms, out, (COUL_H, 0.0))
    for _ in range(2):
        call()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    pairs = float(side) * side * m
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = SFU_PER_SM_CLK * sms * mhz * 1e6
    achieved = pairs / (ms * 1e-3)
    atoms.close()
    out.close()
    return {"metric": "point-atom pairs per second", "value": round(achieved / 1e12, 3), "unit": "Tpairs/s",
            "ms": round(ms, 3), "config": {"grid": [side, side], "atoms": m, "h": COUL_H},
            "roofline": {"bound": "alu", "unit": "Tpairs/s", "peak": round(peak / 1e12, 3),
                         "frac": round(achieved / peak, 3),
                         "peak_basis": f"{SFU_PER_SM_CLK} rsqrt/clk/SM x {sms} SMs x {mhz:.0f} MHz"},
            "variant": list(sk.skel_last_variant("maparray"))}


# ----------------------------------------- the other workload configurations --
def _event_ms(torch, stream, fn, reps, lead_ns=0):
    """Median device time of fn over reps runs.  lead_ns > 0 puts a sleep
    kernel of about that length ahead of each run, so that the host's time
    to enqueue the run's launches is not counted as device time."""
    ts = []
    for _ in range(reps):
        if lead_ns:
            torch.cuda._sleep(int(lead_ns * 2))           # about 2 cycles per ns at the GB300's clocks
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def launch_floor(sk, torch, stream, count: int = 200) -> float:
    """Microseconds per launch of an empty kernel, launched back to back
    (after a sleep kernel that covers the host's enqueue time)."""
    sk.skel_probe_empty_launches(16)
    ms = _event_ms(torch, stream, lambda: sk.skel_probe_empty_launches(count), 5, lead_ns=2_000_000)
    return ms * 1e3 / count


def l2_random_rate(sk, torch, stream, m: int = 1 << 20, reads: int = 1 << 28):
    """Random 4-byte reads per second from an L2-resident table of m floats
    (the gather's table size): the gather's measured ceiling."""
    dev = torch.device("cuda")
    table = torch.from_numpy(syn.uniform_f32(syn.SEED_X + 8, m)).to(dev)
    sink = torch.zeros(1, device=dev)
    made = sk.skel_probe_l2_random(table, reads, sink)
    ms = _event_ms(torch, stream, lambda: sk.skel_probe_l2_random(table, reads, sink), 5)
    return made / (ms * 1e-3), ms


def chains_leg(sk, torch, stream, steps: int = 10, reps: int = 3):
    """Ten chained 2D MapOverlap calls (5- and 9-point, clamp) on square grids
    of side 512, 2048, 8192 and 16384 from an input valid only in pinned host
    memory: the composed chain (variant and steps per pass from the table)
    against ten single calls; device time of the chain on device-resident
    data, and host-timed end to end (input marked host-valid, chain, result
    read on the host) with and without the final device-to-host read;
    transfers counted over one end-to-end run."""
    res = {}
    for side in (512, 2048, 8192, 16384):
        x = torch.from_numpy(syn.uniform_f32(syn.SEED_GRID, side * side, 0.0, 1.0).reshape(side, side)).pin_memory()
        cin = sk.Container.from_host(x.numpy())
        a, b = sk.Container.empty((side, side)), sk.Container.empty((side, side))
        for kind in ("stencil5", "stencil9"):
            forms = {"composed": lambda: sk.skel_mapoverlap_chain(kind, None, "clamp", steps, cin, b, a)}

            def single():
                src = cin
                for k in range(steps):
                    dst = a if k % 2 == 0 else b
                    sk.skel_mapoverlap(kind, 1, None, "clamp", src, dst)
                    src = dst
            forms["single_calls"] = single
            for fname, fn in forms.items():
                outc = a if fname == "composed" or steps % 2 == 1 else b

                def e2e(read_back):
                    cin.mark(sk.UNIT_HOST)
                    fn()
                    if read_back:
                        outc.host_ptr(sk.READ, stream)
                    else:
                        torch.cuda.synchronize()
                e2e(True)
                s0 = (cin.stats(), outc.stats())
                e2e(True)
                s1 = (cin.stats(), outc.stats())
                fn()                                      # input now device-valid: device time only
                ms_dev = _event_ms(torch, stream, fn, reps, lead_ns=1_000_000)
                variant = list(sk.skel_last_variant("chain2d")) if fname == "composed" else None
                t_in, t_all = [], []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    e2e(False)
                    t_in.append(time.perf_counter() - t0)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    e2e(True)
                    t_all.append(time.perf_counter() - t0)
                key = f"{kind[7:]}pt_{side}sq"
                res.setdefault(key, {})[fname] = {
                    "ms_device": round(ms_dev, 3),
                    "GB/s_per_call": round(8 * side * side * steps / (ms_dev * 1e-3) / 1e9, 1),
                    "ms_e2e_excl_d2h": round(1e3 * statistics.median(t_in), 3),
                    "ms_e2e_incl_d2h": round(1e3 * statistics.median(t_all), 3),
                    "transfers_h2d_d2h": [s1[0]["h2d"] - s0[0]["h2d"], s1[1]["d2h"] - s0[1]["d2h"]],
                    **({"variant": variant} if variant else {})}
            r = res[f"{kind[7:]}pt_{side}sq"]
            r["speedup_composed"] = round(r["single_calls"]["ms_device"] / r["composed"]["ms_device"], 3)
        for c in (cin, a, b):
            c.close()
        del x
    return res


# per-kernel algorithmic bytes per grid point of the composed loss's calls
AUTOGRAD_BYTES = {"fwd_map_tanh": 8, "fwd_mapoverlap_9pt": 8, "fwd_sumsq_stencil": 4, "fwd_row_scan": 8,
                  "fwd_sumsq_scan": 4, "fwd_combine": 0, "bwd_scale": 0, "bwd_sumsq_stencil": 8,
                  "bwd_mapoverlap_9pt": 8, "bwd_sumsq_scan": 8, "bwd_reverse_scan": 8, "bwd_map_tanh_sum": 16}


def autograd_per_kernel(torch, stream, xg, reps: int = 5):
    """Device time and GB/s of every skeleton call of the composed loss's
    forward and backward (events around each call; a sleep kernel ahead of
    each pass keeps the host's enqueue time out of the intervals)."""
    from paper_1405_2915_gb300.autograd import composed_loss
    pts = xg.numel()
    acc = {}
    for _ in range(reps):
        evs = []

        def step(name, fn):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            fn()
            e1.record(torch.cuda.current_stream())
            evs.append((name, e0, e1))
        xg.grad = None
        torch.cuda._sleep(40_000_000)
        composed_loss(xg, step=step).backward()
        torch.cuda.synchronize()
        for name, e0, e1 in evs:
            acc.setdefault(name, []).append(e0.elapsed_time(e1))
    res = {}
    for name, ts in acc.items():
        ms = statistics.median(ts)
        nb = AUTOGRAD_BYTES.get(name, 0) * pts
        res[name] = {"ms": round(ms, 4), **({"GB/s": round(nb / (ms * 1e-3) / 1e9, 1)} if nb else {})}
    return res


def overhead_leg(sk, torch, stream, per_sk):
    """Host cost of a skeleton call (argument checks, table lookup, coherence
    steps of three containers, launch) against a bare launch of the same
    kernel, measured inside the library; as a fraction of the kernel's device
    time for axpy at 2^20, 2^24 and 2^28 elements (Sec. IV: container
    overhead)."""
    us_call, us_launch = sk.skel_probe_call_overhead(200, 1024)
    over = us_call - us_launch
    dev = torch.device("cuda")
    kern = {}
    for k in (20, 24):
        n = 1 << k
        x, y, o = (torch.empty(n, device=dev).uniform_() for _ in range(3))
        cx, cy, co = (sk.Container.from_tensor(t) for t in (x, y, o))
        fn = lambda: sk.skel_map("axpy", [cx, cy], co, [2.5])
        fn()
        kern[f"2^{k}"] = _event_ms(torch, stream, fn, 5, lead_ns=500_000) * 1e3
        for c in (cx, cy, co):
            c.close()
    if "map_axpy" in per_sk:
        kern["2^28"] = per_sk["map_axpy"]["ms"] * 1e3
    return {"us_per_call": round(us_call, 3), "us_per_bare_launch": round(us_launch, 3),
            "overhead_us": round(over, 3),
            "overhead_frac_of_axpy_kernel": {k: round(over / v, 5) for k, v in kern.items()},
            "axpy_kernel_us": {k: round(v, 2) for k, v in kern.items()}}


def config_legs(sk, torch, stream):
    """Measurements of the other workload configurations, reported apart
    from the step: dot at n = 2^20 (latency-bound, cold and warm L2), a
    10-call 9-point stencil chain on 8192^2 (composed vs one call per step),
    the batched instances as one CUDA-graph replay against 2 x 4096 separate
    calls, forward + backward of the composed loss on 8192^2, the composed
    Map -> MapOverlap -> MapReduce chain per call and fused, and the host
    edge variants on host-resident inputs."""
    dev = torch.device("cuda")
    out = {}
    # dot, n = 2^20
    n = 1 << 20
    x = torch.from_numpy(syn.uniform_f32(syn.SEED_X, n)).to(dev)
    y = torch.from_numpy(syn.uniform_f32(syn.SEED_Y, n)).to(dev)
    r = torch.zeros(1, device=dev)
    cx, cy, cr = (sk.Container.from_tensor(t) for t in (x, y, r))
    dot = lambda: sk.skel_mapreduce("mul", "add", [cx, cy], cr, host=False)
    for _ in range(3):
        dot()
    # warm: 20 calls back to back on the device (a sleep kernel ahead of them
    # covers the host's time to enqueue them)
    torch.cuda._sleep(4_000_000)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        dot()
    e1.record(stream)
    e1.synchronize()
    warm = e0.elapsed_time(e1) / 20
    flush = torch.empty(1 << 28, dtype=torch.float32, device=dev)
    cold = []
    for _ in range(10):
        flush.sum()                                   # evict the operands from L2
        cold.append(_event_ms(torch, stream, dot, 1))
    # error against the exact sum: float32 products are exact in float64 and
    # math.fsum rounds the exact sum once
    xh, yh = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
    prods = xh * yh
    exact, abs_sum = math.fsum(prods.tolist()), math.fsum(np.abs(prods).tolist())
    got = float(sk.skel_mapreduce("mul", "add", [cx, cy]))
    l0 = sk.lib.skel_launch_count()
    dot()
    launches = sk.lib.skel_launch_count() - l0
    floor = launch_floor(sk, torch, stream)
    out["dot_2e20"] = {"us_warm": round(warm * 1e3, 2), "us_cold": round(statistics.median(cold) * 1e3, 2),
                       "GB/s_warm": round(8 * n / (warm * 1e-3) / 1e9, 1),
                       "GB/s_cold": round(8 * n / (statistics.median(cold) * 1e-3) / 1e9, 1),
                       "error_ratio": round(abs(got - exact) / (2.0 ** -20 * abs_sum), 4),
                       "error_ratio_def": "|gpu - exact| / (2^-20 * sum |x_i y_i|), exact = math.fsum of the float64 products",
                       "launches_per_call": launches, "variant": list(sk.skel_last_variant("mapreduce")),
                       "launch_floor_us": round(launches * floor, 2),
                       "launch_floor_def": f"{launches} back-to-back launches of an empty kernel ({floor:.2f} us each)"}
    del flush
    out["chains_10x"] = chains_leg(sk, torch, stream)
    # batched: graph replay against per-instance calls
    lens = syn.loguniform_lengths(syn.SEED_BATCH_LEN, BATCH_B)
    off = syn.csr_offsets(lens)
    total = int(off[-1])
    bv = torch.from_numpy(syn.uniform_f32(syn.SEED_BATCH_VAL, total)).to(dev)
    boff = torch.from_numpy(off).to(dev)
    bres, bsc = torch.empty(BATCH_B, device=dev), torch.empty(total, device=dev)
    cv, cof, cre, csc = (sk.Container.from_tensor(v) for v in (bv, boff, bres, bsc))
    plan = sk.Plan(cv, cof, cre, csc, True)
    plan.launch()
    ms_graph = _event_ms(torch, stream, plan.launch, 5)
    views = [(cv.view(int(off[b]), (int(lens[b]),)), csc.view(int(off[b]), (int(lens[b]),)),
              cre.view(b, (1,))) for b in range(BATCH_B) if lens[b] > 0]

    def separate():
        for v, sv, rv in views:
            sk.skel_mapreduce("sq", "add", [v], rv, host=False)
            sk.skel_scan("add", True, v, sv)
    separate()
    ms_sep = _event_ms(torch, stream, separate, 2)
    fused_b = 8 * total + 8 * (BATCH_B + 1) + 4 * BATCH_B
    two_pass_b = 12 * total + 8 * (BATCH_B + 1) + 4 * BATCH_B
    out["batched_4096"] = {"ms_graph": round(ms_graph, 3), "ms_separate_calls": round(ms_sep, 3),
                           "speedup": round(ms_sep / ms_graph, 2), "calls_separate": 2 * len(views),
                           "elements": total,
                           "GB/s_fused_bytes": round(fused_b / (ms_graph * 1e-3) / 1e9, 1),
                           "GB/s_two_pass_bytes": round(two_pass_b / (ms_graph * 1e-3) / 1e9, 1),
                           "bytes_def": "fused: 8 B/elem (read + write once) + offsets and results; "
                                        "two passes: 12 B/elem (the sum of squares reads the values again)",
                           "variant": list(sk.skel_last_variant("batched"))}
    for v, sv, rv in views:
        v.close(); sv.close(); rv.close()
    plan.close()
    for c in (cv, cof, cre, csc):
        c.close()
    # composed loss forward + backward, 8192^2
    from paper_1405_2915_gb300.autograd import composed_loss
    side = 8192
    xg = torch.from_numpy(syn.uniform_f32(syn.SEED_GRAD, side * side).reshape(side, side)).to(dev)
    xg.requires_grad_(True)

    def fwd_bwd():
        xg.grad = None
        composed_loss(xg).backward()
    fwd_bwd()
    ms_ad = _event_ms(torch, stream, fwd_bwd, 5, lead_ns=20_000_000)
    out["autograd_8192sq"] = {"ms_fwd_bwd": round(ms_ad, 3), "per_kernel": autograd_per_kernel(torch, stream, xg)}
    # the composed chain tanh -> 9-point stencil -> sum of squares, 8192^2,
    # per call (three dispatched calls) against fused (one pass)
    cxg = sk.Container.from_tensor(xg.detach())
    rr = torch.zeros(1, device=dev)
    crr = sk.Container.from_tensor(rr)
    comp = {}
    for vname, v in (("per_call", 0), ("fused", 1)):
        sk.skel_force_variant("compose", v)
        try:
            fn = lambda: sk.skel_compose_map_stencil_sumsq("tanh", "stencil9", cxg, result_dev=crr, host=False)
            fn()
            comp[vname] = _event_ms(torch, stream, fn, 5, lead_ns=1_000_000)
        finally:
            sk.skel_force_variant("compose", -1)
    out["compose_8192sq"] = {"ms_per_call": round(comp["per_call"], 3), "ms_fused": round(comp["fused"], 3),
                             "speedup": round(comp["per_call"] / comp["fused"], 2),
                             "fused_GB/s": round(4 * side * side / comp["fused"] / 1e6, 1)}
    out["host_edge_2e26"] = host_edge_leg(sk, torch, stream)
    return out


def host_edge_leg(sk, torch, stream):
    """Map (axpy), Reduce (sum) and MapReduce (dot) on 2^26-element inputs
    valid only in pinned host memory at every call, through each host-edge
    variant (whole copy, chunked copy pipeline, direct reads of host memory):
    ms per call and GB/s of the bytes that cross the host link."""
    n = 1 << 26
    dev = torch.device("cuda")
    hx = torch.from_numpy(syn.uniform_f32(syn.SEED_X, n)).pin_memory()
    hy = torch.from_numpy(syn.uniform_f32(syn.SEED_Y, n)).pin_memory()
    cx, cy = sk.Container.from_host(hx.numpy()), sk.Container.from_host(hy.numpy())
    o, r = torch.empty(n, device=dev), torch.zeros(1, device=dev)
    co, cr = sk.Container.from_tensor(o), sk.Container.from_tensor(r)
    calls = {"map_axpy": (lambda: sk.skel_map("axpy", [cx, cy], co, [2.5]), 8 * n),
             "reduce_sum": (lambda: sk.skel_reduce("add", cx, cr, host=False), 4 * n),
             "mapreduce_dot": (lambda: sk.skel_mapreduce("mul", "add", [cx, cy], cr, host=False), 8 * n)}
    res = {}
    for vname, (v, tile) in {"copy": (0, 0), "chunked_8MiB": (1, 0), "chunked_32MiB": (1, 1),
                             "direct": (2, 0)}.items():
        sk.skel_force_variant("edge", v, 0, 0, tile)
        try:
            for cname, (fn, link_bytes) in calls.items():
                def one():
                    cx.mark(sk.UNIT_HOST)
                    cy.mark(sk.UNIT_HOST)
                    fn()
                one()
                ms = _event_ms(torch, stream, one, 5)
                res.setdefault(cname, {})[vname] = {"ms": round(ms, 3), "link_GB/s": round(link_bytes / ms / 1e6, 1)}
        finally:
            sk.skel_force_variant("edge", -1)
    for c in (cx, cy, co, cr):
        c.close()
    return res


# -------------------------------------------------------------------- main --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-default", action="store_true", help="profiling: skip the default-variant leg")
    ap.add_argument("--no-next", action="store_true", help="profiling: skip the Coulombic-potential leg")
    ap.add_argument("--only", default=None,
                    help="profiling: comma-separated call names; times only those calls (no default-variant, "
                         "e2e or CPU legs)")
    ap.add_argument("--force", action="append", default=[], metavar="SKELETON=V[,BLOCK,EPT,TILE]",
                    help="profiling: force a variant (e.g. scan=5,256,4,0); implies --only semantics for legs")
    ap.add_argument("--n-log2", type=int, default=28, help="profiling: elements per skeleton (even, >= 16)")
    ap.add_argument("--batched-instances", type=int, default=4096, help="profiling: batched instance count")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global N, SIDE, BATCH_B
    if args.n_log2 != 28:
        if args.n_log2 % 2 or args.n_log2 < 16:
            ap.error("--n-log2 must be even and >= 16")
        N, SIDE = 1 << args.n_log2, 1 << (args.n_log2 // 2)
    BATCH_B = args.batched_instances
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_2915_gb300 as sk

    tuned = os.path.exists(TABLE)
    if tuned:
        sk.skel_load_dispatch_table(TABLE)
    wl = Workload(sk, torch, rank)
    calls = wl.calls()
    for f in args.force:
        name, _, spec = f.partition("=")
        try:
            sk.skel_force_variant(name, *[int(v) for v in spec.split(",")])
        except (KeyError, ValueError, TypeError):
            ap.error(f"--force {f}: expected SKELETON=V[,BLOCK,EPT,TILE]")
        args.no_e2e = args.no_cpu = True
    if args.only:
        keep = set(args.only.split(","))
        calls = [c for c in calls + wl.extra_calls() if c[0] in keep]
        if not calls:
            ap.error("--only matched no call")
        args.no_e2e = args.no_cpu = True
    stream = torch.cuda.current_stream()
    step_bytes = sum(b for _, b, _ in calls)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # warm-up, then the timed region (per-call events on the launching stream)
    run_steps(torch, calls, args.warmup, stream, per_call=False)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    barrier()
    l0 = sk.lib.skel_launch_count()
    total_ms, per = run_steps(torch, calls, args.steps, stream)
    launches = sk.lib.skel_launch_count() - l0
    barrier()
    clocks = sampler.stop()
    sk.skel_check_device()
    t_max = max_over_ranks(total_ms)
    ms_step = t_max / args.steps
    value = whole_job_gbs(step_bytes, world, args.steps, t_max)

    # the fixed default variants (empty table), same steps
    if args.only or args.force or args.no_default:
        def_ms, per_def = total_ms, per
    else:
        sk.skel_load_dispatch_table(None)
        run_steps(torch, calls, 3, stream, per_call=False)
        barrier()
        def_ms, per_def = run_steps(torch, calls, args.steps, stream)
        barrier()
        if tuned:
            sk.skel_load_dispatch_table(TABLE)

    hbm, peak_kind = peaks()
    per_sk = {}
    for name, b, _ in calls:
        ms = per[name] / args.steps
        gbs = b / (ms * 1e-3) / 1e9
        per_sk[name] = {"GB/s": round(gbs, 1), "frac": round(gbs / hbm, 3), "ms": round(ms, 4),
                        "default_ms": round(per_def[name] / args.steps, 4),
                        "tuned_vs_default": round(per_def[name] / per[name], 3)}
    dom = max(calls, key=lambda c: per[c[0]])
    dom_ms = per[dom[0]] / args.steps
    dom_gbs = dom[1] / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom[0], "achieved": round(dom_gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(dom_gbs / hbm, 3), "peak_kind": peak_kind,
                "traffic": committed_traffic(dom[0])}
    l2 = None
    if not args.force:
        rate, l2_ms = l2_random_rate(sk, torch, stream)
        l2 = {"reads_per_s": round(rate / 1e9, 2), "unit": "1e9 reads/s", "ms": round(l2_ms, 4),
              "what": "random 4-byte reads from a 4 MiB table (2^20 floats), one wave of 8 blocks per SM"}
        if "maparray_gather" in per:
            g_ms = per["maparray_gather"] / args.steps
            g_rate = N / (g_ms * 1e-3)
            l2["gather_frac"] = round(g_rate / rate, 3)
            if dom[0] == "maparray_gather":
                # the gather's table reads are random L2 sectors: its roofline is
                # the measured random-read rate, in the gather's own units (8
                # algorithmic bytes per read: the index read and the output write)
                roofline = {"bound": "l2", "kernel": dom[0], "achieved": round(dom_gbs, 1),
                            "peak": round(8 * rate / 1e9, 1), "unit": "GB/s", "frac": round(g_rate / rate, 3),
                            "peak_kind": "measured (skel_probe_l2_random), 8 algorithmic bytes per random read",
                            "hbm_peak": hbm, "hbm_frac": round(dom_gbs / hbm, 3), "traffic": committed_traffic(dom[0])}

    line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(),
            "frac_of_peak": round(value / world / hbm, 3),
            "tuned_vs_default_speedup": round(def_ms / total_ms, 3), "dispatch_table": tuned,
            "per_skeleton": per_sk, "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
            "input_gen_s": round(wl.gen_s, 1), "l2_random_probe": l2}
    try:
        import cpu_baseline as cb
        line["host"] = cb.host_cpu()
    except Exception as e:  # the host description is informative only
        line["host"] = {"error": str(e)}
    del wl, calls
    torch.cuda.empty_cache()
    if not args.only and not args.force and not args.no_next:
        line["next"] = {"coulomb_grid": coulomb_leg(sk, torch, stream, clocks)}
        line["configs"] = config_legs(sk, torch, stream)
        line["configs"]["call_overhead"] = overhead_leg(sk, torch, stream, per_sk)
    if not args.no_e2e:
        dt, h2d, d2h, cpus, per_step = e2e_run(sk, torch, min(args.steps, 5), stream)
        dt = max_over_ranks(dt * 1e3) / 1e3
        line["e2e"] = {"value": round(world * step_bytes / dt / 1e9, 1), "unit": "GB/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": round(dt * 1e3, 2),
                       "step_ms": [round(x * 1e3, 1) for x in per_step],
                       "host_cpus": "gpu-local" if cpus else "unchanged"}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_parallel"] = cpu_parallel_leg()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
