"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws numbers and nothing else: it holds none of the skeleton
arithmetic (no map functor, reduction, scan or stencil).  Every value comes
from the counter-based SplitMix64 generator (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the finaliser
constants are the published "mix13" variant), evaluated at counter i as

    z   = seed + (i + 1) * 0x9E3779B97F4A7C15        (mod 2^64)
    z   = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z   = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

so that element i of a stream does not depend on how the stream is chunked.

Derived draws:
  * ``uniform_f32(seed, n, lo, hi)``: u = (out >> 40) * 2^-24 in [0, 1) on a
    2^-24 grid, v = lo + (hi - lo) * u rounded to float32.  For the two ranges
    the workloads use, [0, 1) and [-1, 1), v is exactly representable, so the
    float32 the GPU receives and the float64 the oracle widens are the same number.
  * ``uniform_int(seed, n, lo, hi)``: lo + out mod (hi - lo + 1) as int32.
  * ``loguniform_lengths(seed, count, lo, hi)``: floor(lo * (hi/lo)^u) clamped
    to [lo, hi], u = (out >> 11) * 2^-53 -- the uneven instance lengths of the
    batched workload (4096 instances, lengths in [64, 2^20]).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Fixed seeds of the workloads (any integer works; these name the workload).
SEED_X = 1405291501
SEED_Y = 1405291502
SEED_INT = 1405291503
SEED_GRID = 1405291504
SEED_BATCH_LEN = 1405291505
SEED_BATCH_VAL = 1405291506
SEED_IDX = 1405291507
SEED_MAT = 1405291508
SEED_GRAD = 1405291509

_CHUNK = 1 << 22


def _mix_chunk(seed: int, start: int, count: int) -> np.ndarray:
    """SplitMix64 outputs for counters start .. start+count-1."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _chunked(n: int, fill) -> None:
    """Run fill(start, count) over [0, n) in chunks, on a few host threads
    (numpy releases the GIL inside these array operations)."""
    spans = [(s, min(_CHUNK, n - s)) for s in range(0, n, _CHUNK)]
    if len(spans) <= 1:
        for s, c in spans:
            fill(s, c)
        return
    workers = max(1, min(len(spans), (os.cpu_count() or 1), 16))
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(lambda sc: fill(*sc), spans))


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Raw uint64 stream: counters start .. start+n-1."""
    out = np.empty(n, dtype=np.uint64)

    def fill(s, c):
        out[s:s + c] = _mix_chunk(seed, start + s, c)

    _chunked(n, fill)
    return out


def uniform_f32(seed: int, n: int, lo: float = -1.0, hi: float = 1.0,
                out: np.ndarray | None = None) -> np.ndarray:
    """float32 values lo + (hi - lo) * k * 2^-24, k uniform in [0, 2^24)."""
    if out is None:
        out = np.empty(n, dtype=np.float32)
    scale = float(hi) - float(lo)

    def fill(s, c):
        k = (_mix_chunk(seed, s, c) >> np.uint64(40)).astype(np.float64)
        out[s:s + c] = (lo + scale * (k * 2.0 ** -24)).astype(np.float32)

    _chunked(n, fill)
    return out


def uniform_int(seed: int, n: int, lo: int = 0, hi: int = 100,
                dtype=np.int32) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by remainder."""
    out = np.empty(n, dtype=dtype)
    span = np.uint64(hi - lo + 1)

    def fill(s, c):
        out[s:s + c] = ((_mix_chunk(seed, s, c) % span).astype(np.int64) + lo).astype(dtype)

    _chunked(n, fill)
    return out


def loguniform_lengths(seed: int, count: int, lo: int = 64, hi: int = 1 << 20) -> np.ndarray:
    """int64 lengths floor(lo * (hi/lo)^u), u uniform in [0, 1), clamped to [lo, hi]."""
    u = (_mix_chunk(seed, 0, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    lens = np.floor(lo * np.exp2(u * np.log2(hi / lo))).astype(np.int64)
    return np.clip(lens, lo, hi)


def csr_offsets(lengths: np.ndarray) -> np.ndarray:
    """int64 offsets[0..B] of instances laid end to end (offsets[0] = 0)."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lengths, dtype=np.int64)
    return off
