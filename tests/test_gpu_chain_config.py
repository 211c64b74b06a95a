"""The MapOverlap 2D chain workload at its full sizes: 5-point and 9-point
clamp stencils, ten chained calls on square grids of side 512, 2048, 8192 and
16384 (seeded U[0, 1)), dispatched through the committed GB300 execution-plan
table as the benchmark runs them, with the input valid only in host memory
before the chain and the result read on the host after it (Sec. IV: the
smart container keeps the intermediate grids on the device, so the chain
makes one host-to-device and one device-to-host copy).

Two forms are checked: the composed chain (skel_mapoverlap_chain, whose
variant and steps per pass the table picks) and ten single MapOverlap calls
ping-ponging between two containers.  Both are compared element by element
with the oracle's float64 chain: on the whole grid up to 2048^2, and at 8192^2
and 16384^2 on nine windows (the four corners, the four edge midpoints and the
centre), each computed by the oracle from an input window widened by one cell
per step on every side that does not lie on the grid's edge, so that every
compared output's ten-step neighbourhood is inside it.  Tolerance: steps x
1e-6 absolute (each averaging step adds a few float32 roundings of values
<= 1 and does not amplify earlier ones)."""
import os

import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import assert_elem_close, skel

STEPS = 10
WIN = 192
TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1405_2915_gb300",
                     "dispatch_gb300.tbl")


@pytest.fixture(scope="module")
def sk():
    s = skel()
    if os.path.exists(TABLE):
        s.skel_load_dispatch_table(TABLE)
    yield s
    s.skel_load_dispatch_table(None)


def windows(side: int, whole_up_to: int = 2048):
    """(r0, c0) of the compared WIN x WIN output windows (None: the whole grid)."""
    if side <= whole_up_to:
        return None
    lo, mid, hi = 0, side // 2 - WIN // 2, side - WIN
    return [(r, c) for r in (lo, mid, hi) for c in (lo, mid, hi)]


def oracle_window(x, w, r0, c0):
    """The oracle's chain on the output window [r0, r0+WIN) x [c0, c0+WIN):
    computed on the input widened by STEPS cells on every side inside the
    grid (the window's clamp then acts only where the grid's own edge is)."""
    side = x.shape[0]
    a0, a1 = max(0, r0 - STEPS), min(side, r0 + WIN + STEPS)
    b0, b1 = max(0, c0 - STEPS), min(side, c0 + WIN + STEPS)
    ref = oracle.mapoverlap2d_chain_f32(x[a0:a1, b0:b1], 1, w, "clamp", STEPS)
    return ref[r0 - a0:r0 - a0 + WIN, c0 - b0:c0 - b0 + WIN]


def check(got, x, w, what):
    wins = windows(x.shape[0])
    if wins is None:
        ref = oracle.mapoverlap2d_chain_f32(x, 1, w, "clamp", STEPS)
        assert_elem_close(got, ref, what, atol=STEPS * 1e-6)
        return
    for r0, c0 in wins:
        assert_elem_close(got[r0:r0 + WIN, c0:c0 + WIN], oracle_window(x, w, r0, c0),
                          f"{what} window ({r0}, {c0})", atol=STEPS * 1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("side", [512, 2048, 8192, 16384])
@pytest.mark.parametrize("kind", ["stencil5", "stencil9"])
@pytest.mark.parametrize("form", ["composed", "single_calls"])
def test_chain_config_full_size(sk, side, kind, form):
    x = syn.uniform_f32(syn.SEED_GRID, side * side, 0.0, 1.0).reshape(side, side)
    w = oracle.stencil_weights("5pt" if kind == "stencil5" else "9pt")
    cin = sk.Container.from_host(x)                         # valid only on the host
    a, b = sk.Container.empty((side, side)), sk.Container.empty((side, side))
    if form == "composed":
        sk.skel_mapoverlap_chain(kind, None, "clamp", STEPS, cin, b, a)
        res = a
    else:
        src = cin
        for k in range(STEPS):
            dst = a if k % 2 == 0 else b
            sk.skel_mapoverlap(kind, 1, None, "clamp", src, dst)
            src = dst
        res = src
    got = res.to_numpy()
    s_in, s_out = cin.stats(), res.stats()
    assert (s_in["h2d"], s_in["d2h"]) == (1, 0), s_in      # one copy in ...
    assert (s_out["h2d"], s_out["d2h"]) == (0, 1), s_out   # ... and one copy out
    check(got, x, w, f"{form} {kind} {side}^2 x{STEPS}")
    for c in (cin, a, b):
        c.close()


def test_windowed_oracle_equals_the_whole_grid_oracle():
    """On a grid the oracle finishes whole, every window computed from its
    widened input equals the whole-grid chain bit for bit (the compared
    outputs' ten-step neighbourhoods lie inside the widened input), and a
    chain one step short differs by far more than the tolerance, so the
    windowed check cannot pass by construction."""
    side = 640
    x = syn.uniform_f32(syn.SEED_GRID, side * side, 0.0, 1.0).reshape(side, side)
    for kind in ("5pt", "9pt"):
        w = oracle.stencil_weights(kind)
        full = oracle.mapoverlap2d_chain_f32(x, 1, w, "clamp", STEPS)
        for r0, c0 in windows(side, whole_up_to=0):
            assert np.array_equal(oracle_window(x, w, r0, c0), full[r0:r0 + WIN, c0:c0 + WIN]), (kind, r0, c0)
        short = oracle.mapoverlap2d_chain_f32(x, 1, w, "clamp", STEPS - 1)
        assert np.abs(short - full).max() > STEPS * 1e-6
