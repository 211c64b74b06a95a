"""Parity of the Coulombic potential grid (MapArray over grid positions)
against the float64 oracle: whole small grids with ragged shapes, and
sampled points of a large grid."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import SUM_REL, dev_empty, dev_tensor, forced, skel, to_np, wrap

pytestmark = pytest.mark.gpu


def atoms_for(m, rows, cols, h, seed=syn.SEED_X):
    """m atoms uniform over the grid's extent, 0.5..4.5 above the plane z0 = 0,
    charges uniform in [-1, 1)."""
    a = np.empty((m, 4), np.float32)
    a[:, 0] = syn.uniform_f32(seed, m, 0.0, 1.0) * np.float32(cols * h)
    a[:, 1] = syn.uniform_f32(seed + 1, m, 0.0, 1.0) * np.float32(rows * h)
    a[:, 2] = syn.uniform_f32(seed + 2, m, 0.5, 4.5)
    a[:, 3] = syn.uniform_f32(seed + 3, m)
    return a


def check(gpu, ref, ab, what):
    err = np.abs(gpu.astype(np.float64) - ref)
    tol = SUM_REL * ab
    assert np.all(err <= tol), f"{what}: worst err/(2^-20 sum|q/r|) = {float(np.max(err / tol)):.3f}"


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("rows,cols,m", [(1, 1, 1), (8, 256, 4), (13, 300, 7), (5, 1000, 1025), (33, 77, 2048),
                                         (3, 5, 0)])
def test_coulomb_grid_small(variant, rows, cols, m):
    import torch
    sk = skel()
    h, z0 = 0.5, 0.0
    a = atoms_for(m, rows, cols, h)
    out = dev_empty((rows, cols), torch.float32)
    with forced("maparray", variant):
        sk.skel_maparray_grid("coulomb", wrap(dev_tensor(a)), wrap(out), (h, z0))
    ref, ab = oracle.coulomb_grid_f32(a, rows, cols, h, z0)
    if m == 0:
        assert np.array_equal(to_np(out), np.zeros((rows, cols), np.float32))
        return
    check(to_np(out), ref, ab, f"v{variant} {rows}x{cols} m={m}")


@pytest.mark.parametrize("variant", [0, 1])
def test_coulomb_large_grid_sampled(variant):
    """2048 x 2048 points, 4096 atoms; 400 sampled points against the oracle."""
    import torch
    sk = skel()
    rows = cols = 2048
    m, h, z0 = 4096, 0.125, 0.0
    a = atoms_for(m, rows, cols, h, seed=syn.SEED_Y)
    out = dev_empty((rows, cols), torch.float32)
    with forced("maparray", variant):
        sk.skel_maparray_grid("coulomb", wrap(dev_tensor(a)), wrap(out), (h, z0))
    g = to_np(out)
    ii = syn.uniform_int(syn.SEED_IDX, 400, 0, rows - 1)
    jj = syn.uniform_int(syn.SEED_IDX + 1, 400, 0, cols - 1)
    ref, ab = oracle.coulomb_points_f32(a, ii, jj, h, z0)
    check(g[ii, jj], ref, ab, f"v{variant} sampled")


def test_coulomb_variants_agree_and_dispatch():
    import torch
    sk = skel()
    rows, cols, m = 64, 512, 3000
    a = atoms_for(m, rows, cols, 1.0)
    outs = []
    for v in (0, 1):
        o = dev_empty((rows, cols), torch.float32)
        with forced("maparray", v):
            sk.skel_maparray_grid("coulomb", wrap(dev_tensor(a)), wrap(o), (1.0, 0.0))
        outs.append(to_np(o))
    ref, ab = oracle.coulomb_grid_f32(a, rows, cols, 1.0, 0.0)
    for g in outs:
        check(g, ref, ab, "variant")
    o = dev_empty((rows, cols), torch.float32)
    sk.skel_maparray_grid("coulomb", wrap(dev_tensor(a)), wrap(o), (1.0, 0.0))   # dispatched
    check(to_np(o), ref, ab, "dispatched")


def test_coulomb_rejects_bad_arguments():
    import torch
    sk = skel()
    a = wrap(dev_tensor(atoms_for(10, 4, 4, 1.0)))
    out = wrap(dev_empty((4, 4), torch.float32))
    with pytest.raises(sk.SkelError):
        sk.skel_maparray_grid("coulomb", a, out, (0.0, 0.0))           # h must be > 0
    with pytest.raises(sk.SkelError):
        sk.skel_maparray_grid("coulomb", a, out, (1.0,))               # two params
    bad = wrap(dev_tensor(np.zeros((10, 3), np.float32)))
    with pytest.raises(sk.SkelError):
        sk.skel_maparray_grid("coulomb", bad, out, (1.0, 0.0))         # atoms must be (m, 4)
    with pytest.raises(sk.SkelError):
        sk.skel_maparray_grid("gather", a, out, (1.0, 0.0))            # only COULOMB
