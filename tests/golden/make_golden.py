"""Writes the regression fixtures in this folder.  Calls only the oracle and
the seeded input generator; run it from the repository root:

    python tests/golden/make_golden.py

The paper prints no worked example (it is a survey without numeric results),
so these fixtures are not the paper's values: they freeze the oracle's
outputs on tiny seeded inputs, so that any later change to the oracle's
arithmetic shows up as a failing test and has to be justified.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synthetic as syn  # noqa: E402


def cases():
    x = syn.uniform_f32(101, 37)
    y = syn.uniform_f32(102, 37)
    xi = syn.uniform_int(103, 37)
    g = syn.uniform_f32(104, 6 * 7).reshape(6, 7)
    w9 = oracle.stencil_weights("9pt")
    w5 = oracle.stencil_weights("5pt")
    w1 = syn.uniform_f32(105, 7, 0.0, 1.0)
    yield "map_axpy", oracle.map_f32("axpy", x, y, a=2.5)
    yield "map_tanh", oracle.map_f32("tanh", x)
    yield "reduce_add_f32", np.array([oracle.reduce_f32("add", x)[0]])
    yield "reduce_max_f32", np.array([oracle.reduce_f32("max", x)[0]])
    yield "mapreduce_dot", np.array([oracle.mapreduce_f32("mul", x, y)[0]])
    yield "scan_incl_i32", oracle.scan_i32(xi, True).astype(np.float64)
    yield "scan_excl_f32", oracle.scan_f32(x, False)[0]
    yield "scan_bwd_incl_f32", oracle.scan_bwd_f32(x, True)[0]
    yield "mapoverlap1d_r3_clamp", oracle.mapoverlap1d_f32(x, 3, w1, "clamp")
    yield "mapoverlap2d_9pt_clamp", oracle.mapoverlap2d_f32(g, 1, w9, "clamp").ravel()
    yield "mapoverlap2d_5pt_clamp", oracle.mapoverlap2d_f32(g, 1, w5, "clamp").ravel()
    yield "mapoverlap2d_9pt_clamp_bwd", oracle.mapoverlap2d_bwd_f32(g, 1, w9, "clamp").ravel()
    yield "composed_loss_grad", oracle.composed_loss_f32(g, 1, w9, "clamp")[1].ravel()
    yield "mapoverlap2d_chain_9pt_zero_x3", oracle.mapoverlap2d_chain_f32(g, 1, w9, "zero", 3).ravel()
    yield "chain_tanh_9pt_sumsq_periodic", np.array(oracle.chain_map_stencil_sumsq_f32("tanh", g, 1, w9, "periodic"))
    M = syn.uniform_f32(106, 5 * 37).reshape(5, 37)
    yield "maparray_rowdot", oracle.rowdot_f32(x, M)[0]
    idx = syn.uniform_int(107, 11, 0, 36)
    yield "maparray_gather", oracle.gather_f32(x, idx)
    atoms = syn.uniform_f32(108, 3 * 4, 0.0, 1.0).reshape(3, 4)
    yield "coulomb_points", oracle.coulomb_points_f32(atoms, np.array([0, 2, 5]), np.array([1, 0, 3]), 0.25, -1.0)[0]
    off = np.array([0, 0, 5, 6, 37], np.int64)
    sumsq, scan, _ = oracle.batched_f32(x, off, True)
    yield "batched_sumsq", sumsq
    yield "batched_scan_incl", scan


def main():
    for name, arr in cases():
        with open(os.path.join(HERE, name + ".txt"), "w") as f:
            f.write(f"# oracle output on tiny seeded inputs, written by make_golden.py\n")
            for v in np.asarray(arr, dtype=np.float64):
                f.write(repr(float(v)) + "\n")


if __name__ == "__main__":
    main()
