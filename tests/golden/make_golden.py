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


def main():
    for name, arr in cases():
        with open(os.path.join(HERE, name + ".txt"), "w") as f:
            f.write(f"# oracle output on tiny seeded inputs, written by make_golden.py\n")
            for v in np.asarray(arr, dtype=np.float64):
                f.write(repr(float(v)) + "\n")


if __name__ == "__main__":
    main()
