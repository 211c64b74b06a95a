"""Pins of the CPU oracle to things other than itself (closed forms, library
routines, brute force on tiny inputs, invariants, finite differences).

Each pin is chosen so that a plausible slip in the oracle -- a dropped term,
a wrong sign or index, a transposed operand, a wrong boundary map -- fails at
least one of them.  No GPU is needed.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic as syn

scipy_ndimage = pytest.importorskip("scipy.ndimage")

SCIPY_MODE = {"clamp": "nearest", "zero": "constant", "periodic": "grid-wrap"}


def dyadic(n, seed, bits=8):
    """float32 values k / 2^bits, k in [-2^bits, 2^bits): every sum of a few
    thousand of them is exact in float64."""
    k = syn.uniform_int(seed, n, -(1 << bits), (1 << bits) - 1).astype(np.float64)
    return (k / (1 << bits)).astype(np.float32)


# ------------------------------------------------------------------ Map ---
def test_map_axpy_exact_on_dyadic():
    x, y = dyadic(257, 1), dyadic(257, 2)
    out = oracle.map_f32("axpy", x, y, a=2.5)
    expect = [Fraction(5, 2) * Fraction(float(a)) + Fraction(float(b)) for a, b in zip(x, y)]
    assert all(Fraction(float(o)) == e for o, e in zip(out, expect))


def test_map_tanh_closed_form_and_symmetry():
    x = syn.uniform_f32(3, 200, -4.0, 4.0)
    out = oracle.map_f32("tanh", x)
    for xi, oi in zip(x.astype(np.float64), out):
        e = math.expm1(2 * xi) / (math.exp(2 * xi) + 1.0)   # tanh = (e^2x - 1)/(e^2x + 1)
        assert abs(oi - e) <= 4e-16 * max(1.0, abs(e))
    assert np.array_equal(oracle.map_f32("tanh", -x), -out)
    assert oracle.map_f32("tanh", np.zeros(3, np.float32)).tolist() == [0.0, 0.0, 0.0]


def test_map_binary_functors_against_numpy():
    x, y = syn.uniform_f32(4, 100), syn.uniform_f32(5, 100)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    assert np.array_equal(oracle.map_f32("mul", x, y), np.multiply(xd, yd))
    assert np.array_equal(oracle.map_f32("add", x, y), np.add(xd, yd))
    assert np.array_equal(oracle.map_f32("sub", x, y), np.subtract(xd, yd))
    assert np.array_equal(oracle.map_f32("max", x, y), np.maximum(xd, yd))
    assert np.array_equal(oracle.map_f32("sq", x), np.square(xd))
    assert np.array_equal(oracle.map_f32("scale", x, a=-3.0), -3.0 * xd)


@pytest.mark.parametrize("fn,nin", [("axpy", 2), ("mul", 2), ("add", 2), ("sub", 2),
                                    ("tanh", 1), ("sq", 1), ("scale", 1)])
def test_map_bwd_is_derivative(fn, nin):
    """Central differences in float64 around float32 points."""
    x = syn.uniform_f32(6, 50)
    y = syn.uniform_f32(7, 50) if nin == 2 else None
    g = syn.uniform_f32(8, 50)
    gx, gy = oracle.map_bwd_f32(fn, g, x, y, a=2.5)
    h = 1e-6
    xd = x.astype(np.float64)
    yd = y.astype(np.float64) if y is not None else None

    def f(xv, yv):
        return {"axpy": lambda: 2.5 * xv + yv, "mul": lambda: xv * yv, "add": lambda: xv + yv,
                "sub": lambda: xv - yv, "tanh": lambda: np.tanh(xv), "sq": lambda: xv * xv,
                "scale": lambda: 2.5 * xv}[fn]()

    fd_x = (f(xd + h, yd) - f(xd - h, yd)) / (2 * h) * g
    assert np.allclose(gx, fd_x, rtol=1e-7, atol=1e-8)
    if nin == 2:
        fd_y = (f(xd, yd + h) - f(xd, yd - h)) / (2 * h) * g
        assert np.allclose(gy, fd_y, rtol=1e-7, atol=1e-8)


# --------------------------------------------------------------- Reduce ---
@pytest.mark.parametrize("n", [0, 1, 2, 17, 1000, 4099])
def test_reduce_int_closed_forms(n):
    x = np.arange(n, dtype=np.int32)
    assert oracle.reduce_i32("add", x) == n * (n - 1) // 2
    perm = syn.splitmix64(11, n).argsort().astype(np.int32)      # a permutation of 0..n-1
    assert oracle.reduce_i32("max", perm) == (n - 1 if n else -(1 << 31))
    assert oracle.reduce_i32("add", perm) == n * (n - 1) // 2


def test_reduce_f32_exact_on_dyadic_and_identities():
    x = dyadic(5001, 12)
    v, a = oracle.reduce_f32("add", x)
    assert Fraction(v) == sum(Fraction(float(t)) for t in x)
    assert Fraction(a) == sum(abs(Fraction(float(t))) for t in x)
    assert oracle.reduce_f32("max", x)[0] == float(max(x.tolist()))
    assert oracle.reduce_f32("add", np.zeros(0, np.float32)) == (0.0, 0.0)
    assert oracle.reduce_f32("max", np.zeros(0, np.float32))[0] == -math.inf


def test_reduce_equals_last_of_inclusive_scan():
    x = syn.uniform_f32(13, 3000)
    assert oracle.reduce_f32("add", x)[0] == oracle.scan_f32(x, True)[0][-1]
    xi = syn.uniform_int(14, 3000)
    assert oracle.reduce_i32("add", xi) == oracle.scan_i32(xi, True)[-1]


def test_reduce_sum_wraps_to_int32_like_numpy():
    """(oracle sum) mod 2^32 == numpy's wrapping int32 accumulation."""
    x = np.full(5, 2**31 - 1, dtype=np.int32)
    s = oracle.reduce_i32("add", x)
    assert s == 5 * (2**31 - 1)
    assert np.int64(s).astype(np.int32) == np.add.reduce(x, dtype=np.int32)


# ------------------------------------------------------------ MapReduce ---
def test_mapreduce_dot_and_sumsq():
    n = 3000
    ones = np.ones(n, np.float32)
    assert oracle.mapreduce_f32("mul", ones, ones) == (float(n), float(n))
    x, y = dyadic(n, 15), dyadic(n, 16)
    v, a = oracle.mapreduce_f32("mul", x, y)
    assert Fraction(v) == sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(x, y))
    assert Fraction(a) == sum(abs(Fraction(float(p)) * Fraction(float(q))) for p, q in zip(x, y))
    v2, _ = oracle.mapreduce_f32("sq", x)
    assert Fraction(v2) == sum(Fraction(float(p)) ** 2 for p in x)


def test_mapreduce_is_reduce_of_map():
    x, y = syn.uniform_f32(17, 4000), syn.uniform_f32(18, 4000)
    # sequential float64 summation error is at most (n-1) * 2^-53 * sum |t|
    for fn, yy in (("mul", y), ("sq", None)):
        mapped = oracle.map_f32(fn, x, yy)
        bound = len(x) * 2.0 ** -53 * math.fsum(np.abs(mapped))
        assert abs(oracle.mapreduce_f32(fn, x, yy)[0] - math.fsum(mapped)) <= bound


# ----------------------------------------------------------------- Scan ---
@pytest.mark.parametrize("n", [0, 1, 5, 64])
def test_scan_brute_force(n):
    x = syn.uniform_int(20, n)
    inc = oracle.scan_i32(x, True)
    exc = oracle.scan_i32(x, False)
    xl = [int(t) for t in x]
    assert inc.tolist() == [sum(xl[:i + 1]) for i in range(n)]
    assert exc.tolist() == [sum(xl[:i]) for i in range(n)]
    xf = dyadic(n, 21)
    fl = [Fraction(float(t)) for t in xf]
    inc_f, ab = oracle.scan_f32(xf, True)
    exc_f, abe = oracle.scan_f32(xf, False)
    assert [Fraction(v) for v in inc_f] == [sum(fl[:i + 1]) for i in range(n)]
    assert [Fraction(v) for v in exc_f] == [sum(fl[:i]) for i in range(n)]
    assert [Fraction(v) for v in ab] == [sum(abs(t) for t in fl[:i + 1]) for i in range(n)]
    assert [Fraction(v) for v in abe] == [sum(abs(t) for t in fl[:i]) for i in range(n)]


def test_scan_ones_and_incl_minus_excl():
    n = 5000
    assert oracle.scan_i32(np.ones(n, np.int32), True).tolist() == list(range(1, n + 1))
    assert oracle.scan_i32(np.ones(n, np.int32), False).tolist() == list(range(n))
    x = syn.uniform_int(22, n)
    assert np.array_equal(oracle.scan_i32(x, True) - oracle.scan_i32(x, False), x.astype(np.int64))


def test_scan_int32_wraparound_matches_numpy_cumsum():
    """The GPU int32 scan wraps modulo 2^32; (oracle mod 2^32) must equal
    numpy's wrapping int32 cumulative sum."""
    x = syn.uniform_int(23, 1 << 16, 0, 2**31 - 1)
    ref = np.cumsum(x, dtype=np.int32)
    assert np.array_equal(oracle.scan_i32(x, True).astype(np.int32), ref)


def test_scan_bwd_adjoint_identity_and_dense():
    n = 300
    x, y = dyadic(n, 24), dyadic(n, 25)
    for inclusive in (True, False):
        sx, _ = oracle.scan_f32(x, inclusive)
        ry, _ = oracle.scan_bwd_f32(y, inclusive)
        lhs = sum(Fraction(float(a)) * Fraction(b) for a, b in zip(sx, y.astype(np.float64)))
        rhs = sum(Fraction(float(a)) * Fraction(b) for a, b in zip(x.astype(np.float64), ry))
        assert lhs == rhs
        # dense: column sums of the (strictly) lower triangular ones matrix
        L = np.tril(np.ones((n, n)), 0 if inclusive else -1)
        assert np.array_equal(ry, L.T @ y.astype(np.float64))


# ----------------------------------------------------------- MapOverlap ---
def binom_weights(r):
    w = np.array([math.comb(2 * r, k) for k in range(2 * r + 1)], dtype=np.float64)
    return (w / w.sum()).astype(np.float32)


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("r,n", [(1, 1), (1, 7), (3, 5), (4, 100), (16, 40), (16, 1000)])
def test_mapoverlap1d_against_scipy(boundary, r, n):
    x = syn.uniform_f32(30 + r, n)
    w = syn.uniform_f32(31 + r, 2 * r + 1, 0.0, 1.0)
    out = oracle.mapoverlap1d_f32(x, r, w, boundary)
    ref = scipy_ndimage.correlate1d(x.astype(np.float64), w.astype(np.float64),
                                    mode=SCIPY_MODE[boundary], cval=0.0)
    assert np.allclose(out, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("shape,r", [((1, 1), 1), ((3, 4), 1), ((8, 8), 1), ((33, 17), 1),
                                     ((10, 12), 2)])
def test_mapoverlap2d_against_scipy(boundary, shape, r):
    x = syn.uniform_f32(40, shape[0] * shape[1]).reshape(shape)
    w = syn.uniform_f32(41, (2 * r + 1) ** 2, -1.0, 1.0).reshape(2 * r + 1, 2 * r + 1)
    out = oracle.mapoverlap2d_f32(x, r, w, boundary)
    ref = scipy_ndimage.correlate(x.astype(np.float64), w.astype(np.float64),
                                  mode=SCIPY_MODE[boundary], cval=0.0)
    assert np.allclose(out, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", ["5pt", "9pt"])
def test_stencil_weights_and_constant_grid(kind):
    w = oracle.stencil_weights(kind)
    assert float(w.astype(np.float64).sum()) == 1.0
    assert np.array_equal(w, w[::-1, ::-1]) and np.array_equal(w, w.T)
    c = np.full((9, 13), 0.375, np.float32)
    for b in ("clamp", "periodic"):
        assert np.all(oracle.mapoverlap2d_f32(c, 1, w, b) == 0.375)
    z = oracle.mapoverlap2d_f32(c, 1, w, "zero")
    assert np.all(z[1:-1, 1:-1] == 0.375) and np.all(z[0, 1:-1] < 0.375)


def test_stencil_preserves_linear_field_in_interior():
    i, j = np.meshgrid(np.arange(20), np.arange(24), indexing="ij")
    x = (0.25 * i - 0.5 * j).astype(np.float32)
    for kind in ("5pt", "9pt"):
        out = oracle.mapoverlap2d_f32(x, 1, oracle.stencil_weights(kind), "clamp")
        assert np.array_equal(out[1:-1, 1:-1], x[1:-1, 1:-1].astype(np.float64))


def dense_stencil_matrix_2d(rows, cols, r, w, boundary):
    """S with (S x)_flat == stencil(x)_flat, built column by column by
    applying scipy's correlate to unit grids."""
    S = np.zeros((rows * cols, rows * cols))
    for p in range(rows * cols):
        e = np.zeros(rows * cols)
        e[p] = 1.0
        S[:, p] = scipy_ndimage.correlate(e.reshape(rows, cols), w.astype(np.float64),
                                          mode=SCIPY_MODE[boundary], cval=0.0).ravel()
    return S


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("shape,r", [((1, 1), 1), ((2, 3), 1), ((5, 4), 1), ((8, 8), 1), ((7, 6), 2)])
def test_mapoverlap2d_bwd_is_dense_transpose(boundary, shape, r):
    w = syn.uniform_f32(50, (2 * r + 1) ** 2, -1.0, 1.0).reshape(2 * r + 1, 2 * r + 1)
    g = syn.uniform_f32(51, shape[0] * shape[1]).reshape(shape)
    S = dense_stencil_matrix_2d(shape[0], shape[1], r, w, boundary)
    ref = (S.T @ g.astype(np.float64).ravel()).reshape(shape)
    out = oracle.mapoverlap2d_bwd_f32(g, r, w, boundary)
    assert np.allclose(out, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("shape,steps", [((1, 1), 3), ((6, 5), 1), ((6, 5), 4), ((9, 12), 10)])
def test_mapoverlap2d_chain_is_matrix_power(boundary, shape, steps):
    """A chain of k calls is S^k applied to x (numpy matrix power of the
    dense stencil matrix built with scipy's correlate)."""
    w = syn.uniform_f32(52, 9, -1.0, 1.0).reshape(3, 3)
    x = syn.uniform_f32(53, shape[0] * shape[1]).reshape(shape)
    S = dense_stencil_matrix_2d(shape[0], shape[1], 1, w, boundary)
    ref = (np.linalg.matrix_power(S, steps) @ x.astype(np.float64).ravel()).reshape(shape)
    out = oracle.mapoverlap2d_chain_f32(x, 1, w, boundary, steps)
    assert np.allclose(out, ref, rtol=0, atol=1e-12 * max(1.0, float(np.abs(ref).max())))


def test_mapoverlap2d_chain_constant_and_single_step():
    c = np.full((7, 9), 0.375, np.float32)
    for kind in ("5pt", "9pt"):
        assert np.array_equal(oracle.mapoverlap2d_chain_f32(c, 1, oracle.stencil_weights(kind), "clamp", 10),
                              c.astype(np.float64))
    x = syn.uniform_f32(54, 63).reshape(7, 9)
    w = oracle.stencil_weights("9pt")
    assert np.array_equal(oracle.mapoverlap2d_chain_f32(x, 1, w, "zero", 1), oracle.mapoverlap2d_f32(x, 1, w, "zero"))
    assert np.array_equal(oracle.mapoverlap2d_chain_f32(x, 1, w, "zero", 0), x.astype(np.float64))


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("r,n", [(1, 1), (1, 9), (3, 5), (16, 40)])
def test_mapoverlap1d_bwd_is_dense_transpose(boundary, r, n):
    w = syn.uniform_f32(52, 2 * r + 1, -1.0, 1.0)
    g = syn.uniform_f32(53, n)
    S = np.zeros((n, n))
    for p in range(n):
        e = np.zeros(n)
        e[p] = 1.0
        S[:, p] = scipy_ndimage.correlate1d(e, w.astype(np.float64), mode=SCIPY_MODE[boundary])
    assert np.allclose(oracle.mapoverlap1d_bwd_f32(g, r, w, boundary),
                       S.T @ g.astype(np.float64), rtol=0, atol=1e-13)


def test_mapoverlap2d_adjoint_identity_large():
    rows, cols = 200, 173
    w = oracle.stencil_weights("9pt")
    x = syn.uniform_f32(54, rows * cols).reshape(rows, cols)
    y = syn.uniform_f32(55, rows * cols).reshape(rows, cols)
    for b in ("clamp", "zero", "periodic"):
        lhs = float(np.vdot(oracle.mapoverlap2d_f32(x, 1, w, b), y.astype(np.float64)))
        rhs = float(np.vdot(x.astype(np.float64), oracle.mapoverlap2d_bwd_f32(y, 1, w, b)))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-9


# ------------------------------------------------------------- MapArray ---
def test_gather_copy_and_clamp():
    A = syn.uniform_f32(60, 100)
    assert np.array_equal(oracle.gather_f32(A, np.arange(100)), A.astype(np.float64))
    idx = np.array([-5, 0, 99, 100, 2**31 - 1, 50], np.int32)
    assert oracle.gather_f32(A, idx).tolist() == [float(A[0]), float(A[0]), float(A[99]),
                                                  float(A[99]), float(A[99]), float(A[50])]


def test_rowdot_identity_and_matmul():
    A = syn.uniform_f32(61, 64)
    out, _ = oracle.rowdot_f32(A, np.eye(64, dtype=np.float32))
    assert np.array_equal(out, A.astype(np.float64))
    M = syn.uniform_f32(62, 37 * 64).reshape(37, 64)
    out, ab = oracle.rowdot_f32(A, M)
    assert np.allclose(out, M.astype(np.float64) @ A.astype(np.float64), rtol=0, atol=1e-12)
    assert np.allclose(ab, np.abs(M.astype(np.float64)) @ np.abs(A.astype(np.float64)),
                       rtol=0, atol=1e-12)


# ------------------------------------------------ Coulombic potential ---
def test_coulomb_pythagorean_distances_and_orientation():
    """One charge q = 2 at (3, 0, 4) over the plane z0 = 0, spacing 1:
    distance 5 at the origin, 4 at (x=3, y=0) -- column j = 3 of row i = 0 --
    and sqrt(34) at (x=0, y=3), which tells the row and column axes apart."""
    atoms = np.array([[3.0, 0.0, 4.0, 2.0]], np.float32)
    v, ab = oracle.coulomb_grid_f32(atoms, 4, 4, 1.0, 0.0)
    assert v[0, 0] == 2.0 / 5.0
    assert v[0, 3] == 0.5
    assert v[3, 0] == 2.0 / math.sqrt(34.0)
    assert np.array_equal(ab, v)                       # one positive charge


def test_coulomb_square_of_charges_and_spacing():
    """Four charges at the corners (3 +- 3, 4 +- 4, 12) of a rectangle; the
    point below its centre, (3, 4, 0) = grid point (i=8, j=6) at spacing
    0.5, is 13 from each corner: V = sum q / 13."""
    q = [1.0, -2.0, 0.5, 4.0]
    atoms = np.array([[0, 0, 12, q[0]], [6, 0, 12, q[1]], [0, 8, 12, q[2]], [6, 8, 12, q[3]]], np.float32)
    v, ab = oracle.coulomb_points_f32(atoms, [8], [6], 0.5, 0.0)
    assert abs(v[0] - sum(q) / 13.0) < 1e-15
    assert abs(ab[0] - sum(abs(x) for x in q) / 13.0) < 1e-15


def test_coulomb_superposition_and_charge_scaling():
    a = syn.uniform_f32(81, 40 * 4, 0.0, 16.0).reshape(40, 4)
    a[:, 2] += 1.0                                      # atoms above the plane z0 = 0
    a[:, 3] = syn.uniform_f32(82, 40)                   # charges in [-1, 1)
    v_all, _ = oracle.coulomb_grid_f32(a, 9, 7, 2.0, 0.0)
    v1, _ = oracle.coulomb_grid_f32(a[:17], 9, 7, 2.0, 0.0)
    v2, _ = oracle.coulomb_grid_f32(a[17:], 9, 7, 2.0, 0.0)
    assert np.allclose(v_all, v1 + v2, rtol=0, atol=1e-12)
    b = a.copy()
    b[:, 3] *= 4.0                                      # exact in float32
    vb, _ = oracle.coulomb_grid_f32(b, 9, 7, 2.0, 0.0)
    assert np.allclose(vb, 4.0 * v_all, rtol=1e-15, atol=0)


def test_coulomb_far_field_monopole_bound():
    """Far from a cluster of extent a around c, |V - Q/R| <= sum|q| a / (R (R - a))
    (triangle inequality on each 1/r)."""
    a = syn.uniform_f32(83, 25 * 4, -1.0, 1.0).reshape(25, 4)
    c = np.array([100.0, 200.0, 3.0])
    a[:, :3] += c.astype(np.float32)
    ext = float(np.max(np.linalg.norm(a[:, :3].astype(np.float64) - c, axis=1)))
    Q, Qa = float(a[:, 3].astype(np.float64).sum()), float(np.abs(a[:, 3].astype(np.float64)).sum())
    for i, j in [(0, 0), (4000, 0), (0, 5000), (3000, 3000)]:
        v, _ = oracle.coulomb_points_f32(a, [i], [j], 1.0, 0.0)
        R = float(np.linalg.norm(np.array([j, i, 0.0]) - c))
        assert abs(v[0] - Q / R) <= Qa * ext / (R * (R - ext)) + 1e-15


# -------------------------------------------------------------- Batched ---
def test_batched_equals_per_instance_calls():
    lens = np.array([0, 1, 64, 5, 0, 300, 4097], np.int64)
    off = syn.csr_offsets(lens)
    v = syn.uniform_f32(70, int(off[-1]))
    for inclusive in (True, False):
        sumsq, sc, ab = oracle.batched_f32(v, off, inclusive)
        for b in range(len(lens)):
            seg = v[off[b]:off[b + 1]]
            assert sumsq[b] == oracle.mapreduce_f32("sq", seg)[0]
            ref, refab = oracle.scan_f32(seg, inclusive)
            assert np.array_equal(sc[off[b]:off[b + 1]], ref)
            assert np.array_equal(ab[off[b]:off[b + 1]], refab)
    assert sumsq[0] == 0.0 and sumsq[4] == 0.0


# -------------------------------------------------------- Composed loss ---
def composed_loss_numpy(x64, w, boundary):
    """Independent restatement through numpy/scipy library routines."""
    t = np.tanh(x64)
    u = scipy_ndimage.correlate(t, w.astype(np.float64), mode=SCIPY_MODE[boundary])
    s = np.cumsum(t, axis=1)
    return float(np.sum(u * u) + np.sum(s * s) / x64.size)


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
def test_composed_loss_value_and_gradient_fd(boundary):
    rows, cols = 16, 16
    w = oracle.stencil_weights("9pt")
    x = syn.uniform_f32(80, rows * cols).reshape(rows, cols)
    L, g = oracle.composed_loss_f32(x, 1, w, boundary)
    assert abs(L - composed_loss_numpy(x.astype(np.float64), w, boundary)) <= 1e-12 * abs(L)
    h = 1e-4
    x64 = x.astype(np.float64)
    for (i, j) in [(0, 0), (0, 15), (15, 0), (15, 15), (7, 8), (1, 14), (8, 0)]:
        xp, xm = x64.copy(), x64.copy()
        xp[i, j] += h
        xm[i, j] -= h
        fd = (oracle.composed_loss_f64(xp, 1, w, boundary) -
              oracle.composed_loss_f64(xm, 1, w, boundary)) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-7 * max(1.0, abs(g[i, j])), (i, j, fd, g[i, j])


@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
def test_composed_loss_local_delta_equals_full_difference(boundary):
    rows, cols = 12, 10
    w = oracle.stencil_weights("9pt")
    x = syn.uniform_f32(81, rows * cols).reshape(rows, cols)
    x64 = x.astype(np.float64)
    base = oracle.composed_loss_f64(x64, 1, w, boundary)
    for (i, j) in [(0, 0), (11, 9), (5, 0), (0, 4), (6, 5)]:
        h = 1e-3
        xp = x64.copy()
        xp[i, j] += h
        full = oracle.composed_loss_f64(xp, 1, w, boundary) - base
        local = oracle.composed_loss_delta_f32(x, 1, w, i, j, h, boundary)
        assert abs(full - local) <= 1e-12 * max(1.0, abs(base))


# ------------------------------------- Map -> MapOverlap -> MapReduce chain ---
UNARY = {"copy": lambda t, a: t, "sq": lambda t, a: t * t, "scale": lambda t, a: a * t, "tanh": lambda t, a: np.tanh(t)}


@pytest.mark.parametrize("fn,a", [("copy", 0.0), ("sq", 0.0), ("scale", 2.5), ("tanh", 0.0)])
@pytest.mark.parametrize("boundary", ["clamp", "periodic"])
def test_chain_constant_grid_closed_form(fn, a, boundary):
    """A constant grid c: every stencil output is f(c) (weights sum to 1,
    CLAMP and PERIODIC read only c), so the chain is rows * cols * f(c)^2."""
    c = 0.625
    x = np.full((9, 13), c, np.float32)
    for kind in ("5pt", "9pt"):
        v, bound = oracle.chain_map_stencil_sumsq_f32(fn, x, 1, oracle.stencil_weights(kind), boundary, a)
        fc = UNARY[fn](c, a) if fn != "tanh" else math.tanh(c)
        assert v == pytest.approx(9 * 13 * fc * fc, rel=1e-14)
        assert bound == pytest.approx(v, rel=1e-14)   # nonnegative weights and values: no cancellation


@pytest.mark.parametrize("boundary,scale", [("clamp", 1.0), ("periodic", 1.0), ("zero", 0.25)])
def test_chain_one_cell_grid(boundary, scale):
    """1 x 1 grid, 9-point weights: CLAMP and PERIODIC read the cell at every
    tap (sum of weights 1), ZERO only at the centre (weight 1/4)."""
    x = np.array([[0.75]], np.float32)
    v, _ = oracle.chain_map_stencil_sumsq_f32("scale", x, 1, oracle.stencil_weights("9pt"), boundary, 2.0)
    assert v == (scale * 1.5) ** 2


@pytest.mark.parametrize("fn,a", [("copy", 0.0), ("sq", 0.0), ("scale", -1.5), ("tanh", 0.0)])
@pytest.mark.parametrize("boundary", ["clamp", "zero", "periodic"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 4), (6, 6)])
def test_chain_is_dense_matrix_form(fn, a, boundary, shape):
    """r = |S f(x)|^2 with S the dense stencil matrix (built by scipy's
    correlate) and f applied by numpy."""
    w = syn.uniform_f32(60, 9, -1.0, 1.0).reshape(3, 3)
    x = syn.uniform_f32(61, shape[0] * shape[1]).reshape(shape)
    S = dense_stencil_matrix_2d(shape[0], shape[1], 1, w, boundary)
    u = S @ UNARY[fn](x.astype(np.float64).ravel(), a)
    v, bound = oracle.chain_map_stencil_sumsq_f32(fn, x, 1, w, boundary, a)
    assert v == pytest.approx(float(u @ u), rel=1e-12, abs=1e-300)
    # sum over the taps of |w| |t| per output: the stencil matrix of |w|
    # (taps that read the same cell add up, each with its own |w|)
    Sa = dense_stencil_matrix_2d(shape[0], shape[1], 1, np.abs(w), boundary)
    m = Sa @ np.abs(UNARY[fn](x.astype(np.float64).ravel(), a))
    assert bound == pytest.approx(float(m @ m), rel=1e-12, abs=1e-300)
    assert bound >= v - 1e-12 * abs(v)


def test_chain_copy_is_mapoverlap_then_sumsq():
    x = syn.uniform_f32(62, 33 * 47).reshape(33, 47)
    for kind, boundary in (("9pt", "clamp"), ("5pt", "zero"), ("9pt", "periodic")):
        w = oracle.stencil_weights(kind)
        u = oracle.mapoverlap2d_f32(x, 1, w, boundary)
        v, _ = oracle.chain_map_stencil_sumsq_f32("copy", x, 1, w, boundary)
        assert v == pytest.approx(float(np.sum(u * u)), rel=1e-13)


def test_chain_periodic_is_shift_invariant():
    x = syn.uniform_f32(63, 17 * 24).reshape(17, 24)
    w = syn.uniform_f32(64, 9, -1.0, 1.0).reshape(3, 3)
    v0, _ = oracle.chain_map_stencil_sumsq_f32("tanh", x, 1, w, "periodic")
    v1, _ = oracle.chain_map_stencil_sumsq_f32("tanh", np.roll(x, (5, -7), axis=(0, 1)), 1, w, "periodic")
    assert v1 == pytest.approx(v0, rel=1e-13)


# -------------------------------------------------------------- Generator ---
def test_generator_published_splitmix64_values():
    """First outputs of SplitMix64 from seed 0 (Vigna's reference
    implementation, state advanced by the golden gamma before mixing)."""
    z = syn.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_generator_ranges_and_exact_float32():
    x = syn.uniform_f32(90, 1 << 16)
    assert x.min() >= -1.0 and x.max() < 1.0
    k = (x.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.array_equal(k, np.round(k))            # on the 2^-23 grid: exact in float32
    u = syn.uniform_f32(91, 1 << 16, 0.0, 1.0)
    assert u.min() >= 0.0 and u.max() < 1.0
    lens = syn.loguniform_lengths(92, 4096)
    assert lens.min() >= 64 and lens.max() <= 1 << 20
    assert 0.9e5 < lens.mean() < 1.3e5               # E[len] = (2^20 - 64) / ln(2^14) ~ 1.08e5
