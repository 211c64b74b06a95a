/*
 * CPU oracle for the skeleton hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file.  The product library never links, calls or includes it, and
 * this file includes nothing of the product (no shared header, table or
 * helper).  It is deliberately plain and slow: one sequential loop per
 * definition, float64 arithmetic for float32 inputs (every float32 widens
 * exactly) and int64 arithmetic for int32 inputs.
 *
 * Definitions followed (Kessler, Dastgeer, Li, "Optimized Composition", 2014):
 *   - Sec. III: skeletons are generic components derived from the
 *     higher-order functions map, scan and reduce, instantiated with a user
 *     function; the SkePU set adds mapoverlap (a map whose user function also
 *     reads a fixed neighbourhood of each element).
 *   - Sec. II (related work, Merge): MapReduce, here read as a reduce over a
 *     mapped sequence, r = (+)_i f(x_i, y_i).
 *   - MapArray has no definition in the paper; the reading used is
 *     out[i] = f(A, B[i]) with A read whole (random access) and B per element
 *     (or, for the Coulombic potential grid of Sec. III, the element's own
 *     grid position).
 *   - Sec. II (composition of components): a chain of calls is the
 *     definitions applied one after the other, every intermediate kept in
 *     float64 (oracle_mapoverlap2d_chain_f32, the composed loss and
 *     oracle_chain_map_stencil_sumsq_f32).
 *   - Backward passes are the adjoints of these linear/elementwise maps,
 *     written from their definitions (scatter form), not from the GPU design.
 *
 * Boundary handling of mapoverlap is not given by the paper.  Reading used:
 *   clamp (edge replicate), zero (outside reads as 0) and periodic (wrap).
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared oracle.c -lm.
 * -ffp-contract=off keeps every multiply and add separately rounded, so the
 * results are the same on x86-64 and AArch64 hosts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Oracle-local codes (the Python wrapper maps names onto these). */
enum { OR_AXPY = 0, OR_MUL = 1, OR_ADD = 2, OR_TANH = 3, OR_SQ = 4, OR_SCALE = 5,
       OR_COPY = 6, OR_SUB = 7, OR_MAX = 8 };
enum { OR_CLAMP = 0, OR_ZERO = 1, OR_PERIODIC = 2 };

/* ---------------------------------------------------------------- Map --- */

/* Sec. III map: out[i] = f(x[i], y[i]) for every i.  y may be NULL for the
 * unary functions.  a is the scalar parameter (axpy, scale). */
static double map_fn(int fn, double a, double x, double y)
{
    switch (fn) {
    case OR_AXPY:  return a * x + y;
    case OR_MUL:   return x * y;
    case OR_ADD:   return x + y;
    case OR_SUB:   return x - y;
    case OR_MAX:   return x > y ? x : y;
    case OR_TANH:  return tanh(x);
    case OR_SQ:    return x * x;
    case OR_SCALE: return a * x;
    case OR_COPY:  return x;
    default:       return NAN;
    }
}

int oracle_map_f32(int fn, double a, const float *x, const float *y, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = map_fn(fn, a, (double)x[i], y ? (double)y[i] : 0.0);
    return 0;
}

/* Backward of map (adjoint of an elementwise map is elementwise):
 *   gx[i] = g[i] * df/dx(x[i], y[i]),  gy[i] = g[i] * df/dy(x[i], y[i]).
 * gy may be NULL for unary functions. */
int oracle_map_bwd_f32(int fn, double a, const float *x, const float *y, const float *g,
                       int64_t n, double *gx, double *gy)
{
    for (int64_t i = 0; i < n; ++i) {
        double xi = x ? (double)x[i] : 0.0, yi = y ? (double)y[i] : 0.0, gi = (double)g[i];
        double dx = 0.0, dy = 0.0;
        switch (fn) {
        case OR_AXPY:  dx = a;   dy = 1.0; break;
        case OR_MUL:   dx = yi;  dy = xi;  break;
        case OR_ADD:   dx = 1.0; dy = 1.0; break;
        case OR_SUB:   dx = 1.0; dy = -1.0; break;
        case OR_TANH: { double t = tanh(xi); dx = 1.0 - t * t; } break;
        case OR_SQ:    dx = 2.0 * xi; break;
        case OR_SCALE: dx = a; break;
        case OR_COPY:  dx = 1.0; break;
        default:       dx = NAN; dy = NAN; break;
        }
        gx[i] = gi * dx;
        if (gy) gy[i] = gi * dy;
    }
    return 0;
}

/* ------------------------------------------------------------- Reduce --- */

/* Sec. III reduce with (+): sequential sum in float64.  *abs_sum receives
 * sum |x_i| (the scale of the rounding-error bound). */
double oracle_reduce_sum_f32(const float *x, int64_t n, double *abs_sum)
{
    double s = 0.0, a = 0.0;
    for (int64_t i = 0; i < n; ++i) { s += (double)x[i]; a += fabs((double)x[i]); }
    if (abs_sum) *abs_sum = a;
    return s;
}

/* Sec. III reduce with max; the identity of max is -infinity (n = 0). */
double oracle_reduce_max_f32(const float *x, int64_t n)
{
    double m = -INFINITY;
    for (int64_t i = 0; i < n; ++i) if ((double)x[i] > m) m = (double)x[i];
    return m;
}

/* Integer (+): exact int64 sum; the int32 result of the GPU is this modulo 2^32. */
int64_t oracle_reduce_sum_i32(const int32_t *x, int64_t n)
{
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) s += (int64_t)x[i];
    return s;
}

int32_t oracle_reduce_max_i32(const int32_t *x, int64_t n)
{
    int32_t m = INT32_MIN;
    for (int64_t i = 0; i < n; ++i) if (x[i] > m) m = x[i];
    return m;
}

/* MapReduce: r = sum_i f(x_i, y_i), f one of the map functions above (dot:
 * f = mul; sum of squares: f = sq).  Products of two float32 values are exact
 * in float64, so each mapped term is exact.  *abs_sum = sum_i |f(x_i, y_i)|. */
double oracle_mapreduce_f32(int fn, double a, const float *x, const float *y, int64_t n,
                            double *abs_sum)
{
    double s = 0.0, as = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = map_fn(fn, a, (double)x[i], y ? (double)y[i] : 0.0);
        s += t;
        as += fabs(t);
    }
    if (abs_sum) *abs_sum = as;
    return s;
}

/* --------------------------------------------------------------- Scan --- */

/* Sec. III scan with (+).  inclusive: out[i] = sum_{j<=i} x[j];
 * exclusive: out[0] = 0, out[i] = sum_{j<i} x[j].  int64, exact. */
void oracle_scan_i32(const int32_t *x, int64_t n, int inclusive, int64_t *out)
{
    int64_t run = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (inclusive) { run += (int64_t)x[i]; out[i] = run; }
        else           { out[i] = run; run += (int64_t)x[i]; }
    }
}

/* float32 input, float64 running sum.  abs_prefix[i] is the matching running
 * sum of |x| (same index range as out[i]), the scale of the error bound. */
void oracle_scan_f32(const float *x, int64_t n, int inclusive, double *out, double *abs_prefix)
{
    double run = 0.0, arun = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (inclusive) {
            run += (double)x[i]; arun += fabs((double)x[i]);
            out[i] = run; if (abs_prefix) abs_prefix[i] = arun;
        } else {
            out[i] = run; if (abs_prefix) abs_prefix[i] = arun;
            run += (double)x[i]; arun += fabs((double)x[i]);
        }
    }
}

/* Backward of scan (+).  The scan is the linear map out = L x with L lower
 * triangular (inclusive) or strictly lower triangular (exclusive); its adjoint
 * is gx = L^T g, i.e. gx[j] = sum_{i>=j} g[i] (inclusive) or sum_{i>j} g[i]
 * (exclusive).  Written here as the column sums of L, one loop per j would be
 * O(n^2), so the suffix is accumulated from the end -- the same sums. */
void oracle_scan_bwd_f32(const float *g, int64_t n, int inclusive, double *gx, double *abs_suffix)
{
    double run = 0.0, arun = 0.0;
    for (int64_t j = n - 1; j >= 0; --j) {
        if (inclusive) {
            run += (double)g[j]; arun += fabs((double)g[j]);
            gx[j] = run; if (abs_suffix) abs_suffix[j] = arun;
        } else {
            gx[j] = run; if (abs_suffix) abs_suffix[j] = arun;
            run += (double)g[j]; arun += fabs((double)g[j]);
        }
    }
}

/* --------------------------------------------------------- MapOverlap --- */

/* Index map of the boundary reading: returns the source index for a logical
 * index k of an axis of length n, or -1 when the read is the value 0. */
static int64_t bmap(int64_t k, int64_t n, int boundary)
{
    if (k >= 0 && k < n) return k;
    switch (boundary) {
    case OR_CLAMP:    return k < 0 ? 0 : n - 1;
    case OR_PERIODIC: { int64_t m = k % n; return m < 0 ? m + n : m; }
    default:          return -1;
    }
}

/* 1D mapoverlap: out[i] = sum_{k=-r..r} w[k+r] * x[b(i+k)].  w holds the
 * float32 weights the GPU receives (widened exactly). */
void oracle_mapoverlap1d_f32(const float *x, int64_t n, int r, const float *w, int boundary,
                             double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = -r; k <= r; ++k) {
            int64_t src = bmap(i + k, n, boundary);
            double v = src < 0 ? 0.0 : (double)x[src];
            s += (double)w[k + r] * v;
        }
        out[i] = s;
    }
}

/* 2D mapoverlap on a row-major rows x cols grid:
 * out[i,j] = sum_{di,dj in [-r,r]} w[di,dj] * x[b(i+di), b(j+dj)],
 * w row-major (2r+1) x (2r+1), w[(di+r)*(2r+1) + (dj+r)].  The boundary map
 * acts on each axis separately.  A 5-point cross is the 3x3 case with zero
 * corners. */
void oracle_mapoverlap2d_f32(const float *x, int64_t rows, int64_t cols, int r, const float *w,
                             int boundary, double *out)
{
    const int side = 2 * r + 1;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            double s = 0.0;
            for (int di = -r; di <= r; ++di) {
                int64_t si = bmap(i + di, rows, boundary);
                for (int dj = -r; dj <= r; ++dj) {
                    int64_t sj = bmap(j + dj, cols, boundary);
                    double v = (si < 0 || sj < 0) ? 0.0 : (double)x[si * cols + sj];
                    s += (double)w[(di + r) * side + (dj + r)] * v;
                }
            }
            out[i * cols + j] = s;
        }
}

/* A chain of `steps` 2D mapoverlap applications, out = S^steps(x), every
 * intermediate kept in float64 (the composition of the definition above). */
void oracle_mapoverlap2d_chain_f32(const float *x, int64_t rows, int64_t cols, int r, const float *w,
                                   int boundary, int steps, double *out)
{
    const int side = 2 * r + 1;
    const int64_t n = rows * cols;
    double *cur = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *nxt = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t p = 0; p < n; ++p) cur[p] = (double)x[p];
    for (int k = 0; k < steps; ++k) {
        for (int64_t i = 0; i < rows; ++i)
            for (int64_t j = 0; j < cols; ++j) {
                double s = 0.0;
                for (int di = -r; di <= r; ++di) {
                    int64_t si = bmap(i + di, rows, boundary);
                    for (int dj = -r; dj <= r; ++dj) {
                        int64_t sj = bmap(j + dj, cols, boundary);
                        double v = (si < 0 || sj < 0) ? 0.0 : cur[si * cols + sj];
                        s += (double)w[(di + r) * side + (dj + r)] * v;
                    }
                }
                nxt[i * cols + j] = s;
            }
        double *t = cur; cur = nxt; nxt = t;
    }
    for (int64_t p = 0; p < n; ++p) out[p] = cur[p];
    free(cur);
    free(nxt);
}

/* Backward of 1D mapoverlap, by scatter from the forward definition: each
 * forward output i read x[b(i+k)] with weight w[k], so g[i] * w[k] flows back
 * to source index b(i+k).  Clamped taps therefore fold onto the edge. */
void oracle_mapoverlap1d_bwd_f32(const float *g, int64_t n, int r, const float *w, int boundary,
                                 double *gx)
{
    for (int64_t i = 0; i < n; ++i) gx[i] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int k = -r; k <= r; ++k) {
            int64_t src = bmap(i + k, n, boundary);
            if (src >= 0) gx[src] += (double)w[k + r] * (double)g[i];
        }
}

/* Backward of 2D mapoverlap, by scatter (see the 1D case). */
void oracle_mapoverlap2d_bwd_f32(const float *g, int64_t rows, int64_t cols, int r,
                                 const float *w, int boundary, double *gx)
{
    const int side = 2 * r + 1;
    for (int64_t p = 0; p < rows * cols; ++p) gx[p] = 0.0;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            double gij = (double)g[i * cols + j];
            for (int di = -r; di <= r; ++di) {
                int64_t si = bmap(i + di, rows, boundary);
                if (si < 0) continue;
                for (int dj = -r; dj <= r; ++dj) {
                    int64_t sj = bmap(j + dj, cols, boundary);
                    if (sj < 0) continue;
                    gx[si * cols + sj] += (double)w[(di + r) * side + (dj + r)] * gij;
                }
            }
        }
}

/* ----------------------------------------------------------- MapArray --- */

/* gather: out[i] = A[clamp(idx[i], 0, m-1)]. */
void oracle_gather_f32(const float *A, int64_t m, const int32_t *idx, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = idx[i];
        if (k < 0) k = 0;
        if (k > m - 1) k = m - 1;
        out[i] = m > 0 ? (double)A[k] : 0.0;
    }
}

/* rowdot: out[i] = sum_k A[k] * M[i, k], M row-major n x m.
 * abs_out[i] = sum_k |A[k] * M[i, k]|. */
void oracle_rowdot_f32(const float *A, int64_t m, const float *M, int64_t n, double *out,
                       double *abs_out)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, a = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            double t = (double)A[k] * (double)M[i * m + k];
            s += t; a += fabs(t);
        }
        out[i] = s;
        if (abs_out) abs_out[i] = a;
    }
}

/* Coulombic potential grid (Sec. III, the application of Fig. 2, written
 * there as a MapArray over the atoms): grid point (i, j) sits at
 * (j*h, i*h, z0); atoms[k] = (x, y, z, q) as float32, row-major m x 4.
 *   out[p] = sum_k q_k / sqrt((x_p - x_k)^2 + (y_p - y_k)^2 + (z0 - z_k)^2)
 *   abs_out[p] = sum_k |q_k| / r_k
 * for the npts points (ii[p], jj[p]); float64 throughout (a coinciding atom
 * gives an infinite term, as the definition does). */
void oracle_coulomb_points_f32(const float *atoms, int64_t m, const int64_t *ii, const int64_t *jj, int64_t npts,
                               double h, double z0, double *out, double *abs_out)
{
    for (int64_t p = 0; p < npts; ++p) {
        const double x = (double)jj[p] * h, y = (double)ii[p] * h;
        double s = 0.0, a = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            const double dx = x - (double)atoms[4 * k], dy = y - (double)atoms[4 * k + 1];
            const double dz = z0 - (double)atoms[4 * k + 2], q = (double)atoms[4 * k + 3];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            s += q / r;
            a += fabs(q) / r;
        }
        out[p] = s;
        if (abs_out) abs_out[p] = a;
    }
}

/* ------------------------------------------------------------ Batched --- */

/* Independent instances laid end to end: instance b is v[off[b] .. off[b+1]).
 * Per instance: sumsq[b] = sum x^2 (MapReduce) and the inclusive or exclusive
 * scan (+) of its elements, written at the same positions.  abs_prefix as in
 * oracle_scan_f32, restarted per instance. */
void oracle_batched_f32(const float *v, const int64_t *off, int64_t B, int inclusive,
                        double *sumsq, double *scan_out, double *abs_prefix)
{
    for (int64_t b = 0; b < B; ++b) {
        int64_t lo = off[b], hi = off[b + 1];
        if (sumsq) sumsq[b] = oracle_mapreduce_f32(OR_SQ, 0.0, v + lo, NULL, hi - lo, NULL);
        if (scan_out)
            oracle_scan_f32(v + lo, hi - lo, inclusive, scan_out + lo,
                            abs_prefix ? abs_prefix + lo : NULL);
    }
}

/* ----------------------------------------------- Composed differentiable --- */

/* Row-wise inclusive scan of a rows x cols grid (each row an instance). */
static void row_scan(const double *t, int64_t rows, int64_t cols, double *s)
{
    for (int64_t i = 0; i < rows; ++i) {
        double run = 0.0;
        for (int64_t j = 0; j < cols; ++j) { run += t[i * cols + j]; s[i * cols + j] = run; }
    }
}

/* 2D mapoverlap of a float64 grid (same definition as above). */
static void stencil2d_f64(const double *x, int64_t rows, int64_t cols, int r, const float *w,
                          int boundary, double *out)
{
    const int side = 2 * r + 1;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            double s = 0.0;
            for (int di = -r; di <= r; ++di) {
                int64_t si = bmap(i + di, rows, boundary);
                for (int dj = -r; dj <= r; ++dj) {
                    int64_t sj = bmap(j + dj, cols, boundary);
                    double v = (si < 0 || sj < 0) ? 0.0 : x[si * cols + sj];
                    s += (double)w[(di + r) * side + (dj + r)] * v;
                }
            }
            out[i * cols + j] = s;
        }
}

/* Composed loss on a rows x cols grid x:
 *   t = tanh(x)                      (Map)
 *   u = S t                          (MapOverlap, weights w, radius r, boundary)
 *   L1 = sum u^2                     (MapReduce: sq, +)
 *   s = row-wise inclusive scan of t (Scan per row)
 *   C = (1 / (rows * cols)) * sum s^2
 *   L = L1 + C
 * The gradient (if grad != NULL) follows the chain rule in the reverse order:
 *   gu = 2u, gt = S^T gu (scatter form), gs = 2 s / (rows*cols),
 *   gt += reverse row-scan of gs, gx = gt * (1 - t^2).
 * Returns L.  Work arrays are allocated here (malloc). */
double oracle_composed_loss_f32(const float *x, int64_t rows, int64_t cols, int r, const float *w,
                                int boundary, double *grad)
{
    const int64_t N = rows * cols;
    const int side = 2 * r + 1;
    double *t = malloc(sizeof(double) * N), *u = malloc(sizeof(double) * N),
           *s = malloc(sizeof(double) * N);
    if (!t || !u || !s) { free(t); free(u); free(s); return NAN; }
    for (int64_t p = 0; p < N; ++p) t[p] = tanh((double)x[p]);
    stencil2d_f64(t, rows, cols, r, w, boundary, u);
    row_scan(t, rows, cols, s);
    double L1 = 0.0, C = 0.0;
    for (int64_t p = 0; p < N; ++p) L1 += u[p] * u[p];
    for (int64_t p = 0; p < N; ++p) C += s[p] * s[p];
    C /= (double)N;
    if (grad) {
        /* gt = S^T (2u), scatter */
        for (int64_t p = 0; p < N; ++p) grad[p] = 0.0;
        for (int64_t i = 0; i < rows; ++i)
            for (int64_t j = 0; j < cols; ++j) {
                double gu = 2.0 * u[i * cols + j];
                for (int di = -r; di <= r; ++di) {
                    int64_t si = bmap(i + di, rows, boundary);
                    if (si < 0) continue;
                    for (int dj = -r; dj <= r; ++dj) {
                        int64_t sj = bmap(j + dj, cols, boundary);
                        if (sj < 0) continue;
                        grad[si * cols + sj] += (double)w[(di + r) * side + (dj + r)] * gu;
                    }
                }
            }
        /* + reverse row-scan of gs = 2 s / N */
        for (int64_t i = 0; i < rows; ++i) {
            double run = 0.0;
            for (int64_t j = cols - 1; j >= 0; --j) {
                run += 2.0 * s[i * cols + j] / (double)N;
                grad[i * cols + j] += run;
            }
        }
        /* through tanh */
        for (int64_t p = 0; p < N; ++p) grad[p] *= 1.0 - t[p] * t[p];
    }
    free(t); free(u); free(s);
    return L1 + C;
}

/* The same loss evaluated on a float64 grid (for finite differences, where a
 * probe perturbs x by h and float32 would round the perturbation away). */
double oracle_composed_loss_f64(const double *x, int64_t rows, int64_t cols, int r,
                                const float *w, int boundary)
{
    const int64_t N = rows * cols;
    double *t = malloc(sizeof(double) * N), *u = malloc(sizeof(double) * N),
           *s = malloc(sizeof(double) * N);
    if (!t || !u || !s) { free(t); free(u); free(s); return NAN; }
    for (int64_t p = 0; p < N; ++p) t[p] = tanh(x[p]);
    stencil2d_f64(t, rows, cols, r, w, boundary, u);
    row_scan(t, rows, cols, s);
    double L1 = 0.0, C = 0.0;
    for (int64_t p = 0; p < N; ++p) L1 += u[p] * u[p];
    for (int64_t p = 0; p < N; ++p) C += s[p] * s[p];
    free(t); free(u); free(s);
    return L1 + C / (double)N;
}

/* The chain Map -> MapOverlap -> MapReduce as three composed skeleton calls
 * (Sec. II: a composition of components; here the definitions applied one
 * after the other, every intermediate in float64):
 *   t = f(x)                   Sec. III map with a unary user function
 *   u = S t                    2D mapoverlap, the definition of
 *                              oracle_mapoverlap2d_f32 applied to t
 *   result = sum_p u_p^2       MapReduce with sq and +
 * *bound receives sum_p (sum_taps |w| |t|)^2, the scale of the rounding error
 * of a float32 evaluation of the chain (every tap of every stencil output at
 * its largest magnitude, squared).  Returns the result. */
double oracle_chain_map_stencil_sumsq_f32(int fn, double a, const float *x, int64_t rows, int64_t cols, int r,
                                          const float *w, int boundary, double *bound)
{
    const int64_t N = rows * cols;
    const int side = 2 * r + 1;
    double *t = malloc(sizeof(double) * (N > 0 ? N : 1)), *u = malloc(sizeof(double) * (N > 0 ? N : 1));
    if (!t || !u) { free(t); free(u); return NAN; }
    for (int64_t p = 0; p < N; ++p) t[p] = map_fn(fn, a, (double)x[p], 0.0);
    stencil2d_f64(t, rows, cols, r, w, boundary, u);
    double sum = 0.0, scale = 0.0;
    for (int64_t p = 0; p < N; ++p) sum += u[p] * u[p];
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            double m = 0.0;
            for (int di = -r; di <= r; ++di) {
                int64_t si = bmap(i + di, rows, boundary);
                for (int dj = -r; dj <= r; ++dj) {
                    int64_t sj = bmap(j + dj, cols, boundary);
                    if (si < 0 || sj < 0) continue;
                    m += fabs((double)w[(di + r) * side + (dj + r)]) * fabs(t[si * cols + sj]);
                }
            }
            scale += m * m;
        }
    if (bound) *bound = scale;
    free(t); free(u);
    return sum;
}

/* Local change of the composed loss when x[pi,pj] moves from x0 to x0 + h,
 * evaluated on the float32 grid widened to float64.  Only the outputs that
 * read the probe change: the (2r+1)^2 stencil outputs around it (squared
 * pointwise) and the suffix of its row scan.  Returning L(x+h e) - L(x)
 * directly, instead of differencing two full sums of size rows*cols, keeps
 * cancellation out of the finite difference. */
double oracle_composed_loss_delta_f32(const float *x, int64_t rows, int64_t cols, int r,
                                      const float *w, int boundary, int64_t pi, int64_t pj,
                                      double h)
{
    const int side = 2 * r + 1;
    const int64_t N = rows * cols;
    const double x0 = (double)x[pi * cols + pj];
    const double dt = tanh(x0 + h) - tanh(x0);
    /* stencil term: outputs (i,j) that read source (pi,pj) through some tap */
    double d1 = 0.0;
    /* Every output (i,j) with a tap whose mapped source is (pi,pj): a row i
     * qualifies when some di maps i+di onto pi, a column likewise; with clamp
     * or periodic boundaries this includes outputs beyond distance r. */
    for (int64_t i = 0; i < rows; ++i) {
        int row_hit = 0;
        for (int di = -r; di <= r && !row_hit; ++di) row_hit = (bmap(i + di, rows, boundary) == pi);
        if (!row_hit) continue;
        for (int64_t j = 0; j < cols; ++j) {
            int col_hit = 0;
            for (int dj = -r; dj <= r && !col_hit; ++dj) col_hit = (bmap(j + dj, cols, boundary) == pj);
            if (!col_hit) continue;
            double old = 0.0, delta = 0.0;
            for (int di = -r; di <= r; ++di) {
                int64_t si = bmap(i + di, rows, boundary);
                for (int dj = -r; dj <= r; ++dj) {
                    int64_t sj = bmap(j + dj, cols, boundary);
                    if (si < 0 || sj < 0) continue;
                    double wv = (double)w[(di + r) * side + (dj + r)];
                    old += wv * tanh((double)x[si * cols + sj]);
                    if (si == pi && sj == pj) delta += wv * dt;
                }
            }
            d1 += delta * (2.0 * old + delta);
        }
    }
    /* scan term: s[pi, j] for j >= pj changes by dt */
    double run = 0.0, d2 = 0.0;
    for (int64_t j = 0; j < cols; ++j) {
        run += tanh((double)x[pi * cols + j]);
        if (j >= pj) d2 += dt * (2.0 * run + dt);
    }
    return d1 + d2 / (double)N;
}
