// Parallel float32 CPU baseline of the skeleton hot path -- MEASUREMENT ONLY.
//
// A multi-core CPU implementation of the same skeleton calls, in float32
// (int32 for the integer scan), run over as many std::threads as the caller
// asks for (the benchmark passes the cores of its affinity mask).  It is the
// CPU reference point for the GPU's throughput, separate from the float64
// oracle (which is sequential and exists to check results): it shares no
// code with the oracle or with libskel.so.  Every function splits its index
// range into one contiguous chunk per thread.
//
// Definitions (Sec. III skeletons; the readings of the weights and
// boundaries are those of the GPU library): axpy out = a x + y; reduce sum /
// max; dot = sum x y; scans inclusive / exclusive by two passes (chunk sums,
// then each chunk rescanned from its prefix); the 3 x 3 stencil and the 1D
// stencil of radius r with clamped (edge-replicated) neighbours; rowdot
// out[i] = sum_k A[k] M[i, k]; gather out[i] = A[clamp(idx[i])]; batched sum
// of squares and inclusive scan per CSR instance; backward: tanh adjoint,
// reverse inclusive scan, transposed 3 x 3 clamp stencil (gather form).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

template <class F>
void par_for(int nthreads, int64_t n, F fn)
{
    if (nthreads < 1) nthreads = 1;
    if (n < (int64_t)nthreads * 1024) nthreads = 1;
    if (nthreads == 1) {
        fn(int64_t(0), n, 0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nthreads);
    for (int t = 0; t < nthreads; ++t) {
        const int64_t lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
        th.emplace_back([=] { fn(lo, hi, t); });
    }
    for (auto &x : th) x.join();
}

inline int64_t clampi(int64_t i, int64_t n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

template <class T, bool INCL>
void scan_two_pass(const T *x, T *out, int64_t n, int nthreads)
{
    if (n < (int64_t)nthreads * 1024) nthreads = 1;
    std::vector<T> sums(nthreads + 1, T(0));
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        T s = T(0);
        for (int64_t i = lo; i < hi; ++i) s += x[i];
        sums[t + 1] = s;
    });
    for (int t = 0; t < nthreads; ++t) sums[t + 1] += sums[t];
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        T run = sums[t];
        for (int64_t i = lo; i < hi; ++i) {
            if (INCL) {
                run += x[i];
                out[i] = run;
            } else {
                out[i] = run;
                run += x[i];
            }
        }
    });
}

}  // namespace

extern "C" {

void cpu_map_axpy(const float *x, const float *y, float *out, int64_t n, float a, int nthreads)
{
    par_for(nthreads, n, [=](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; ++i) out[i] = a * x[i] + y[i];
    });
}

float cpu_reduce_sum(const float *x, int64_t n, int nthreads)
{
    std::vector<float> part(std::max(nthreads, 1), 0.f);
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int64_t i = lo;
        for (; i + 8 <= hi; i += 8)
            for (int k = 0; k < 8; ++k) a[k] += x[i + k];
        for (; i < hi; ++i) a[0] += x[i];
        part[t] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    });
    float s = 0.f;
    for (float v : part) s += v;
    return s;
}

float cpu_reduce_max(const float *x, int64_t n, int nthreads)
{
    std::vector<float> part(std::max(nthreads, 1), -INFINITY);
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        float a[8];
        for (int k = 0; k < 8; ++k) a[k] = -INFINITY;
        int64_t i = lo;
        for (; i + 8 <= hi; i += 8)
            for (int k = 0; k < 8; ++k) a[k] = std::max(a[k], x[i + k]);
        for (; i < hi; ++i) a[0] = std::max(a[0], x[i]);
        float m = a[0];
        for (int k = 1; k < 8; ++k) m = std::max(m, a[k]);
        part[t] = m;
    });
    float m = -INFINITY;
    for (float v : part) m = std::max(m, v);
    return m;
}

float cpu_dot(const float *x, const float *y, int64_t n, int nthreads)
{
    std::vector<float> part(std::max(nthreads, 1), 0.f);
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int64_t i = lo;
        for (; i + 8 <= hi; i += 8)
            for (int k = 0; k < 8; ++k) a[k] += x[i + k] * y[i + k];
        for (; i < hi; ++i) a[0] += x[i] * y[i];
        part[t] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    });
    float s = 0.f;
    for (float v : part) s += v;
    return s;
}

// int32 scans wrap modulo 2^32 (unsigned arithmetic on the bit patterns).
void cpu_scan_i32(const int32_t *x, int32_t *out, int64_t n, int inclusive, int nthreads)
{
    const uint32_t *ux = reinterpret_cast<const uint32_t *>(x);
    uint32_t *uo = reinterpret_cast<uint32_t *>(out);
    if (inclusive) scan_two_pass<uint32_t, true>(ux, uo, n, nthreads);
    else scan_two_pass<uint32_t, false>(ux, uo, n, nthreads);
}

void cpu_scan_f32(const float *x, float *out, int64_t n, int inclusive, int nthreads)
{
    if (inclusive) scan_two_pass<float, true>(x, out, n, nthreads);
    else scan_two_pass<float, false>(x, out, n, nthreads);
}

// Reverse inclusive scan: out[i] = x[i] + ... + x[n-1] (the adjoint of the
// inclusive scan), two passes over the chunks from the end.
void cpu_scan_bwd_f32(const float *g, float *out, int64_t n, int nthreads)
{
    if (n < (int64_t)nthreads * 1024) nthreads = 1;
    std::vector<float> sums(nthreads + 1, 0.f);
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        float s = 0.f;
        for (int64_t i = lo; i < hi; ++i) s += g[i];
        sums[t] = s;
    });
    for (int t = nthreads - 1; t >= 0; --t) sums[t] += sums[t + 1];   // sums[t] = suffix from chunk t
    par_for(nthreads, n, [&](int64_t lo, int64_t hi, int t) {
        float run = sums[t + 1];
        for (int64_t i = hi - 1; i >= lo; --i) {
            run += g[i];
            out[i] = run;
        }
    });
}

// 3 x 3 stencil, w row-major over (di, dj) in [-1, 1]^2, clamp boundary.
void cpu_stencil2d(const float *x, float *out, int64_t rows, int64_t cols, const float *w, int nthreads)
{
    par_for(nthreads, rows, [=](int64_t r0, int64_t r1, int) {
        for (int64_t i = r0; i < r1; ++i) {
            const float *rm = x + clampi(i - 1, rows) * cols, *rc = x + i * cols, *rp = x + clampi(i + 1, rows) * cols;
            auto at = [&](int64_t j, int64_t jm, int64_t jp) {
                return w[0] * rm[jm] + w[1] * rm[j] + w[2] * rm[jp] + w[3] * rc[jm] + w[4] * rc[j] + w[5] * rc[jp] +
                       w[6] * rp[jm] + w[7] * rp[j] + w[8] * rp[jp];
            };
            float *o = out + i * cols;
            o[0] = at(0, 0, clampi(1, cols));
            for (int64_t j = 1; j < cols - 1; ++j) o[j] = at(j, j - 1, j + 1);   // interior: no clamping
            if (cols > 1) o[cols - 1] = at(cols - 1, cols - 2, cols - 1);
        }
    });
}

void cpu_stencil1d(const float *x, float *out, int64_t n, int r, const float *w, int nthreads)
{
    par_for(nthreads, n, [=](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; ++i) {
            float s = 0.f;
            if (i >= r && i + r < n) {
                const float *xi = x + i - r;
                for (int k = 0; k <= 2 * r; ++k) s += w[k] * xi[k];
            } else {
                for (int k = -r; k <= r; ++k) s += w[k + r] * x[clampi(i + k, n)];
            }
            out[i] = s;
        }
    });
}

// Transposed 3 x 3 clamp stencil as a gather: the outputs o whose tap
// (di, dj) reads p.  Along one axis, output o reaches p = clamp(o + d):
// o = p - d inside, and additionally o + d = -1 at p = 0 and o + d = N at
// p = N - 1 (the clamped reads).
void cpu_stencil2d_bwd(const float *g, float *out, int64_t rows, int64_t cols, const float *w, int nthreads)
{
    auto sources = [](int64_t p, int d, int64_t n, int64_t *o) {   // o: up to 2 outputs
        int c = 0;
        const int64_t a = p - d;
        if (a >= 0 && a < n) o[c++] = a;
        if (p == 0 && -1 - d >= 0 && -1 - d < n) o[c++] = -1 - d;
        if (p == n - 1 && n - d >= 0 && n - d < n) o[c++] = n - d;
        return c;
    };
    par_for(nthreads, rows, [=](int64_t r0, int64_t r1, int) {
        for (int64_t i = r0; i < r1; ++i)
            for (int64_t j = 0; j < cols; ++j) {
                if (i > 0 && i < rows - 1 && j > 0 && j < cols - 1) {
                    // interior: exactly one output per tap, o = p - d
                    const float *gm = g + (i + 1) * cols + j, *gc = g + i * cols + j, *gp = g + (i - 1) * cols + j;
                    out[i * cols + j] = w[0] * gm[1] + w[1] * gm[0] + w[2] * gm[-1] + w[3] * gc[1] + w[4] * gc[0] +
                                        w[5] * gc[-1] + w[6] * gp[1] + w[7] * gp[0] + w[8] * gp[-1];
                    continue;
                }
                float s = 0.f;
                for (int di = -1; di <= 1; ++di) {
                    int64_t oi[2];
                    const int ni = sources(i, di, rows, oi);
                    for (int dj = -1; dj <= 1; ++dj) {
                        int64_t oj[2];
                        const int nj = sources(j, dj, cols, oj);
                        const float wv = w[(di + 1) * 3 + (dj + 1)];
                        for (int a = 0; a < ni; ++a)
                            for (int b = 0; b < nj; ++b) s += wv * g[oi[a] * cols + oj[b]];
                    }
                }
                out[i * cols + j] = s;
            }
    });
}

void cpu_rowdot(const float *A, const float *M, int64_t rows, int64_t m, float *out, int nthreads)
{
    par_for(nthreads, rows, [=](int64_t r0, int64_t r1, int) {
        for (int64_t i = r0; i < r1; ++i) {
            const float *row = M + i * m;
            float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            int64_t k = 0;
            for (; k + 8 <= m; k += 8)
                for (int q = 0; q < 8; ++q) a[q] += A[k + q] * row[k + q];
            for (; k < m; ++k) a[0] += A[k] * row[k];
            out[i] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        }
    });
}

void cpu_gather(const float *A, int64_t m, const int32_t *idx, int64_t n, float *out, int nthreads)
{
    par_for(nthreads, n, [=](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; ++i) out[i] = A[clampi(idx[i], m)];
    });
}

void cpu_map_tanh_bwd(const float *x, const float *g, float *out, int64_t n, int nthreads)
{
    par_for(nthreads, n, [=](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; ++i) {
            const float t = std::tanh(x[i]);
            out[i] = g[i] * (1.f - t * t);
        }
    });
}

// Batched instances: each thread takes whole instances from a shared counter.
void cpu_batched(const float *v, const int64_t *off, int64_t B, float *res, float *scan, int nthreads)
{
    std::atomic<int64_t> next(0);
    const int nt = std::max(1, std::min<int>(nthreads, (int)std::max<int64_t>(B, 1)));
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (int64_t b; (b = next.fetch_add(1)) < B;) {
                float q = 0.f, run = 0.f;
                for (int64_t i = off[b]; i < off[b + 1]; ++i) {
                    q += v[i] * v[i];
                    run += v[i];
                    scan[i] = run;
                }
                res[b] = q;
            }
        });
    for (auto &x : th) x.join();
}

}  // extern "C"
