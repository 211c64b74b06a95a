// MapArray over a grid: the Coulombic potential of a set of point charges on
// a regular 2D slice (the Coulombic potential grid application written with
// SkePU skeletons, Sec. III, Fig. 2).  A holds the m atoms (x, y, z, q); the
// element of out[i, j] is its own grid position (j*h, i*h, z0):
//
//   out[i, j] = sum_k q_k / sqrt((j*h - x_k)^2 + (i*h - y_k)^2 + (z0 - z_k)^2)
//
// The work is m reciprocal square roots per point, so the bound is the SFU
// (MUFU) rate, not HBM: one reciprocal square root, three FP32 operations and
// the share of a compensated add per (point, atom) pair.
//
// Accumulation: the terms of four consecutive atoms are summed pairwise and
// that partial is added to the point's total with Kahan compensation, so the
// rounding stays a few units of 2^-24 of sum |q_k / r_k| however many atoms
// there are (a plain float32 running sum over 4096 atoms would not).
//
// Variants:
//   0 direct  one point per thread, atoms read through the read-only path
//             (every lane of a warp reads the same atom: one broadcast).
//   1 tiled   a block stages 1024 atoms at a time in shared memory; each
//             thread owns 8 points of one row (stride 32, coalesced stores)
//             and shares (y, z) distances across them.
#include "common.cuh"

namespace skel {
namespace {

constexpr int kChunk = 1024;   // atoms staged per round (16 KiB)
constexpr int kPts = 8;        // points per thread (tiled)

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float y)
    {
        const float yc = y - c;
        const float t = s + yc;
        c = (t - s) - yc;
        s = t;
    }
};

// Hardware reciprocal square root (PTX rsqrt.approx.ftz.f32, max relative
// error 2^-22.9 per the PTX ISA).  A squared distance below 2^-126 is
// flushed to 0 and gives an infinite term, like a coinciding atom.
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The (point, atom) reciprocal distance; FMA-contracted squared distance.
__device__ __forceinline__ float rinv(float dx, float dyz2) { return rsqrt_hw(fmaf(dx, dx, dyz2)); }

// The (point, atom) term.
__device__ __forceinline__ float term(float dx, float dyz2, float q) { return q * rinv(dx, dyz2); }

__global__ void __launch_bounds__(256)
coulomb_direct(const float4 *__restrict__ atoms, int64_t m, float *__restrict__ out, int64_t rows, int64_t cols,
               float h, float z0)
{
    const int64_t total = rows * cols;
    for (int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x; p < total; p += (int64_t)gridDim.x * 256) {
        const int64_t i = p / cols, j = p - i * cols;
        const float x = (float)j * h, y = (float)i * h;
        Kahan acc;
        int64_t k = 0;
        for (; k + 4 <= m; k += 4) {
            float t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 a = __ldg(atoms + k + u);
                const float dy = y - a.y, dz = z0 - a.z;
                t[u] = term(x - a.x, fmaf(dy, dy, dz * dz), a.w);
            }
            acc.add((t[0] + t[1]) + (t[2] + t[3]));
        }
        for (; k < m; ++k) {
            const float4 a = __ldg(atoms + k);
            const float dy = y - a.y, dz = z0 - a.z;
            acc.add(term(x - a.x, fmaf(dy, dy, dz * dz), a.w));
        }
        out[p] = acc.s;
    }
}

// Block: 8 warps = 8 rows; lane l owns columns j0 + l + 32u, u < kPts.
__global__ void __launch_bounds__(256)
coulomb_tiled(const float4 *__restrict__ atoms, int64_t m, float *__restrict__ out, int64_t rows, int64_t cols,
              float h, float z0)
{
    __shared__ float4 sa[kChunk];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.y * 8 + w;
    const int64_t j0 = (int64_t)blockIdx.x * (32 * kPts) + lane;
    const float y = (float)i * h;
    float x[kPts];
#pragma unroll
    for (int u = 0; u < kPts; ++u) x[u] = (float)(j0 + 32 * u) * h;
    Kahan acc[kPts];
    for (int64_t c0 = 0; c0 < m; c0 += kChunk) {
        // stage the chunk; past the last atom: zero charges far away (term 0,
        // finite distance, so no 0 * inf)
        for (int t = threadIdx.x; t < kChunk; t += 256)
            sa[t] = c0 + t < m ? __ldg(atoms + c0 + t) : make_float4(1e18f, 1e18f, 1e18f, 0.f);
        __syncthreads();
        const int cnt = m - c0 < kChunk ? (int)(m - c0) : kChunk;
        const int groups = (cnt + 3) / 4;   // the padded atoms complete the last group
        for (int g = 0; g < groups; ++g) {
            float part[kPts];
#pragma unroll
            for (int u = 0; u < kPts; ++u) part[u] = 0.f;
            float t01[kPts];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 a = sa[4 * g + q];        // same address in every lane: broadcast
                const float dy = y - a.y, dz = z0 - a.z;
                const float dyz2 = fmaf(dy, dy, dz * dz);
#pragma unroll
                for (int u = 0; u < kPts; ++u) {
                    // pairwise: (t0 + t1) + (t2 + t3), the second product of
                    // each pair fused into its add
                    const float r = rinv(x[u] - a.x, dyz2);
                    if (q == 0 || q == 2) t01[u] = a.w * r;
                    else if (q == 1) part[u] = fmaf(a.w, r, t01[u]);
                    else part[u] = part[u] + fmaf(a.w, r, t01[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < kPts; ++u) acc[u].add(part[u]);
        }
        __syncthreads();
    }
    if (i >= rows) return;
#pragma unroll
    for (int u = 0; u < kPts; ++u)
        if (j0 + 32 * u < cols) out[i * cols + j0 + 32 * u] = acc[u].s;
}

int check_launch(const char *what)
{
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), what);
}

}  // namespace

int launch_coulomb(const CoulombLaunch &cl, const Choice &c, cudaStream_t s)
{
    if (cl.rows == 0 || cl.cols == 0) return SKEL_OK;
    if (c.block > 0 && c.block != 256) return fail(SKEL_ERR_INVALID_ARG, "coulomb: block must be 256");
    if (!aligned16(cl.atoms)) return fail(SKEL_ERR_INVALID_ARG, "coulomb: atoms must be 16-byte aligned");
    const float4 *a = reinterpret_cast<const float4 *>(cl.atoms);
    if (c.variant == 0) {
        int64_t g = ceil_div(cl.rows * cl.cols, 256);
        const int64_t cap = (int64_t)device_info().sms * 8 * 16;
        if (g > cap) g = cap;
        launch_kernel(coulomb_direct, (unsigned)g, 256, 0, s, a, cl.m, cl.out, cl.rows, cl.cols, cl.h, cl.z0);
        return check_launch("coulomb direct");
    }
    if (c.variant == 1) {
        const int64_t gx = ceil_div(cl.cols, 32 * kPts), gy = ceil_div(cl.rows, 8);
        if (gy > 65535 || gx > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "coulomb tiled: grid too large");
        launch_kernel(coulomb_tiled, dim3((unsigned)gx, (unsigned)gy), 256, 0, s, a, cl.m, cl.out, cl.rows, cl.cols,
                      cl.h, cl.z0);
        return check_launch("coulomb tiled");
    }
    return fail(SKEL_ERR_UNSUPPORTED, "coulomb: variant not offered");
}

}  // namespace skel
