// MapOverlap skeleton (SkePU mapoverlap, Sec. III): every output reads a fixed
// neighbourhood of its input position, with a boundary map per axis.
//
// 2D (radius 1; 5-point cross or 3x3 box, weights row-major over (di, dj)):
//   0 direct      one output per thread, nine cached global loads.
//   1 smem_tile   a block stages a 34 x 136 halo tile (128 x 32 outputs) in
//                 shared memory with 16-byte loads, then each thread computes
//                 a 4 x 4 output patch from shared memory.
//   2 tma_tile    the same tile, fetched by one TMA 2D copy
//                 (cp.async.bulk.tensor) completing on an mbarrier; TMA fills
//                 out-of-range cells with zeros, so edge tiles of CLAMP and
//                 PERIODIC grids rewrite their halo cells from global memory.
//   3 column_walk each warp owns a 128-column strip (4 columns per lane, one
//                 16-byte load per row) and walks down `tile` rows holding a
//                 three-row window in registers; left/right neighbours come
//                 from the adjacent lanes by shuffle.  No shared memory.
// 1D (radius 0..16, 2r+1 weights):
//   0 direct      one output per thread, 2r+1 cached global loads.
//   1 smem_tile   a block stages 2048 + 2r inputs in shared memory; each
//                 thread computes 8 consecutive outputs from a register
//                 window of 8 + 2r values.
//   2 bulk_tile   a block owns 4096 outputs; interior blocks fetch their
//                 inputs and halos with one cp.async.bulk on an mbarrier,
//                 each thread computes four 4-output groups from 16-byte
//                 shared-memory windows (input and output 16-byte aligned).
// Adjoint (transpose=true): the mirrored stencil w'(di,dj) = w(-di,-dj) with
// the same boundary for ZERO and PERIODIC.  For CLAMP, taps that the forward
// pass clamped onto an edge element fold their weight back onto that edge:
// only the first and last row/column (1D: the two end elements) receive such
// folded terms, so the interior runs the mirrored stencil and a fix-up kernel
// rewrites the border with the exact folded sums.
#include <cuda.h>

#include <mutex>

#include "stencil.cuh"

namespace skel {
namespace {

// ------------------------------------------------------------ 2D direct --
template <bool TAPS5>
__global__ void __launch_bounds__(256)
st2_direct(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t cols, int b, W9 w)
{
    const int64_t c = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    if (c >= cols) return;
    for (int64_t r = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.y * 8) {
        out[r * cols + c] = stencil9<TAPS5>(
            w, at2(in, r - 1, c - 1, rows, cols, b), at2(in, r - 1, c, rows, cols, b), at2(in, r - 1, c + 1, rows, cols, b),
            at2(in, r, c - 1, rows, cols, b), at2(in, r, c, rows, cols, b), at2(in, r, c + 1, rows, cols, b),
            at2(in, r + 1, c - 1, rows, cols, b), at2(in, r + 1, c, rows, cols, b), at2(in, r + 1, c + 1, rows, cols, b));
    }
}

// ------------------------------------------------------ 2D tiled (smem) --
constexpr int kTX = 128, kTY = 32;            // outputs per tile
constexpr int kSW = kTX + 8, kSH = kTY + 2;   // staged tile: cols tx0-4 .. tx0+131, rows ty0-1 .. ty0+32

// Computes the tile's outputs from the staged tile s (kSH x kSW floats):
// thread (tx, ty) of a 32 x 8 block owns columns 4tx..4tx+3 and rows 4ty..4ty+3.
template <bool TAPS5>
__device__ __forceinline__ void tile_compute(const float *s, float *__restrict__ out, int64_t tx0, int64_t ty0,
                                             int64_t rows, int64_t cols, const W9 &w)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // a warp is one row of 32 lanes
    const int64_t c = tx0 + 4 * tx;
    float rr[6][6];   // rows 4ty-1 .. 4ty+4, columns 4tx-1 .. 4tx+4
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float *row = s + (4 * ty + i) * kSW + 4 * tx + 4;   // staged row of output row 4ty+i-1
        const float4 q = *reinterpret_cast<const float4 *>(row);
        // left / right neighbours from the adjacent lanes; the warp's two edge
        // lanes read theirs from shared memory
        const float l = __shfl_up_sync(0xffffffffu, q.w, 1);
        const float r = __shfl_down_sync(0xffffffffu, q.x, 1);
        rr[i][0] = tx == 0 ? row[-1] : l;
        rr[i][1] = q.x; rr[i][2] = q.y; rr[i][3] = q.z; rr[i][4] = q.w;
        rr[i][5] = tx == 31 ? row[4] : r;
    }
    if (c >= cols) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = ty0 + 4 * ty + i;
        if (r >= rows) break;
        float4 o;
        float *op = &o.x;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            op[j] = stencil9<TAPS5>(w, rr[i][j], rr[i][j + 1], rr[i][j + 2], rr[i + 1][j], rr[i + 1][j + 1],
                                    rr[i + 1][j + 2], rr[i + 2][j], rr[i + 2][j + 1], rr[i + 2][j + 2]);
        dev::st_stream(reinterpret_cast<float4 *>(out + r * cols + c), o);
    }
}

template <bool TAPS5>
__global__ void __launch_bounds__(256)
st2_smem(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t cols, int b, W9 w)
{
    __shared__ __align__(16) float s[kSH * kSW];
    const int64_t tx0 = (int64_t)blockIdx.x * kTX, ty0 = (int64_t)blockIdx.y * kTY;
    // stage: kSH rows x kSW/4 groups of 4 columns (cols % 4 == 0: a group is
    // either entirely inside the grid or entirely outside)
    for (int g = threadIdx.x; g < kSH * (kSW / 4); g += 256) {
        const int sr = g / (kSW / 4), sg = g % (kSW / 4);
        const int64_t r = ty0 - 1 + sr, c = tx0 - 4 + 4 * sg;
        const int64_t gr = bmap(r, rows, b);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gr >= 0) {
            if (c >= 0 && c + 3 < cols) {
                v = dev::ld_stream(reinterpret_cast<const float4 *>(in + gr * cols + c));
            } else {
                float *vp = &v.x;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t gc = bmap(c + j, cols, b);
                    vp[j] = gc < 0 ? 0.f : __ldg(in + gr * cols + gc);
                }
            }
        }
        *reinterpret_cast<float4 *>(s + sr * kSW + 4 * sg) = v;
    }
    __syncthreads();
    tile_compute<TAPS5>(s, out, tx0, ty0, rows, cols, w);
}

// -------------------------------------------------------- 2D TMA tiled --
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <bool TAPS5>
__global__ void __launch_bounds__(256)
st2_tma(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ in, float *__restrict__ out,
        int64_t rows, int64_t cols, int b, W9 w, Control *ctl)
{
    // dynamic shared memory only (no static shared variables), so the tile
    // starts at the 1024-byte aligned base; the mbarrier follows the tile
    extern __shared__ __align__(1024) unsigned char dyn[];
    float *s = reinterpret_cast<float *>(dyn);
    uint64_t *bar = reinterpret_cast<uint64_t *>(dyn + kSH * kSW * 4);
    const int64_t tx0 = (int64_t)blockIdx.x * kTX, ty0 = (int64_t)blockIdx.y * kTY;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(smem_addr(bar)), "r"((uint32_t)(kSH * kSW * 4)) : "memory");
        const int x = (int)(tx0 - 4), y = (int)(ty0 - 1);   // x * 4 bytes is a multiple of 16
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3}], [%4];"
                     :: "r"(smem_addr(s)), "l"(&tmap), "r"(x), "r"(y), "r"(smem_addr(bar)) : "memory");
    }
    // every thread waits for phase 0 of the barrier, with an iteration bound
    uint32_t done = 0;
    for (uint32_t it = 0; it < (1u << 22) && !done; ++it) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(smem_addr(bar)) : "memory");
    }
    if (!__syncthreads_and(done)) {
        if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
        return;
    }
    // Edge tiles of CLAMP / PERIODIC grids: TMA filled out-of-range cells with
    // 0; rewrite them with the mapped values.
    if (b != SKEL_ZERO && (tx0 == 0 || ty0 == 0 || tx0 + kTX + 4 > cols || ty0 + kTY + 1 > rows)) {
        for (int i = threadIdx.x; i < kSH * kSW; i += 256) {
            const int sr = i / kSW, sc = i % kSW;
            const int64_t r = ty0 - 1 + sr, c = tx0 - 4 + sc;
            if (r < 0 || r >= rows || c < 0 || c >= cols) s[i] = at2(in, r, c, rows, cols, b);
        }
        __syncthreads();
    }
    tile_compute<TAPS5>(s, out, tx0, ty0, rows, cols, w);
}

// --------------------------------------------------- 2D column walk ----
struct Row6 { float l, x0, x1, x2, x3, r; };

template <bool TAPS5, int RH>
__global__ void __launch_bounds__(128)
st2_colwalk(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t cols, int b, W9 w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t strip0 = ((int64_t)blockIdx.x * 4 + warp) * 128;
    if (strip0 >= cols) return;                     // warp-uniform
    const int64_t c0 = strip0 + 4 * lane;
    const bool active = c0 < cols;                  // cols % 4 == 0: all four columns valid
    const int64_t r0 = (int64_t)blockIdx.y * RH;
    const int64_t r1 = r0 + RH < rows ? r0 + RH : rows;
    const int64_t cl = bmap(c0 - 1, cols, b), cr = bmap(c0 + 4, cols, b);
    const bool own_r = lane == 31 || c0 + 4 >= cols;

    auto load = [&](int64_t r) {
        Row6 v{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int64_t gr = bmap(r, rows, b);
        if (gr >= 0 && active) {
            const float4 q = dev::ld_stream(reinterpret_cast<const float4 *>(in + gr * cols + c0));
            v.x0 = q.x; v.x1 = q.y; v.x2 = q.z; v.x3 = q.w;
        }
        return v;
    };
    auto halo = [&](Row6 &v, int64_t r) {
        const float up = __shfl_up_sync(0xffffffffu, v.x3, 1);
        const float dn = __shfl_down_sync(0xffffffffu, v.x0, 1);
        const int64_t gr = bmap(r, rows, b);
        v.l = lane == 0 ? ((gr >= 0 && cl >= 0 && active) ? __ldg(in + gr * cols + cl) : 0.f) : up;
        v.r = own_r ? ((gr >= 0 && cr >= 0 && active) ? __ldg(in + gr * cols + cr) : 0.f) : dn;
    };

    Row6 a = load(r0 - 1), m = load(r0);
    halo(a, r0 - 1);
    halo(m, r0);
    constexpr int U = 4;
    for (int64_t r = r0; r < r1; r += U) {
        Row6 nx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) nx[u] = load(r + 1 + u);   // rows past r1 are loaded but unused
#pragma unroll
        for (int u = 0; u < U; ++u) halo(nx[u], r + 1 + u);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (r + u < r1 && active) {
                const Row6 &p = a, &q = m, &z = nx[u];
                float4 o;
                o.x = stencil9<TAPS5>(w, p.l, p.x0, p.x1, q.l, q.x0, q.x1, z.l, z.x0, z.x1);
                o.y = stencil9<TAPS5>(w, p.x0, p.x1, p.x2, q.x0, q.x1, q.x2, z.x0, z.x1, z.x2);
                o.z = stencil9<TAPS5>(w, p.x1, p.x2, p.x3, q.x1, q.x2, q.x3, z.x1, z.x2, z.x3);
                o.w = stencil9<TAPS5>(w, p.x2, p.x3, p.r, q.x2, q.x3, q.r, z.x2, z.x3, z.r);
                dev::st_stream(reinterpret_cast<float4 *>(out + (r + u) * cols + c0), o);
            }
            a = m;
            m = nx[u];
        }
    }
}

// ------------------------------------------- 2D clamp adjoint border ----
// Exact adjoint at the border cells of a CLAMP stencil: for every output
// (i, j) within one cell of (p, q) and every tap (di, dj) whose clamped
// source is (p, q), adds w(di, dj) * g(i, j).  Overwrites gin(p, q).
template <bool TAPS5>
__global__ void st2_fold_border(const float *__restrict__ g, float *__restrict__ gin, int64_t rows, int64_t cols, W9 w)
{
    const int64_t nb = rows == 1 ? cols : (cols == 1 ? rows : 2 * cols + 2 * (rows - 2));
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t p, q;
        if (rows == 1) { p = 0; q = k; }
        else if (cols == 1) { p = k; q = 0; }
        else if (k < cols) { p = 0; q = k; }
        else if (k < 2 * cols) { p = rows - 1; q = k - cols; }
        else { p = 1 + (k - 2 * cols) / 2; q = ((k - 2 * cols) & 1) ? cols - 1 : 0; }
        float acc = 0.f;
        for (int64_t i = p - 1; i <= p + 1; ++i) {
            if (i < 0 || i >= rows) continue;
            for (int64_t j = q - 1; j <= q + 1; ++j) {
                if (j < 0 || j >= cols) continue;
                const float gij = g[i * cols + j];
                for (int di = -1; di <= 1; ++di) {
                    if (bmap(i + di, rows, SKEL_CLAMP) != p) continue;
                    for (int dj = -1; dj <= 1; ++dj) {
                        if (TAPS5 && di != 0 && dj != 0) continue;
                        if (bmap(j + dj, cols, SKEL_CLAMP) != q) continue;
                        acc = fmaf(w.w[(di + 1) * 3 + (dj + 1)], gij, acc);
                    }
                }
            }
        }
        gin[p * cols + q] = acc;
    }
}

// --------------------------------------------------------------- 1D ----
template <int R>
__global__ void __launch_bounds__(256)
st1_direct(const float *__restrict__ in, float *__restrict__ out, int64_t n, int b, W33 w)
{
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        float acc = 0.f;
#pragma unroll
        for (int k = -R; k <= R; ++k) {
            const int64_t s = bmap(i + k, n, b);
            acc = fmaf(w.w[k + R], s < 0 ? 0.f : __ldg(in + s), acc);
        }
        out[i] = acc;
    }
}

constexpr int k1Per = 8, k1Tile = 256 * k1Per;

template <int R>
__global__ void __launch_bounds__(256)
st1_smem(const float *__restrict__ in, float *__restrict__ out, int64_t n, int b, W33 w)
{
    constexpr int WV = (k1Per + 2 * R + 3) / 4;        // 16-byte reads per window
    constexpr int SW = k1Tile + 4 * WV;                // window of the last thread stays in bounds
    __shared__ __align__(16) float s[SW];
    const int64_t t0 = (int64_t)blockIdx.x * k1Tile;
    if (t0 - R >= 0 && t0 + k1Tile + R <= n) {         // interior block: no boundary map
        for (int j = threadIdx.x; j < k1Tile + 2 * R; j += 256) s[j] = __ldg(in + t0 - R + j);
    } else {
        for (int j = threadIdx.x; j < k1Tile + 2 * R; j += 256) {
            const int64_t src = bmap(t0 - R + j, n, b);
            s[j] = src < 0 ? 0.f : __ldg(in + src);
        }
    }
    for (int j = k1Tile + 2 * R + threadIdx.x; j < SW; j += 256) s[j] = 0.f;
    __syncthreads();
    // thread t owns outputs 8t .. 8t+7; its window s[8t .. 8t+8+2R) is read as
    // 16-byte vectors (a 32-byte stride between threads: two-way bank sharing)
    const int base = threadIdx.x * k1Per;
    float win[4 * WV];
#pragma unroll
    for (int j = 0; j < WV; ++j) {
        const float4 q = *reinterpret_cast<const float4 *>(s + base + 4 * j);
        win[4 * j] = q.x; win[4 * j + 1] = q.y; win[4 * j + 2] = q.z; win[4 * j + 3] = q.w;
    }
    float o[k1Per];
#pragma unroll
    for (int q = 0; q < k1Per; ++q) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(w.w[k], win[q + k], acc);
        o[q] = acc;
    }
    const int64_t i0 = t0 + base;
    if (i0 + k1Per <= n && ((uintptr_t)(out + i0) & 15u) == 0) {
        dev::st_stream(reinterpret_cast<float4 *>(out + i0), make_float4(o[0], o[1], o[2], o[3]));
        dev::st_stream(reinterpret_cast<float4 *>(out + i0 + 4), make_float4(o[4], o[5], o[6], o[7]));
    } else {
#pragma unroll
        for (int q = 0; q < k1Per; ++q)
            if (i0 + q < n) out[i0 + q] = o[q];
    }
}

// 1D bulk-copy tile: 4096 outputs per block.  An interior block fetches its
// 4096 + 2*HP inputs (HP = R rounded up to a multiple of 4, so every piece
// stays 16-byte aligned) with one cp.async.bulk completing on an mbarrier;
// the first and last blocks gather through the boundary map instead.  Thread
// t computes the 4-output groups t, t + 256, t + 512, t + 768, reading each
// group's 4 + 2*HP window as 16-byte vectors (consecutive threads 16 bytes
// apart: no bank conflicts).
constexpr int kBT = 4096;

template <int R>
__global__ void __launch_bounds__(256)
st1_bulk(const float *__restrict__ in, float *__restrict__ out, int64_t n, int b, W33 w, Control *ctl)
{
    constexpr int HP = (R + 3) / 4 * 4;
    constexpr int NV = 1 + 2 * HP / 4;                 // 16-byte reads per group window
    __shared__ __align__(128) float s[kBT + 2 * HP];
    __shared__ __align__(8) uint64_t bar;
    const int64_t t0 = (int64_t)blockIdx.x * kBT;
    const bool interior = t0 - HP >= 0 && t0 + kBT + HP <= n;
    if (interior) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            constexpr uint32_t bytes = (kBT + 2 * HP) * 4;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(smem_addr(&bar)), "r"(bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_addr(s)), "l"(in + t0 - HP), "r"(bytes), "r"(smem_addr(&bar)) : "memory");
        }
        __syncthreads();                               // the barrier is initialised before anyone polls it
        uint32_t done = 0;
        for (uint32_t it = 0; it < (1u << 22) && !done; ++it) {
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done) : "r"(smem_addr(&bar)) : "memory");
        }
        if (!__syncthreads_and(done)) {
            if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
            return;
        }
    } else {
        for (int j = threadIdx.x; j < kBT + 2 * HP; j += 256) {
            const int64_t k = t0 - HP + j;
            const int64_t src = k < n + R ? bmap(k, n, b) : -1;
            s[j] = src < 0 ? 0.f : __ldg(in + src);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kBT / 1024; ++u) {
        const int g = threadIdx.x + 256 * u;
        const int64_t i0 = t0 + 4 * g;
        if (i0 >= n) break;
        float win[4 * NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float4 q = *reinterpret_cast<const float4 *>(s + 4 * g + 4 * v);
            win[4 * v] = q.x; win[4 * v + 1] = q.y; win[4 * v + 2] = q.z; win[4 * v + 3] = q.w;
        }
        float o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) acc = fmaf(w.w[k], win[q + HP - R + k], acc);
            o[q] = acc;
        }
        if (i0 + 4 <= n) {
            dev::st_stream(reinterpret_cast<float4 *>(out + i0), make_float4(o[0], o[1], o[2], o[3]));
        } else {
            for (int q = 0; q < 4 && i0 + q < n; ++q) out[i0 + q] = o[q];
        }
    }
}

// Exact CLAMP adjoint at the two ends of a 1D stencil (overwrites gin[0],
// gin[n-1]): sums w[k] g[i] over outputs i and taps k with clamp(i+k) == p.
__global__ void st1_fold_ends(const float *__restrict__ g, float *__restrict__ gin, int64_t n, int r, W33 w)
{
    const int which = threadIdx.x;   // 0: p = 0, 1: p = n-1
    if (which > 1 || (which == 1 && n == 1)) return;
    const int64_t p = which == 0 ? 0 : n - 1;
    const int64_t ilo = which == 0 ? 0 : (n - 1 - r > 0 ? n - 1 - r : 0);
    const int64_t ihi = which == 0 ? (r < n - 1 ? r : n - 1) : n - 1;
    float acc = 0.f;
    for (int64_t i = ilo; i <= ihi; ++i)
        for (int k = -r; k <= r; ++k)
            if (bmap(i + k, n, SKEL_CLAMP) == p) acc = fmaf(w.w[k + r], g[i], acc);
    gin[p] = acc;
}

// ---------------------------------------------------------------- host --
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

int check_launch(const char *what)
{
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), what);
}

template <bool TAPS5>
int run2d(const StencilLaunch &st, const Choice &c, const float *in, float *out, int b, const W9 &w, cudaStream_t s)
{
    const int64_t rows = st.rows, cols = st.cols;
    const bool vec_ok = cols % 4 == 0 && aligned16(in) && aligned16(out);
    if (c.variant != 0 && !vec_ok)
        return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 2D: tiled variants need cols % 4 == 0 and 16-byte aligned grids");
    if (c.variant == 0) {
        const int64_t gy = ceil_div(rows, 8);
        launch_kernel(st2_direct<TAPS5>, dim3((unsigned)ceil_div(cols, 32), (unsigned)(gy < 65535 ? gy : 65535)), 256, 0, s,
            in, out, rows, cols, b, w);
        return check_launch("mapoverlap2d direct");
    }
    if (ceil_div(rows, kTY) > 65535) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 2D: too many tile rows");
    const dim3 grid((unsigned)ceil_div(cols, kTX), (unsigned)ceil_div(rows, kTY));
    if (c.variant == 1) {
        launch_kernel(st2_smem<TAPS5>, grid, 256, 0, s, in, out, rows, cols, b, w);
        return check_launch("mapoverlap2d smem");
    }
    if (c.variant == 2) {
        EncodeTiled enc = encode_fn();
        if (!enc) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 2D: cuTensorMapEncodeTiled unavailable");
        if (rows > 0x7fffffff || cols > 0x7fffffff) return fail(SKEL_ERR_UNSUPPORTED, "TMA: grid too large");
        CUtensorMap map;
        const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
        const cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kSW, (cuuint32_t)kSH};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(in), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 2D: tensor map encoding failed");
        Scratch scr{};
        int rc = get_scratch(s, 0, 0, &scr);
        if (rc) return rc;
        const int smem = kSH * kSW * 4 + 16;   // tile + mbarrier
        launch_kernel(st2_tma<TAPS5>, grid, 256, smem, s, map, in, out, rows, cols, b, w, scr.ctl);
        return check_launch("mapoverlap2d tma");
    }
    if (c.variant == 3) {
        const int rh = c.tile > 0 ? c.tile : 32;
        const int64_t gy = ceil_div(rows, rh);
        if (gy > 65535) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 2D: too many row segments");
        const dim3 g2((unsigned)ceil_div(cols, 512), (unsigned)gy);
        switch (rh) {
        case 16: launch_kernel(st2_colwalk<TAPS5, 16>, g2, 128, 0, s, in, out, rows, cols, b, w); break;
        case 32: launch_kernel(st2_colwalk<TAPS5, 32>, g2, 128, 0, s, in, out, rows, cols, b, w); break;
        case 64: launch_kernel(st2_colwalk<TAPS5, 64>, g2, 128, 0, s, in, out, rows, cols, b, w); break;
        case 128: launch_kernel(st2_colwalk<TAPS5, 128>, g2, 128, 0, s, in, out, rows, cols, b, w); break;
        default: return fail(SKEL_ERR_INVALID_ARG, "column_walk: tile (rows per walk) must be 16, 32, 64 or 128");
        }
        return check_launch("mapoverlap2d column_walk");
    }
    return fail(SKEL_ERR_INVALID_ARG, "mapoverlap 2D: unknown variant");
}

template <int R>
int run1d_r(const Choice &c, const float *in, float *out, int64_t n, int b, const W33 &w, cudaStream_t s)
{
    if (c.variant == 0) {
        int64_t grid = ceil_div(n, 256);
        const int64_t cap = (int64_t)device_info().sms * 32;
        if (grid > cap) grid = cap;
        launch_kernel(st1_direct<R>, (unsigned)grid, 256, 0, s, in, out, n, b, w);
        return check_launch("mapoverlap1d direct");
    }
    if (c.variant == 1) {
        const int64_t grid = ceil_div(n, k1Tile);
        if (grid > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "mapoverlap1d: too long");
        launch_kernel(st1_smem<R>, (unsigned)grid, 256, 0, s, in, out, n, b, w);
        return check_launch("mapoverlap1d smem");
    }
    if (c.variant == 2) {
        if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u))
            return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 1D bulk: input and output must be 16-byte aligned");
        const int64_t grid = ceil_div(n, kBT);
        if (grid > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "mapoverlap1d: too long");
        Scratch scr{};
        int rc = get_scratch(s, 0, 0, &scr);
        if (rc) return rc;
        launch_kernel(st1_bulk<R>, (unsigned)grid, 256, 0, s, in, out, n, b, w, scr.ctl);
        return check_launch("mapoverlap1d bulk");
    }
    return fail(SKEL_ERR_INVALID_ARG, "mapoverlap 1D: unknown variant");
}

// ------------------------------------------- 2D chains, time-blocked --
// K steps of the same 2D stencil fused into one pass (temporal blocking): a
// block stages its 128 x 32 output tile with a halo of K rows and
// roundup4(K) + 4 columns, runs the K steps in shared memory (ping-pong
// between two buffers, the valid area shrinking by one cell per step) and
// writes only the tile.  HBM traffic drops K-fold against K separate calls.
//
// Boundaries: staged cells outside the grid hold what the single-step
// kernels read there: the clamped neighbour (CLAMP) or 0 (ZERO), re-derived
// after every step from that step's values (the clamped cell of a border
// tile always lies in its computed area).  PERIODIC would need cells of the
// far side of the grid and is not offered.  Each cell is evaluated by
// stencil9 with the taps in the single-step kernels' order, so K fused steps
// give bit-for-bit the result of K single calls.
template <int K>
struct ChainGeom {
    // column halo: K rounded up to 16 bytes, plus one group of 4 so that the
    // 4-column groups computed each step never read outside the staging
    static constexpr int HL = (K + 3) / 4 * 4 + 4;
    static constexpr int SW = kTX + 2 * HL;         // staged width
    static constexpr int SH = kTY + 2 * K;          // staged height
    static constexpr int NG = SW / 4 - 2;           // 4-column groups computed per row (34 or 36)
    static constexpr int SR = (SH - 2 + 6) / 7;     // rows per strip: at most 7 strips, so that
    static constexpr int NS = (SH - 2 + SR - 1) / SR;   // NG * NS <= 256 items, one per thread
    static_assert(NG * NS <= 256, "one item per thread");
    static constexpr int smem_bytes = 2 * SH * SW * 4;
};

template <bool TAPS5, int K>
__global__ void __launch_bounds__(256)
st2_chain(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t cols, int b, W9 w)
{
    using G = ChainGeom<K>;
    extern __shared__ __align__(16) float sm[];
    float *A = sm, *B = sm + G::SH * G::SW;
    const int64_t tx0 = (int64_t)blockIdx.x * kTX, ty0 = (int64_t)blockIdx.y * kTY;
    const int64_t gr0 = ty0 - K, gc0 = tx0 - G::HL;          // global position of staged (0, 0)
    const bool vec = (cols & 3) == 0;
    const int lane = threadIdx.x & 31;
    // stage: groups of 4 columns; a group is wholly inside or outside the
    // grid's columns when cols % 4 == 0 (then one 16-byte load)
    for (int g = threadIdx.x; g < G::SH * (G::SW / 4); g += 256) {
        const int sr = g / (G::SW / 4), sc = 4 * (g % (G::SW / 4));
        const int64_t r = bmap(gr0 + sr, rows, b), c = gc0 + sc;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r >= 0) {
            if (vec && c >= 0 && c + 3 < cols) {
                v = dev::ld_stream(reinterpret_cast<const float4 *>(in + r * cols + c));
            } else {
                float *vp = &v.x;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t cc = bmap(c + j, cols, b);
                    vp[j] = cc < 0 ? 0.f : __ldg(in + r * cols + cc);
                }
            }
        }
        *reinterpret_cast<float4 *>(A + sr * G::SW + sc) = v;
    }
    __syncthreads();
    const bool border = gr0 < 0 || gc0 < 0 || gr0 + G::SH > rows || gc0 + G::SW > cols;   // block-uniform
#pragma unroll 1
    for (int step = 0; step < K; ++step) {
        // B = stencil(A) on rows 1 .. SH-2 and columns 4 .. SW-5.  An item is
        // one group of 4 columns over a strip of SR rows, walked with a
        // 3-row register window: one 16-byte read per row, the outer
        // neighbours from the adjacent lanes (shared memory at warp edges);
        // four independent tap chains per row.
        for (int base = 0; base < G::NG * G::NS; base += 256) {   // block-uniform trip count
            const int item = base + threadIdx.x;
            const bool live = item < G::NG * G::NS;
            const int gcol = 4 * (1 + (live ? item % G::NG : 0));
            const int r0 = 1 + (live ? item / G::NG : 0) * G::SR;
            const int r1 = r0 + G::SR < G::SH - 1 ? r0 + G::SR : G::SH - 1;
            // lanes whose left / right group is another lane's: shuffles need
            // the same item row and adjacent groups
            const int nrow = live ? item / G::NG : -1;
            const int lrow = __shfl_up_sync(0xffffffffu, nrow, 1);
            const int rrow = __shfl_down_sync(0xffffffffu, nrow, 1);
            const bool lsh = lane > 0 && lrow == nrow && gcol > 4;
            const bool rsh = lane < 31 && rrow == nrow && gcol < 4 * G::NG;
            // a row of the window: columns gcol-1 .. gcol+4
            auto load_row = [&](int sr, float (&v)[6]) {
                const float *p = A + sr * G::SW + gcol;
                const float4 q = *reinterpret_cast<const float4 *>(p);
                const float l = __shfl_up_sync(0xffffffffu, q.w, 1);
                const float r = __shfl_down_sync(0xffffffffu, q.x, 1);
                v[0] = lsh ? l : p[-1];
                v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
                v[5] = rsh ? r : p[4];
            };
            // every lane runs SR rows (fully unrolled, so the window rotates
            // by renaming, and the shuffles see all lanes); rows past the
            // strip's end read a clamped row and are not stored
            const int rows_here = live ? r1 - r0 : 0;
            const int rr0 = live ? r0 : 1;
            float rows_buf[G::SR + 2][6];
            load_row(rr0 - 1, rows_buf[0]);
            load_row(rr0, rows_buf[1]);
#pragma unroll
            for (int k = 0; k < G::SR; ++k) {
                const int r = rr0 + k;
                load_row(r + 1 < G::SH ? r + 1 : G::SH - 1, rows_buf[k + 2]);
                float4 o;
                float *op = &o.x;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    op[j] = stencil9<TAPS5>(w, rows_buf[k][j], rows_buf[k][j + 1], rows_buf[k][j + 2],
                                            rows_buf[k + 1][j], rows_buf[k + 1][j + 1], rows_buf[k + 1][j + 2],
                                            rows_buf[k + 2][j], rows_buf[k + 2][j + 1], rows_buf[k + 2][j + 2]);
                if (k < rows_here) *reinterpret_cast<float4 *>(B + r * G::SW + gcol) = o;
            }
        }
        __syncthreads();
        if (border) {
            // cells outside the grid take this step's clamped neighbour, or 0
            constexpr int NC = G::SW - 8;
            for (int i = threadIdx.x; i < (G::SH - 2) * NC; i += 256) {
                const int sr = 1 + i / NC, sc = 4 + i % NC;
                const int64_t r = gr0 + sr, c = gc0 + sc;
                if (r >= 0 && r < rows && c >= 0 && c < cols) continue;
                float v = 0.f;
                if (b == SKEL_CLAMP) {
                    const int64_t rr = r < 0 ? 0 : (r >= rows ? rows - 1 : r);
                    const int64_t cc = c < 0 ? 0 : (c >= cols ? cols - 1 : c);
                    v = B[(rr - gr0) * G::SW + (cc - gc0)];
                }
                B[sr * G::SW + sc] = v;
            }
            __syncthreads();
        }
        float *t = A; A = B; B = t;
    }
    // the tile: staged rows K .. K+kTY-1, columns HL .. HL+kTX-1
    for (int g = threadIdx.x; g < kTY * (kTX / 4); g += 256) {
        const int tr = g / (kTX / 4), tc = 4 * (g % (kTX / 4));
        const int64_t r = ty0 + tr, c = tx0 + tc;
        if (r >= rows) continue;
        const float *src = A + (K + tr) * G::SW + G::HL + tc;
        if (vec && c + 3 < cols) {
            dev::st_stream(reinterpret_cast<float4 *>(out + r * cols + c), *reinterpret_cast<const float4 *>(src));
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c + j < cols) out[r * cols + c + j] = src[j];
        }
    }
}

template <bool TAPS5, int K>
int run_chain_k(const float *in, float *out, int64_t rows, int64_t cols, int b, const W9 &w, cudaStream_t s)
{
    auto kern = st2_chain<TAPS5, K>;
    constexpr int smem = ChainGeom<K>::smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return fail_cuda(e, "mapoverlap chain: shared memory opt-in");
    const int64_t gx = ceil_div(cols, kTX), gy = ceil_div(rows, kTY);
    if (gy > 65535 || gx > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "mapoverlap chain: grid too large");
    launch_kernel(kern, dim3((unsigned)gx, (unsigned)gy), 256, (size_t)smem, s, in, out, rows, cols, b, w);
    return check_launch("mapoverlap chain");
}

template <bool TAPS5>
int run_chain(int k, const float *in, float *out, int64_t rows, int64_t cols, int b, const W9 &w, cudaStream_t s)
{
    switch (k) {
    case 1: return run_chain_k<TAPS5, 1>(in, out, rows, cols, b, w, s);
    case 2: return run_chain_k<TAPS5, 2>(in, out, rows, cols, b, w, s);
    case 3: return run_chain_k<TAPS5, 3>(in, out, rows, cols, b, w, s);
    case 4: return run_chain_k<TAPS5, 4>(in, out, rows, cols, b, w, s);
    case 5: return run_chain_k<TAPS5, 5>(in, out, rows, cols, b, w, s);
    case 6: return run_chain_k<TAPS5, 6>(in, out, rows, cols, b, w, s);
    case 7: return run_chain_k<TAPS5, 7>(in, out, rows, cols, b, w, s);
    case 8: return run_chain_k<TAPS5, 8>(in, out, rows, cols, b, w, s);
    default: return fail(SKEL_ERR_INVALID_ARG, "mapoverlap chain: steps per pass must be 1..8");
    }
}

int run1d(const Choice &c, int r, const float *in, float *out, int64_t n, int b, const W33 &w, cudaStream_t s)
{
    switch (r) {
#define SKEL_R(k) case k: return run1d_r<k>(c, in, out, n, b, w, s);
    SKEL_R(0) SKEL_R(1) SKEL_R(2) SKEL_R(3) SKEL_R(4) SKEL_R(5) SKEL_R(6) SKEL_R(7) SKEL_R(8)
    SKEL_R(9) SKEL_R(10) SKEL_R(11) SKEL_R(12) SKEL_R(13) SKEL_R(14) SKEL_R(15) SKEL_R(16)
#undef SKEL_R
    default: return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap 1D: radius must be 0..16");
    }
}

}  // namespace

int stencil_variant_count(int ndim) { return ndim == 1 ? 3 : 4; }
const char *stencil_variant_name(int ndim, int v)
{
    static const char *n1[] = {"direct", "smem_tile", "bulk_tile"};
    static const char *n2[] = {"direct", "smem_tile", "tma_tile", "column_walk"};
    if (ndim == 1) return v >= 0 && v < 3 ? n1[v] : "?";
    return v >= 0 && v < 4 ? n2[v] : "?";
}
Choice stencil_default(int ndim) { return ndim == 1 ? Choice{1, 256, 8, 0} : Choice{1, 256, 0, 0}; }

int launch_stencil(const StencilLaunch &st, const Choice &c, cudaStream_t s)
{
    const int64_t n = st.rows * st.cols;
    if (n == 0) return SKEL_OK;
    // adjoint: mirrored weights; CLAMP runs as ZERO plus the border fix-up
    const int b = (st.transpose && st.boundary == SKEL_CLAMP) ? SKEL_ZERO : st.boundary;
    if (st.ndim == 2) {
        W9 w, wf;
        for (int k = 0; k < 9; ++k) w.w[k] = st.w[k];
        for (int k = 0; k < 9; ++k) wf.w[k] = st.transpose ? st.w[8 - k] : st.w[k];
        if (st.taps5) { wf.w[0] = wf.w[2] = wf.w[6] = wf.w[8] = 0.f; w.w[0] = w.w[2] = w.w[6] = w.w[8] = 0.f; }
        int rc = st.taps5 ? run2d<true>(st, c, st.in, st.out, b, wf, s) : run2d<false>(st, c, st.in, st.out, b, wf, s);
        if (rc || !st.transpose || st.boundary != SKEL_CLAMP) return rc;
        const int64_t nb = st.rows * st.cols;   // upper bound of border cells
        int64_t grid = ceil_div(nb < 4 * (st.rows + st.cols) ? nb : 4 * (st.rows + st.cols), 256);
        if (grid > 4096) grid = 4096;
        if (st.taps5) launch_kernel(st2_fold_border<true>, (unsigned)grid, 256, 0, s, st.in, st.out, st.rows, st.cols, w);
        else launch_kernel(st2_fold_border<false>, (unsigned)grid, 256, 0, s, st.in, st.out, st.rows, st.cols, w);
        return check_launch("mapoverlap2d adjoint border");
    }
    W33 w{}, wf{};
    const int r = st.radius;
    for (int k = 0; k <= 2 * r; ++k) {
        w.w[k] = st.w[k];
        wf.w[k] = st.transpose ? st.w[2 * r - k] : st.w[k];
    }
    int rc = run1d(c, r, st.in, st.out, st.cols, b, wf, s);
    if (rc || !st.transpose || st.boundary != SKEL_CLAMP || r == 0) return rc;
    launch_kernel(st1_fold_ends, 1, 32, 0, s, st.in, st.out, st.cols, r, w);
    return check_launch("mapoverlap1d adjoint ends");
}

int chain_variant_count() { return 2; }
const char *chain_variant_name(int v)
{
    static const char *names[] = {"per_call", "time_blocked"};
    return v >= 0 && v < 2 ? names[v] : "?";
}
Choice chain_default() { return Choice{1, 256, 0, 4}; }

int launch_stencil_chain_fused(const StencilLaunch &st, int steps, float *tmp, const Choice &c, cudaStream_t s)
{
    if (st.ndim != 2 || st.transpose) return fail(SKEL_ERR_INVALID_ARG, "mapoverlap chain: 2D forward stencils only");
    if (st.boundary == SKEL_PERIODIC) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap chain: periodic is not time-blocked");
    const int k = c.tile > 0 ? c.tile : 4;
    if (k < 1 || k > 8) return fail(SKEL_ERR_INVALID_ARG, "mapoverlap chain: tile (steps per pass) must be 1..8");
    const int passes = (steps + k - 1) / k;
    if (passes > 1 && !tmp) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap chain: several passes need tmp");
    W9 w;
    for (int q = 0; q < 9; ++q) w.w[q] = st.w[q];
    if (st.taps5) w.w[0] = w.w[2] = w.w[6] = w.w[8] = 0.f;
    const float *src = st.in;
    for (int p = 0; p < passes; ++p) {
        const int kp = p < passes - 1 ? k : steps - k * (passes - 1);
        float *dst = ((passes - 1 - p) % 2 == 0) ? st.out : tmp;   // the last pass writes out
        int rc = st.taps5 ? run_chain<true>(kp, src, dst, st.rows, st.cols, st.boundary, w, s)
                          : run_chain<false>(kp, src, dst, st.rows, st.cols, st.boundary, w, s);
        if (rc) return rc;
        src = dst;
    }
    return SKEL_OK;
}

}  // namespace skel
