// MapArray skeleton: out[i] = f(A, B[i]) with A read whole (random access)
// and B per element.  The paper names no MapArray; the reading implemented:
//   GATHER  out[i] = A[clamp(idx[i], 0, m-1)]          (idx int32)
//   ROWDOT  out[i] = sum_k A[k] * M[i, k]               (M row-major n x m)
// Variants (gather / rowdot):
//   0 scalar      gather: one output per thread; rowdot: one row per thread
//                 (no constraints; the baseline).
//   1 vec4        gather: 16-byte index loads and output stores, four outputs
//                 per thread; rowdot: one warp per row, 16-byte coalesced
//                 row loads, warp-shuffle sum.
//   2 block_row   rowdot: one block per row, block-tree sum (long rows);
//     vec4_multi  gather: vec4 with ept groups of four per thread per step
//                 (8, 16 or 32 random reads of A in flight per thread).
//   3 split_row   rowdot only: each row split over several blocks (partials
//                 in scratch, then a fixed-order combine): few, long rows.
// A is read through the read-only path; it stays in L1/L2 across rows.
#include "common.cuh"

namespace skel {
namespace {

__device__ __forceinline__ int64_t clampi(int64_t k, int64_t m) { return k < 0 ? 0 : (k >= m ? m - 1 : k); }

__global__ void gather_scalar(const float *__restrict__ A, int64_t m, const int32_t *__restrict__ idx,
                              float *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __ldg(A + clampi(idx[i], m));
}

__global__ void gather_vec4(const float *__restrict__ A, int64_t m, const int32_t *__restrict__ idx,
                            float *__restrict__ out, int64_t n)
{
    const int64_t nv = n / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 k = dev::ld_stream(reinterpret_cast<const uint4 *>(idx) + i);
        float4 o;
        o.x = __ldg(A + clampi((int32_t)k.x, m));
        o.y = __ldg(A + clampi((int32_t)k.y, m));
        o.z = __ldg(A + clampi((int32_t)k.z, m));
        o.w = __ldg(A + clampi((int32_t)k.w, m));
        dev::st_stream(reinterpret_cast<float4 *>(out) + i, o);
    }
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n - 4 * nv) out[4 * nv + t] = __ldg(A + clampi(idx[4 * nv + t], m));
}

// G groups of four indices per thread per step: 4G random reads of A in
// flight per thread (vec4 keeps four), the index loads and output stores
// still 16 bytes and coalesced (group g of a step lies one grid stride after
// group g - 1).
template <int G>
__global__ void gather_vec4_multi(const float *__restrict__ A, int64_t m, const int32_t *__restrict__ idx,
                                  float *__restrict__ out, int64_t n)
{
    const int64_t nv = n / 4;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const uint4 *idx4 = reinterpret_cast<const uint4 *>(idx);
    float4 *out4 = reinterpret_cast<float4 *>(out);
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nv; i0 += T * G) {
        uint4 k[G];
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (i0 + g * T < nv) k[g] = dev::ld_stream(idx4 + i0 + g * T);
        float4 o[G];
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (i0 + g * T < nv) {
                o[g].x = __ldg(A + clampi((int32_t)k[g].x, m));
                o[g].y = __ldg(A + clampi((int32_t)k[g].y, m));
                o[g].z = __ldg(A + clampi((int32_t)k[g].z, m));
                o[g].w = __ldg(A + clampi((int32_t)k[g].w, m));
            }
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (i0 + g * T < nv) dev::st_stream(out4 + i0 + g * T, o[g]);
    }
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n - 4 * nv) out[4 * nv + t] = __ldg(A + clampi(idx[4 * nv + t], m));
}

__global__ void rowdot_thread(const float *__restrict__ A, int64_t m, const float *__restrict__ M,
                              float *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *row = M + i * m;
        float acc = 0.f;
        for (int64_t k = 0; k < m; ++k) acc = fmaf(__ldg(A + k), row[k], acc);
        out[i] = acc;
    }
}

// One warp per row; VEC: row start and A 16-byte aligned, m % 4 == 0.
template <bool VEC>
__global__ void __launch_bounds__(256)
rowdot_warp(const float *__restrict__ A, int64_t m, const float *__restrict__ M, float *__restrict__ out, int64_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * 8;
    for (int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += warps) {
        const float *row = M + i * m;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (VEC) {
            const float4 *r4 = reinterpret_cast<const float4 *>(row);
            const float4 *A4 = reinterpret_cast<const float4 *>(A);
            const int64_t mv = m / 4;
            int64_t k = lane;
            for (; k + 96 < mv; k += 128) {   // four 16-byte row loads in flight per lane
                float4 p[4], ap[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) p[u] = dev::ld_stream(r4 + k + 32 * u);
#pragma unroll
                for (int u = 0; u < 4; ++u) ap[u] = __ldg(A4 + k + 32 * u);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a0 = fmaf(ap[u].x, p[u].x, a0); a1 = fmaf(ap[u].y, p[u].y, a1);
                    a2 = fmaf(ap[u].z, p[u].z, a2); a3 = fmaf(ap[u].w, p[u].w, a3);
                }
            }
            for (; k < mv; k += 32) {
                const float4 p = dev::ld_stream(r4 + k);
                const float4 ap = __ldg(A4 + k);
                a0 = fmaf(ap.x, p.x, a0); a1 = fmaf(ap.y, p.y, a1); a2 = fmaf(ap.z, p.z, a2); a3 = fmaf(ap.w, p.w, a3);
            }
        } else {
            for (int64_t k = lane; k < m; k += 32) a0 = fmaf(__ldg(A + k), row[k], a0);
        }
        float acc = (a0 + a1) + (a2 + a3);
        acc = dev::warp_reduce<dev::AddF>(acc);
        if (lane == 0) out[i] = acc;
    }
}

// One block per row (grid-stride over rows); VEC as above.
template <bool VEC>
__global__ void __launch_bounds__(256)
rowdot_block(const float *__restrict__ A, int64_t m, const float *__restrict__ M, float *__restrict__ out, int64_t n)
{
    __shared__ float smem[32];
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const float *row = M + i * m;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (VEC) {
            const float4 *r4 = reinterpret_cast<const float4 *>(row);
            const float4 *A4 = reinterpret_cast<const float4 *>(A);
            for (int64_t k = threadIdx.x; k < m / 4; k += 256) {
                const float4 p = dev::ld_stream(r4 + k);
                const float4 ap = __ldg(A4 + k);
                a0 = fmaf(ap.x, p.x, a0); a1 = fmaf(ap.y, p.y, a1); a2 = fmaf(ap.z, p.z, a2); a3 = fmaf(ap.w, p.w, a3);
            }
        } else {
            for (int64_t k = threadIdx.x; k < m; k += 256) a0 = fmaf(__ldg(A + k), row[k], a0);
        }
        const float acc = dev::block_reduce<dev::AddF, float, 256>((a0 + a1) + (a2 + a3), smem);
        if (threadIdx.x == 0) out[i] = acc;
    }
}

// Split rows: block (s, i) sums the chunk [s*chunk, (s+1)*chunk) of row i
// into part[i*S + s]; rowdot_combine then adds a row's S partials in a fixed
// order (lane-strided, then the warp tree), so the result is deterministic.
// For few long rows, where one warp or block per row leaves the GPU idle.
template <bool VEC>
__global__ void __launch_bounds__(256)
rowdot_split(const float *__restrict__ A, int64_t m, const float *__restrict__ M, float *__restrict__ part,
             int64_t chunk)
{
    __shared__ float smem[32];
    const int64_t i = blockIdx.y, S = gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    const int64_t c1 = c0 + chunk < m ? c0 + chunk : m;
    const float *row = M + i * m;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (VEC) {   // chunk % 4 == 0 and m % 4 == 0: whole 16-byte groups
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
        const float4 *A4 = reinterpret_cast<const float4 *>(A);
        int64_t k = c0 / 4 + threadIdx.x;
        const int64_t kend = c1 / 4;
        for (; k + 768 < kend; k += 1024) {   // four 16-byte row loads in flight per thread
            float4 p[4], ap[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] = dev::ld_stream(r4 + k + 256 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) ap[u] = __ldg(A4 + k + 256 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a0 = fmaf(ap[u].x, p[u].x, a0); a1 = fmaf(ap[u].y, p[u].y, a1);
                a2 = fmaf(ap[u].z, p[u].z, a2); a3 = fmaf(ap[u].w, p[u].w, a3);
            }
        }
        for (; k < kend; k += 256) {
            const float4 p = dev::ld_stream(r4 + k);
            const float4 ap = __ldg(A4 + k);
            a0 = fmaf(ap.x, p.x, a0); a1 = fmaf(ap.y, p.y, a1); a2 = fmaf(ap.z, p.z, a2); a3 = fmaf(ap.w, p.w, a3);
        }
    } else {
        for (int64_t k = c0 + threadIdx.x; k < c1; k += 256) a0 = fmaf(__ldg(A + k), row[k], a0);
    }
    const float acc = dev::block_reduce<dev::AddF, float, 256>((a0 + a1) + (a2 + a3), smem);
    if (threadIdx.x == 0) part[i * S + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256)
rowdot_combine(const float *__restrict__ part, int64_t S, float *__restrict__ out, int64_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    float acc = 0.f;
    for (int64_t k = lane; k < S; k += 32) acc += part[i * S + k];
    acc = dev::warp_reduce<dev::AddF>(acc);
    if (lane == 0) out[i] = acc;
}

int check_launch(const char *what)
{
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), what);
}

unsigned grid_for(int64_t work, int block)
{
    int64_t g = ceil_div(work, block);
    const int64_t cap = (int64_t)device_info().sms * (2048 / block) * 8;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int maparray_variant_count() { return 4; }
const char *maparray_variant_name(int v)
{
    static const char *names[] = {"scalar", "vec4", "block_row / vec4_multi", "split_row"};
    return v >= 0 && v < 4 ? names[v] : "?";
}
Choice maparray_default() { return Choice{1, 256, 0, 0}; }

int launch_maparray(const MapArrayLaunch &ma, const Choice &c, cudaStream_t s)
{
    if (ma.n == 0) return SKEL_OK;
    const int block = 256;
    if (c.block > 0 && c.block != block) return fail(SKEL_ERR_INVALID_ARG, "maparray: block must be 256");
    if (ma.fn == SKEL_FN_GATHER) {
        const int32_t *idx = static_cast<const int32_t *>(ma.B);
        if (c.variant == 0) {
            launch_kernel(gather_scalar, grid_for(ma.n, block), block, 0, s, ma.A, ma.m, idx, ma.out, ma.n);
            return check_launch("gather scalar");
        }
        if (c.variant == 1) {
            if (!aligned16(idx) || !aligned16(ma.out))
                return fail(SKEL_ERR_UNSUPPORTED, "gather vec4: 16-byte aligned operands needed");
            launch_kernel(gather_vec4, grid_for(ceil_div(ma.n, 4), block), block, 0, s, ma.A, ma.m, idx, ma.out, ma.n);
            return check_launch("gather vec4");
        }
        if (c.variant == 2) {
            if (!aligned16(idx) || !aligned16(ma.out))
                return fail(SKEL_ERR_UNSUPPORTED, "gather vec4 multi: 16-byte aligned operands needed");
            const int G = c.ept > 0 ? c.ept : 2;
            const unsigned g = grid_for(ceil_div(ceil_div(ma.n, 4), G), block);
            switch (G) {
            case 2: launch_kernel(gather_vec4_multi<2>, g, block, 0, s, ma.A, ma.m, idx, ma.out, ma.n); break;
            case 4: launch_kernel(gather_vec4_multi<4>, g, block, 0, s, ma.A, ma.m, idx, ma.out, ma.n); break;
            case 8: launch_kernel(gather_vec4_multi<8>, g, block, 0, s, ma.A, ma.m, idx, ma.out, ma.n); break;
            default: return fail(SKEL_ERR_INVALID_ARG, "gather vec4 multi: ept (groups per thread) must be 2, 4 or 8");
            }
            return check_launch("gather vec4 multi");
        }
        return fail(SKEL_ERR_UNSUPPORTED, "gather: variant not offered");
    }
    if (ma.fn == SKEL_FN_ROWDOT) {
        const float *M = static_cast<const float *>(ma.B);
        const bool vec = aligned16(M) && aligned16(ma.A) && ma.m % 4 == 0;
        if (c.variant == 0) {
            launch_kernel(rowdot_thread, grid_for(ma.n, block), block, 0, s, ma.A, ma.m, M, ma.out, ma.n);
            return check_launch("rowdot thread");
        }
        if (c.variant == 1) {
            const unsigned g = grid_for(ceil_div(ma.n, 8) * 256, block);
            if (vec) launch_kernel(rowdot_warp<true>, g, block, 0, s, ma.A, ma.m, M, ma.out, ma.n);
            else launch_kernel(rowdot_warp<false>, g, block, 0, s, ma.A, ma.m, M, ma.out, ma.n);
            return check_launch("rowdot warp");
        }
        if (c.variant == 2) {
            int64_t g = ma.n;
            const int64_t cap = (int64_t)device_info().sms * 8 * 16;
            if (g > cap) g = cap;
            if (vec) launch_kernel(rowdot_block<true>, (unsigned)g, block, 0, s, ma.A, ma.m, M, ma.out, ma.n);
            else launch_kernel(rowdot_block<false>, (unsigned)g, block, 0, s, ma.A, ma.m, M, ma.out, ma.n);
            return check_launch("rowdot block");
        }
        if (c.variant == 3) {
            // chunks of at least 8192 elements, about 8 blocks per SM in total
            if (ma.n > 65535) return fail(SKEL_ERR_UNSUPPORTED, "rowdot split: at most 65535 rows");
            const int64_t target = (int64_t)device_info().sms * 8;
            int64_t S = ceil_div(target, ma.n);
            const int64_t smax = ceil_div(ma.m, 8192);
            if (S > smax) S = smax;
            if (S < 1) S = 1;
            const int64_t chunk = ma.m > 0 ? ceil_div(ceil_div(ma.m, S), 1024) * 1024 : 1024;
            S = ma.m > 0 ? ceil_div(ma.m, chunk) : 1;   // empty rows: one block writes 0
            Scratch scr{};
            int rc = get_scratch(s, (size_t)(ma.n * S) * sizeof(float), 0, &scr);
            if (rc) return rc;
            float *part = reinterpret_cast<float *>(scr.data);
            const dim3 g((unsigned)S, (unsigned)ma.n);
            if (vec) launch_kernel(rowdot_split<true>, g, block, 0, s, ma.A, ma.m, M, part, chunk);
            else launch_kernel(rowdot_split<false>, g, block, 0, s, ma.A, ma.m, M, part, chunk);
            rc = check_launch("rowdot split");
            if (rc) return rc;
            launch_kernel(rowdot_combine, (unsigned)ceil_div(ma.n, 8), block, 0, s, part, S, ma.out, ma.n);
            return check_launch("rowdot combine");
        }
        return fail(SKEL_ERR_INVALID_ARG, "rowdot: unknown variant");
    }
    return fail(SKEL_ERR_UNSUPPORTED, "maparray: fn must be GATHER or ROWDOT");
}

}  // namespace skel
