// Map skeleton (Sec. III, map as a higher-order function): out[i] = f(x[i], y[i]; a).
//
// Variants (all HBM-streaming; the work per element is one or two flops):
//   0 scalar      grid-stride loop, one float per thread per step; any alignment.
//   1 vec4        one-shot grid, each thread owns `ept` float4 groups (all loads
//                 issued before the first use), 128-bit coalesced accesses.
//   2 vec4_hint   vec4 with L1::no_allocate loads and evict-first (.cs) stores.
//   3 vec4_grid   persistent grid (a multiple of the SM count), grid-stride over
//                 float4 groups, `ept` groups in flight per thread.
// Variants 1-3 need every operand at the same address offset modulo 16 bytes;
// the few elements before the first 16-byte boundary and after the last full
// float4 are handled by scalar threads of the same launch.
//
// In-place calls (out is one of the inputs, m.alias) run each variant's
// access pattern in kernels without __restrict__ and with plain coherent
// loads and stores: the read-only (non-coherent) load path and restrict
// qualifiers both promise that no memory the kernel reads is written during
// the kernel, which an in-place map breaks.
#include "common.cuh"

namespace skel {
namespace {

using dev::MapF;

template <int FN, bool HINT>
__device__ __forceinline__ float4 load4(const float4 *p)
{
    if (HINT) return dev::ld_stream(p);
    return __ldg(p);
}

template <int FN>
__global__ void map_scalar(const float *__restrict__ x, const float *__restrict__ y,
                           float *__restrict__ out, int64_t n, float a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float yv = MapF<FN>::nin == 2 ? y[i] : 0.f;
        out[i] = MapF<FN>::f(x[i], yv, a);
    }
}

// Scalar head/tail elements handled by the first (head + tail) threads.
template <int FN>
__device__ __forceinline__ void map_edges(const float *x, const float *y, float *out, int head,
                                          int64_t nvec, int tail, float a, int64_t gtid)
{
    if (gtid < head + tail) {
        int64_t i = gtid < head ? gtid : head + 4 * nvec + (gtid - head);
        float yv = MapF<FN>::nin == 2 ? y[i] : 0.f;
        out[i] = MapF<FN>::f(x[i], yv, a);
    }
}

template <int FN, int EPT, bool HINT>
__global__ void map_vec(const float *__restrict__ x, const float *__restrict__ y,
                        float *__restrict__ out, int head, int64_t nvec, int tail, float a)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    map_edges<FN>(x, y, out, head, nvec, tail, a, gtid);
    const float4 *x4 = reinterpret_cast<const float4 *>(x + head);
    const float4 *y4 = reinterpret_cast<const float4 *>(y + head);
    float4 *o4 = reinterpret_cast<float4 *>(out + head);
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * EPT + threadIdx.x;
    float4 vx[EPT], vy[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        int64_t i = base + (int64_t)k * blockDim.x;
        if (i < nvec) {
            vx[k] = load4<FN, HINT>(x4 + i);
            if (MapF<FN>::nin == 2) vy[k] = load4<FN, HINT>(y4 + i);
        }
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        int64_t i = base + (int64_t)k * blockDim.x;
        if (i < nvec) {
            float4 q = vx[k], r = MapF<FN>::nin == 2 ? vy[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 o = make_float4(MapF<FN>::f(q.x, r.x, a), MapF<FN>::f(q.y, r.y, a),
                                   MapF<FN>::f(q.z, r.z, a), MapF<FN>::f(q.w, r.w, a));
            if (HINT) dev::st_stream(o4 + i, o); else o4[i] = o;
        }
    }
}

template <int FN, int EPT>
__global__ void map_vec_grid(const float *__restrict__ x, const float *__restrict__ y,
                             float *__restrict__ out, int head, int64_t nvec, int tail, float a)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    map_edges<FN>(x, y, out, head, nvec, tail, a, gtid);
    const float4 *x4 = reinterpret_cast<const float4 *>(x + head);
    const float4 *y4 = reinterpret_cast<const float4 *>(y + head);
    float4 *o4 = reinterpret_cast<float4 *>(out + head);
    const int64_t step = (int64_t)gridDim.x * blockDim.x * EPT;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * EPT + threadIdx.x; base < nvec;
         base += step) {
        float4 vx[EPT], vy[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            int64_t i = base + (int64_t)k * blockDim.x;
            if (i < nvec) {
                vx[k] = dev::ld_stream(x4 + i);
                if (MapF<FN>::nin == 2) vy[k] = dev::ld_stream(y4 + i);
            }
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            int64_t i = base + (int64_t)k * blockDim.x;
            if (i < nvec) {
                float4 q = vx[k], r = MapF<FN>::nin == 2 ? vy[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                dev::st_stream(o4 + i, make_float4(MapF<FN>::f(q.x, r.x, a), MapF<FN>::f(q.y, r.y, a),
                                                   MapF<FN>::f(q.z, r.z, a), MapF<FN>::f(q.w, r.w, a)));
            }
        }
    }
}

// In-place forms (no __restrict__, coherent loads).  Every element is read
// and then written by the same thread, so the result equals the out-of-place
// one element for element.
template <int FN>
__global__ void map_scalar_inplace(const float *x, const float *y, float *out, int64_t n, float a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float yv = MapF<FN>::nin == 2 ? y[i] : 0.f;
        out[i] = MapF<FN>::f(x[i], yv, a);
    }
}

template <int FN, int EPT>
__global__ void map_vec_inplace(const float *x, const float *y, float *out, int head, int64_t nvec, int tail,
                                float a)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    map_edges<FN>(x, y, out, head, nvec, tail, a, gtid);
    const float4 *x4 = reinterpret_cast<const float4 *>(x + head);
    const float4 *y4 = reinterpret_cast<const float4 *>(y + head);
    float4 *o4 = reinterpret_cast<float4 *>(out + head);
    const int64_t step = (int64_t)gridDim.x * blockDim.x * EPT;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * EPT + threadIdx.x; base < nvec; base += step) {
        float4 vx[EPT], vy[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            int64_t i = base + (int64_t)k * blockDim.x;
            if (i < nvec) {
                vx[k] = x4[i];
                if (MapF<FN>::nin == 2) vy[k] = y4[i];
            }
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            int64_t i = base + (int64_t)k * blockDim.x;
            if (i < nvec) {
                float4 q = vx[k], r = MapF<FN>::nin == 2 ? vy[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                o4[i] = make_float4(MapF<FN>::f(q.x, r.x, a), MapF<FN>::f(q.y, r.y, a), MapF<FN>::f(q.z, r.z, a),
                                    MapF<FN>::f(q.w, r.w, a));
            }
        }
    }
}

template <int FN>
int run_map(const MapLaunch &m, const Choice &c, cudaStream_t s)
{
    const int block = c.block > 0 ? c.block : 256;
    if (block % 32 || block > 1024) return fail(SKEL_ERR_INVALID_ARG, "map: block must be a multiple of 32, <= 1024");
    const float a = m.a;
    if (c.variant == 0) {
        int64_t grid = ceil_div(m.n, block);
        const int64_t cap = (int64_t)device_info().sms * (2048 / block) * 4;
        if (grid > cap) grid = cap;
        if (grid < 1) grid = 1;
        if (m.alias) launch_kernel(map_scalar_inplace<FN>, (unsigned)grid, block, 0, s, m.in0, m.in1, m.out, m.n, a);
        else launch_kernel(map_scalar<FN>, (unsigned)grid, block, 0, s, m.in0, m.in1, m.out, m.n, a);
        return cudaPeekAtLastError() == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "map_scalar");
    }
    // vectorised variants: same offset modulo 16 bytes for every operand
    const uintptr_t mis = (uintptr_t)m.out & 15u;
    if (((uintptr_t)m.in0 & 15u) != mis || (MapF<FN>::nin == 2 && ((uintptr_t)m.in1 & 15u) != mis) || (mis & 3u))
        return fail(SKEL_ERR_UNSUPPORTED, "map: vector variants need operands at equal offsets modulo 16 bytes");
    int64_t head = mis ? (int64_t)((16u - mis) / 4u) : 0;
    if (head > m.n) head = m.n;
    const int64_t nvec = (m.n - head) / 4;
    const int tail = (int)(m.n - head - 4 * nvec);
    const int ept = c.ept > 0 ? c.ept : 1;
    int64_t grid;
    if (c.variant == 3) {
        grid = (int64_t)device_info().sms * (2048 / block);
        int64_t need = ceil_div(nvec, (int64_t)block * ept);
        if (grid > need) grid = need;
    } else {
        grid = ceil_div(nvec, (int64_t)block * ept);
    }
    if (grid * block < head + tail) grid = ceil_div(head + tail, block);
    if (grid < 1) grid = 1;
    if (grid > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "map: grid too large");
    const unsigned g = (unsigned)grid;
#define SKEL_MAP_EPT(E)                                                                          \
    do {                                                                                         \
        if (m.alias) launch_kernel(map_vec_inplace<FN, E>, g, block, 0, s, m.in0, m.in1, m.out, (int)head, nvec, tail, a); \
        else if (c.variant == 1) launch_kernel(map_vec<FN, E, false>, g, block, 0, s, m.in0, m.in1, m.out, (int)head, nvec, tail, a); \
        else if (c.variant == 2) launch_kernel(map_vec<FN, E, true>, g, block, 0, s, m.in0, m.in1, m.out, (int)head, nvec, tail, a); \
        else launch_kernel(map_vec_grid<FN, E>, g, block, 0, s, m.in0, m.in1, m.out, (int)head, nvec, tail, a); \
    } while (0)
    switch (ept) {
    case 1: SKEL_MAP_EPT(1); break;
    case 2: SKEL_MAP_EPT(2); break;
    case 4: SKEL_MAP_EPT(4); break;
    default: return fail(SKEL_ERR_INVALID_ARG, "map: ept must be 1, 2 or 4");
    }
#undef SKEL_MAP_EPT
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "map_vec launch");
}

}  // namespace

int map_variant_count() { return 4; }
const char *map_variant_name(int v)
{
    static const char *names[] = {"scalar", "vec4", "vec4_hint", "vec4_grid"};
    return v >= 0 && v < 4 ? names[v] : "?";
}
Choice map_default() { return Choice{1, 256, 1, 0}; }

int launch_map(const MapLaunch &m, const Choice &c, cudaStream_t s)
{
    if (m.n == 0) return SKEL_OK;
    if (c.variant < 0 || c.variant > 3) return fail(SKEL_ERR_INVALID_ARG, "map: unknown variant");
    switch (m.fn) {
    case SKEL_FN_ADD: return run_map<SKEL_FN_ADD>(m, c, s);
    case SKEL_FN_SUB: return run_map<SKEL_FN_SUB>(m, c, s);
    case SKEL_FN_MUL: return run_map<SKEL_FN_MUL>(m, c, s);
    case SKEL_FN_MAX: return run_map<SKEL_FN_MAX>(m, c, s);
    case SKEL_FN_AXPY: return run_map<SKEL_FN_AXPY>(m, c, s);
    case SKEL_FN_TANH: return run_map<SKEL_FN_TANH>(m, c, s);
    case SKEL_FN_SQ: return run_map<SKEL_FN_SQ>(m, c, s);
    case SKEL_FN_SCALE: return run_map<SKEL_FN_SCALE>(m, c, s);
    case SKEL_FN_COPY: return run_map<SKEL_FN_COPY>(m, c, s);
    default: return fail(SKEL_ERR_UNSUPPORTED, "map: function not offered");
    }
}

}  // namespace skel
