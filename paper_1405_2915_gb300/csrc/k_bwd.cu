// Elementwise adjoints: the backward pass of Map (an elementwise map again),
// of MapReduce (the upstream scalar times the map's derivative) and of
// Reduce with (+) (a broadcast of the upstream scalar).
//   gin0[i] = g_i * df/dx(x_i, y_i),  gin1[i] = g_i * df/dy(x_i, y_i)
// where g_i is the per-element upstream gradient (or the sum of two, when
// the map's output fed two calls) or one upstream scalar (a device word or a
// host value).  16-byte accesses when every operand is
// 16-byte aligned, scalar otherwise.
#include "common.cuh"

namespace skel {
namespace {

struct BwdArgs {
    float a;
    int tanh_from_output;
    const float *x;
    const float *y;
    const float *g;        // per element, or NULL
    const float *g2;       // a second per-element gradient added to g, or NULL
    const float *gs_dev;   // scalar on the device, or NULL
    float gs_host;
    float *gx;
    float *gy;
    int64_t n;
};

template <int FN>
__device__ __forceinline__ void dfun(float x, float y, float a, int from_out, float &dx, float &dy)
{
    if constexpr (FN == SKEL_FN_AXPY) { dx = a; dy = 1.f; }
    else if constexpr (FN == SKEL_FN_ADD) { dx = 1.f; dy = 1.f; }
    else if constexpr (FN == SKEL_FN_SUB) { dx = 1.f; dy = -1.f; }
    else if constexpr (FN == SKEL_FN_MUL) { dx = y; dy = x; }
    else if constexpr (FN == SKEL_FN_TANH) { const float t = from_out ? x : tanhf(x); dx = fmaf(-t, t, 1.f); dy = 0.f; }
    else if constexpr (FN == SKEL_FN_SQ) { dx = 2.f * x; dy = 0.f; }
    else if constexpr (FN == SKEL_FN_SCALE) { dx = a; dy = 0.f; }
    else { dx = 1.f; dy = 0.f; }   // COPY (and the broadcast of reduce's adjoint)
}

template <int FN>
__device__ __forceinline__ void one(const BwdArgs &p, int64_t i, float gsc)
{
    float g = p.g ? p.g[i] : gsc;
    if (p.g2) g += p.g2[i];
    const float x = p.x ? p.x[i] : 0.f, y = p.y ? p.y[i] : 0.f;
    float dx, dy;
    dfun<FN>(x, y, p.a, p.tanh_from_output, dx, dy);
    if (p.gx) p.gx[i] = g * dx;
    if (p.gy) p.gy[i] = g * dy;
}

template <int FN, bool VEC>
__global__ void __launch_bounds__(256) map_bwd_kernel(BwdArgs p)
{
    const float gsc = p.gs_dev ? __ldg(p.gs_dev) : p.gs_host;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!VEC) {
        for (int64_t i = t; i < p.n; i += stride) one<FN>(p, i, gsc);
        return;
    }
    const int64_t nv = p.n / 4;
    for (int64_t v = t; v < nv; v += stride) {
        float4 g4 = p.g ? dev::ld_stream(reinterpret_cast<const float4 *>(p.g) + v) : make_float4(gsc, gsc, gsc, gsc);
        if (p.g2) {
            const float4 h4 = dev::ld_stream(reinterpret_cast<const float4 *>(p.g2) + v);
            g4.x += h4.x;
            g4.y += h4.y;
            g4.z += h4.z;
            g4.w += h4.w;
        }
        float4 x4 = p.x ? dev::ld_stream(reinterpret_cast<const float4 *>(p.x) + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 y4 = p.y ? dev::ld_stream(reinterpret_cast<const float4 *>(p.y) + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float *gv = &g4.x, *xv = &x4.x, *yv = &y4.x;
        float4 ox, oy;
        float *oxv = &ox.x, *oyv = &oy.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float dx, dy;
            dfun<FN>(xv[j], yv[j], p.a, p.tanh_from_output, dx, dy);
            oxv[j] = gv[j] * dx;
            oyv[j] = gv[j] * dy;
        }
        if (p.gx) dev::st_stream(reinterpret_cast<float4 *>(p.gx) + v, ox);
        if (p.gy) dev::st_stream(reinterpret_cast<float4 *>(p.gy) + v, oy);
    }
    if (t < p.n - 4 * nv) one<FN>(p, 4 * nv + t, gsc);
}

template <int FN>
int run(const BwdArgs &p, cudaStream_t s)
{
    const bool vec = aligned16(p.x) && aligned16(p.y) && aligned16(p.g) && aligned16(p.g2) && aligned16(p.gx) &&
                     aligned16(p.gy);
    int64_t grid = ceil_div(vec ? ceil_div(p.n, 4) : p.n, 256);
    const int64_t cap = (int64_t)device_info().sms * 8 * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (vec) launch_kernel(map_bwd_kernel<FN, true>, (unsigned)grid, 256, 0, s, p);
    else launch_kernel(map_bwd_kernel<FN, false>, (unsigned)grid, 256, 0, s, p);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "map backward launch");
}

}  // namespace

int launch_map_bwd(const MapBwdLaunch &m, cudaStream_t s)
{
    if (m.n == 0) return SKEL_OK;
    BwdArgs p{m.a, m.tanh_from_output, m.in0, m.in1, m.g, m.g2, m.g_scalar_dev, m.g_scalar_host, m.gin0, m.gin1, m.n};
    switch (m.fn) {
    case SKEL_FN_AXPY: return run<SKEL_FN_AXPY>(p, s);
    case SKEL_FN_ADD: return run<SKEL_FN_ADD>(p, s);
    case SKEL_FN_SUB: return run<SKEL_FN_SUB>(p, s);
    case SKEL_FN_MUL: return run<SKEL_FN_MUL>(p, s);
    case SKEL_FN_TANH: return run<SKEL_FN_TANH>(p, s);
    case SKEL_FN_SQ: return run<SKEL_FN_SQ>(p, s);
    case SKEL_FN_SCALE: return run<SKEL_FN_SCALE>(p, s);
    case SKEL_FN_COPY: return run<SKEL_FN_COPY>(p, s);
    default: return fail(SKEL_ERR_UNSUPPORTED, "map backward: function has no adjoint here");
    }
}

}  // namespace skel
