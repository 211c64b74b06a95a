// A composed chain of three skeleton calls selected as a whole (Sec. II:
// composition of components, implementations selected for the composition
// rather than call by call):
//
//   t = Map f(x)                 f one of TANH, SQ, SCALE, COPY
//   u = MapOverlap S t           2D, radius 1 (5-point or 3x3 weights)
//   result = MapReduce(sq, +) u  sum of squares
//
// Variant 0 (per_call, in api.cpp) runs the three calls, each dispatched as
// usual, through two n-element temporaries: 8 + 8 + 4 = 20 bytes per point
// of HBM traffic.  Variant 1 (fused, here) reads x once: 4 bytes per point.
// Each warp walks a 128-column strip down `tile` rows with a three-row
// register window (the column walk of the MapOverlap skeleton), applies f to
// every value once its row has landed (values outside a ZERO boundary stay
// 0: the boundary pads t, not x, and every offered f has f(0) = 0), keeps
// the next rows' loads in flight meanwhile, computes the stencil outputs with the same
// operations as the stencil skeleton (so u is the same float per point as in
// variant 0), squares them and adds them to a compensated per-thread sum.  A
// block writes one float partial; the caller adds the partials with one
// Reduce call.
#include "stencil.cuh"

namespace skel {
namespace {

struct Row6 { float l, x0, x1, x2, x3, r; };

template <bool TAPS5, int FN, int RH>
__global__ void __launch_bounds__(128, 5)
compose_colwalk(const float *__restrict__ in, int64_t rows, int64_t cols, int b, W9 w, float a,
                float *__restrict__ partials)
{
    __shared__ float wsum[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t strip0 = ((int64_t)blockIdx.x * 4 + warp) * 128;
    float sum = 0.f, comp = 0.f;   // Kahan: the running sum and the low-order part it lost
    if (strip0 < cols) {           // warp-uniform
        const int64_t c0 = strip0 + 4 * lane;
        const bool active = c0 < cols;   // cols % 4 == 0: all four columns valid
        const int64_t r0 = (int64_t)blockIdx.y * RH;
        const int64_t r1 = r0 + RH < rows ? r0 + RH : rows;
        const int64_t cl = bmap(c0 - 1, cols, b), cr = bmap(c0 + 4, cols, b);
        const bool own_r = lane == 31 || c0 + 4 >= cols;
        auto f = [&](float x) { return dev::MapF<FN>::f(x, 0.f, a); };
        // Row r of x as this lane needs it: its four columns, and (lane 0 /
        // the last lane of the row) the neighbour column outside the warp's
        // strip, all loads issued together and nothing waiting on them;
        // cells outside a ZERO boundary stay 0.
        constexpr int U = 4;
        // every row this warp loads lies in [r0 - 1, r1 + U - 1]; a block
        // whose rows are all inside the grid needs no boundary map for rows
        const bool interior = r0 >= 1 && r1 + U <= rows;   // block-uniform
        auto load = [&](int64_t r) {
            Row6 v{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const int64_t gr = interior ? r : bmap(r, rows, b);
            if (gr >= 0 && active) {
                const float *row = in + gr * cols;
                const float4 q = dev::ld_stream(reinterpret_cast<const float4 *>(row + c0));
                if (lane == 0 && cl >= 0) v.l = __ldg(row + cl);
                if (own_r && cr >= 0) v.r = __ldg(row + cr);
                v.x0 = q.x; v.x1 = q.y; v.x2 = q.z; v.x3 = q.w;
            }
            return v;
        };
        // Turns a landed row of x into the row of t = f(x): every offered f
        // has f(0) = 0, so the zero padding stays 0; the other lanes'
        // neighbours come by shuffle.
        auto finish = [&](Row6 &v) {
            v.x0 = f(v.x0); v.x1 = f(v.x1); v.x2 = f(v.x2); v.x3 = f(v.x3);
            const float up = __shfl_up_sync(0xffffffffu, v.x3, 1);
            const float dn = __shfl_down_sync(0xffffffffu, v.x0, 1);
            v.l = lane != 0 ? up : f(v.l);
            v.r = !own_r ? dn : f(v.r);
        };
        Row6 p = load(r0 - 1), m = load(r0);
        finish(p);
        finish(m);
        // batches of U rows, the next batch's loads in flight while the
        // current one is computed
        Row6 cur[U], nxt[U] = {};
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = load(r0 + 1 + u);   // rows past r1 are loaded but unused
        for (int64_t r = r0; r < r1; r += U) {
            if (r + U < r1) {   // warp-uniform
#pragma unroll
                for (int u = 0; u < U; ++u) nxt[u] = load(r + U + 1 + u);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                finish(cur[u]);
                if (r + u < r1 && active) {
                    const Row6 &z = cur[u];
                    const float o0 = stencil9<TAPS5>(w, p.l, p.x0, p.x1, m.l, m.x0, m.x1, z.l, z.x0, z.x1);
                    const float o1 = stencil9<TAPS5>(w, p.x0, p.x1, p.x2, m.x0, m.x1, m.x2, z.x0, z.x1, z.x2);
                    const float o2 = stencil9<TAPS5>(w, p.x1, p.x2, p.x3, m.x1, m.x2, m.x3, z.x1, z.x2, z.x3);
                    const float o3 = stencil9<TAPS5>(w, p.x2, p.x3, p.r, m.x2, m.x3, m.r, z.x2, z.x3, z.r);
                    const float q = (o0 * o0 + o1 * o1) + (o2 * o2 + o3 * o3);
                    const float y = q - comp;
                    const float t = sum + y;
                    comp = (t - sum) - y;
                    sum = t;
                }
                p = m;
                m = cur[u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) cur[u] = nxt[u];
        }
    }
    float v = sum - comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = (wsum[0] + wsum[1]) + (wsum[2] + wsum[3]);
}

template <bool TAPS5, int FN>
int run_fn(const ComposeLaunch &cl, int tile, float *partials, dim3 grid, cudaStream_t s)
{
    W9 w;
    for (int k = 0; k < 9; ++k) w.w[k] = cl.w[k];
    switch (tile) {
    case 0: launch_kernel(compose_colwalk<TAPS5, FN, 32>, grid, 128, 0, s, cl.in, cl.rows, cl.cols, cl.boundary, w, cl.a, partials); break;
    case 1: launch_kernel(compose_colwalk<TAPS5, FN, 64>, grid, 128, 0, s, cl.in, cl.rows, cl.cols, cl.boundary, w, cl.a, partials); break;
    default: launch_kernel(compose_colwalk<TAPS5, FN, 128>, grid, 128, 0, s, cl.in, cl.rows, cl.cols, cl.boundary, w, cl.a, partials); break;
    }
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "fused chain launch");
}

template <bool TAPS5>
int run_taps(const ComposeLaunch &cl, int tile, float *partials, dim3 grid, cudaStream_t s)
{
    switch (cl.map_fn) {
    case SKEL_FN_TANH: return run_fn<TAPS5, SKEL_FN_TANH>(cl, tile, partials, grid, s);
    case SKEL_FN_SQ: return run_fn<TAPS5, SKEL_FN_SQ>(cl, tile, partials, grid, s);
    case SKEL_FN_SCALE: return run_fn<TAPS5, SKEL_FN_SCALE>(cl, tile, partials, grid, s);
    case SKEL_FN_COPY: return run_fn<TAPS5, SKEL_FN_COPY>(cl, tile, partials, grid, s);
    default: return fail(SKEL_ERR_UNSUPPORTED, "fused chain: map function not offered");
    }
}

dim3 grid_of(const ComposeLaunch &cl, int tile)
{
    return dim3((unsigned)ceil_div(cl.cols, 512), (unsigned)ceil_div(cl.rows, (int64_t)32 << tile));
}

}  // namespace

int compose_fused_check(const ComposeLaunch &cl, const Choice &c, int64_t *nparts)
{
    if (c.tile < 0 || c.tile > 2) return fail(SKEL_ERR_INVALID_ARG, "fused chain: tile must be 0..2 (32, 64, 128 rows)");
    if (cl.cols % 4 || !aligned16(cl.in))
        return fail(SKEL_ERR_UNSUPPORTED, "fused chain: 16-byte aligned rows needed (cols % 4 == 0)");
    const dim3 g = grid_of(cl, c.tile);
    if (ceil_div(cl.rows, (int64_t)32 << c.tile) > 65535) return fail(SKEL_ERR_SHAPE, "fused chain: too many rows");
    *nparts = (int64_t)g.x * g.y;
    return SKEL_OK;
}

int launch_compose_fused(const ComposeLaunch &cl, const Choice &c, float *partials, cudaStream_t s)
{
    int64_t np = 0;
    int rc = compose_fused_check(cl, c, &np);
    if (rc) return rc;
    const dim3 g = grid_of(cl, c.tile);
    return cl.taps5 ? run_taps<true>(cl, c.tile, partials, g, s) : run_taps<false>(cl, c.tile, partials, g, s);
}

int compose_variant_count() { return 2; }
const char *compose_variant_name(int v)
{
    static const char *names[] = {"per_call", "fused"};
    return v >= 0 && v < 2 ? names[v] : "?";
}
Choice compose_default() { return Choice{0, 0, 0, 0}; }

}  // namespace skel
