// Reduce and MapReduce skeletons (Sec. III reduce; MapReduce = a reduce over
// mapped elements, r = (+)_i f(x_i, y_i)).
//
// Variants:
//   0 two_pass     kernel 1: a grid of at most one wave of blocks reduces
//                  grid-strided float4/uint4 groups into per-block partials;
//                  kernel 2: one block reduces the partials in index order.
//   1 single_pass  the same first phase; the last block to finish (counter in
//                  the scratch control block, reset by that block) reduces the
//                  partials -- one launch, no second kernel.
//   2 one_block    a single block reduces everything (small n: no partials).
// Every variant combines in an order fixed by (n, block, ept, grid), so the
// float32 result is deterministic.  The map of MapReduce (MUL: dot product,
// SQ: sum of squares) is applied on the load path, so x*y is never stored.
#include "common.cuh"

namespace skel {
namespace {

using dev::AddF;
using dev::AddU;
using dev::MaxF;
using dev::MaxI;

template <class T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<uint32_t> { using type = uint4; };

// Mapped value of one element (MAPF: -1 none, SKEL_FN_MUL, SKEL_FN_SQ).
template <int MAPF, class T>
__device__ __forceinline__ T mapped(T x, T y)
{
    if constexpr (MAPF == SKEL_FN_MUL) return x * y;
    else if constexpr (MAPF == SKEL_FN_SQ) return x * x;
    else return x;
}

template <class Op, int MAPF, class T, class V>
__device__ __forceinline__ T fold4(T acc, V a, V b)
{
    acc = Op::op(acc, mapped<MAPF>(a.x, b.x));
    acc = Op::op(acc, mapped<MAPF>(a.y, b.y));
    acc = Op::op(acc, mapped<MAPF>(a.z, b.z));
    acc = Op::op(acc, mapped<MAPF>(a.w, b.w));
    return acc;
}

struct Span {
    int head;       // scalar elements before the first 16-byte boundary
    int64_t nvec;   // full 4-element groups after the head
    int tail;       // scalar elements after the last group
    bool vec;       // 16-byte path usable
};

// Per-thread partial over the thread's share [tid, stride) of the groups,
// EPT groups in flight, then the scalar edge elements.
template <class Op, int MAPF, int NIN, int EPT, class T>
__device__ __forceinline__ T thread_partial(const T *__restrict__ x, const T *__restrict__ y,
                                            int64_t n, Span sp, int64_t tid, int64_t nthreads)
{
    using V = typename Vec4<T>::type;
    T acc[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) acc[k] = Op::id();
    if (sp.vec) {
        const V *x4 = reinterpret_cast<const V *>(x + sp.head);
        const V *y4 = reinterpret_cast<const V *>(y + sp.head);
        const int64_t step = nthreads * EPT;
        int64_t base = tid;
        for (; base + (EPT - 1) * nthreads < sp.nvec; base += step) {
            V a[EPT], b[EPT];
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                a[k] = dev::ld_stream(x4 + base + k * nthreads);
                if (NIN == 2) b[k] = dev::ld_stream(y4 + base + k * nthreads);
            }
#pragma unroll
            for (int k = 0; k < EPT; ++k) acc[k] = fold4<Op, MAPF>(acc[k], a[k], NIN == 2 ? b[k] : a[k]);
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            int64_t i = base + k * nthreads;
            if (i < sp.nvec) {
                V a = dev::ld_stream(x4 + i);
                V b = NIN == 2 ? dev::ld_stream(y4 + i) : a;
                acc[k] = fold4<Op, MAPF>(acc[k], a, b);
            }
        }
        if (tid < sp.head + sp.tail) {
            int64_t i = tid < sp.head ? tid : sp.head + 4 * sp.nvec + (tid - sp.head);
            acc[0] = Op::op(acc[0], mapped<MAPF>(x[i], NIN == 2 ? y[i] : x[i]));
        }
    } else {
        for (int64_t i = tid; i < n; i += nthreads)
            acc[0] = Op::op(acc[0], mapped<MAPF>(x[i], NIN == 2 ? y[i] : x[i]));
    }
    T r = acc[0];
#pragma unroll
    for (int k = 1; k < EPT; ++k) r = Op::op(r, acc[k]);
    return r;
}

template <class Op, int MAPF, int NIN, int EPT, int BLOCK, class T>
__global__ void __launch_bounds__(BLOCK)
reduce_phase1(const T *__restrict__ x, const T *__restrict__ y, int64_t n, Span sp,
              T *__restrict__ partials, T *__restrict__ out, Control *ctl, int single_pass)
{
    __shared__ T smem[32];
    __shared__ int am_last;
    const int64_t nthreads = (int64_t)gridDim.x * BLOCK;
    const int64_t tid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
    T v = thread_partial<Op, MAPF, NIN, EPT>(x, y, n, sp, tid, nthreads);
    v = dev::block_reduce<Op, T, BLOCK>(v, smem);
    if (gridDim.x == 1) {   // one block: no partials
        if (threadIdx.x == 0) *out = v;
        return;
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v;
        if (single_pass) {
            __threadfence();
            unsigned prev = atomicAdd(&ctl->done, 1u);
            am_last = (prev == gridDim.x - 1);
        }
    }
    if (!single_pass) return;
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    T w = Op::id();
    for (int i = threadIdx.x; i < (int)gridDim.x; i += BLOCK) w = Op::op(w, __ldcg(partials + i));
    w = dev::block_reduce<Op, T, BLOCK>(w, smem);
    if (threadIdx.x == 0) {
        *out = w;
        ctl->done = 0u;   // every block has incremented: safe to reset for the next call
    }
}

template <class Op, int BLOCK, class T>
__global__ void __launch_bounds__(BLOCK)
reduce_phase2(const T *__restrict__ partials, int count, T *__restrict__ out)
{
    __shared__ T smem[32];
    T w = Op::id();
    for (int i = threadIdx.x; i < count; i += BLOCK) w = Op::op(w, partials[i]);
    w = dev::block_reduce<Op, T, BLOCK>(w, smem);
    if (threadIdx.x == 0) *out = w;
}

template <class Op, int MAPF, int NIN, int BLOCK, class T>
int run_reduce_block(const ReduceLaunch &r, const Choice &c, cudaStream_t s)
{
    const T *x = static_cast<const T *>(r.in0);
    const T *y = static_cast<const T *>(r.in1);
    T *out = static_cast<T *>(r.out);
    Span sp{0, 0, 0, false};
    const uintptr_t mis = (uintptr_t)x & 15u;
    if ((mis & 3u) == 0 && (NIN == 1 || ((uintptr_t)y & 15u) == mis)) {
        int64_t head = mis ? (int64_t)((16u - mis) / 4u) : 0;
        if (head > r.n) head = r.n;
        sp.head = (int)head;
        sp.nvec = (r.n - head) / 4;
        sp.tail = (int)(r.n - head - 4 * sp.nvec);
        sp.vec = true;
    }
    const int ept = c.ept > 0 ? c.ept : 4;
    int64_t grid = 1;
    if (c.variant != 2) {
        const int64_t work = sp.vec ? sp.nvec : ceil_div(r.n, 4);
        grid = ceil_div(work, (int64_t)BLOCK * ept);
        const int64_t cap = (int64_t)device_info().sms * (2048 / BLOCK);
        if (grid > cap) grid = cap;
        if (grid < 1) grid = 1;
    }
    Scratch scr{};
    T *partials = nullptr;
    Control *ctl = nullptr;
    if (grid > 1) {
        int rc = get_scratch(s, (size_t)grid * sizeof(T), 0, &scr);
        if (rc) return rc;
        partials = reinterpret_cast<T *>(scr.data);
        ctl = scr.ctl;
    }
    const int single = c.variant == 1 ? 1 : 0;
#define SKEL_RED_EPT(E) launch_kernel(reduce_phase1<Op, MAPF, NIN, E, BLOCK, T>, (unsigned)grid, BLOCK, 0, s, x, y, r.n, sp, partials, out, ctl, single)
    switch (ept) {
    case 1: SKEL_RED_EPT(1); break;
    case 2: SKEL_RED_EPT(2); break;
    case 4: SKEL_RED_EPT(4); break;
    case 8: SKEL_RED_EPT(8); break;
    default: return fail(SKEL_ERR_INVALID_ARG, "reduce: ept must be 1, 2, 4 or 8");
    }
#undef SKEL_RED_EPT
    if (c.variant == 0 && grid > 1)
        launch_kernel(reduce_phase2<Op, BLOCK, T>, 1, BLOCK, 0, s, partials, (int)grid, out);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "reduce launch");
}

template <class Op, int MAPF, int NIN, class T>
int run_reduce(const ReduceLaunch &r, const Choice &c, cudaStream_t s)
{
    const int block = c.block > 0 ? c.block : 256;
    switch (block) {
    case 128: return run_reduce_block<Op, MAPF, NIN, 128, T>(r, c, s);
    case 256: return run_reduce_block<Op, MAPF, NIN, 256, T>(r, c, s);
    case 512: return run_reduce_block<Op, MAPF, NIN, 512, T>(r, c, s);
    case 1024: return run_reduce_block<Op, MAPF, NIN, 1024, T>(r, c, s);
    default: return fail(SKEL_ERR_INVALID_ARG, "reduce: block must be 128, 256, 512 or 1024");
    }
}

// Writes the identity (n = 0).
template <class T>
__global__ void write_scalar(T *out, T v) { *out = v; }

}  // namespace

int reduce_variant_count() { return 3; }
const char *reduce_variant_name(int v)
{
    static const char *names[] = {"two_pass", "single_pass", "one_block"};
    return v >= 0 && v < 3 ? names[v] : "?";
}
Choice reduce_default() { return Choice{0, 256, 4, 0}; }

int launch_reduce(const ReduceLaunch &r, const Choice &c, cudaStream_t s)
{
    if (c.variant < 0 || c.variant > 2) return fail(SKEL_ERR_INVALID_ARG, "reduce: unknown variant");
    if (r.n == 0) {
        if (r.dtype == SKEL_F32)
            launch_kernel(write_scalar<float>, 1, 1, 0, s, (float *)r.out, r.op == SKEL_FN_MAX ? -INFINITY : 0.f);
        else
            launch_kernel(write_scalar<uint32_t>, 1, 1, 0, s, (uint32_t *)r.out, r.op == SKEL_FN_MAX ? 0x80000000u : 0u);
        cudaError_t e = cudaPeekAtLastError();
        return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "reduce identity");
    }
    if (r.dtype == SKEL_F32) {
        if (r.map_fn == SKEL_FN_MUL) {
            if (r.op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce: reduce op must be ADD");
            return run_reduce<AddF, SKEL_FN_MUL, 2, float>(r, c, s);
        }
        if (r.map_fn == SKEL_FN_SQ) {
            if (r.op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce: reduce op must be ADD");
            return run_reduce<AddF, SKEL_FN_SQ, 1, float>(r, c, s);
        }
        if (r.map_fn != -1) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce: map must be MUL or SQ");
        if (r.op == SKEL_FN_ADD) return run_reduce<AddF, -1, 1, float>(r, c, s);
        if (r.op == SKEL_FN_MAX) return run_reduce<MaxF, -1, 1, float>(r, c, s);
        return fail(SKEL_ERR_UNSUPPORTED, "reduce: op must be ADD or MAX");
    }
    if (r.dtype == SKEL_I32) {
        if (r.map_fn != -1) return fail(SKEL_ERR_DTYPE, "mapreduce: float32 only");
        if (r.op == SKEL_FN_ADD) return run_reduce<AddU, -1, 1, uint32_t>(r, c, s);
        if (r.op == SKEL_FN_MAX) return run_reduce<MaxI, -1, 1, uint32_t>(r, c, s);
        return fail(SKEL_ERR_UNSUPPORTED, "reduce: op must be ADD or MAX");
    }
    return fail(SKEL_ERR_DTYPE, "reduce: float32 or int32 only");
}

}  // namespace skel
