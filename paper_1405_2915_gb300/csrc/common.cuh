// Device-side helpers shared by the kernel translation units: cache-hinted
// 128-bit loads/stores, warp/block reductions and scans, the map functors,
// and the acquire/release accesses of the look-back protocol.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <math.h>

#include "internal.h"

namespace skel {
namespace dev {

constexpr int kWarp = 32;

// ------------------------------------------------------ memory accesses ---
// Streaming read: bypass L1 allocation (each byte is read once).
__device__ __forceinline__ float4 ld_stream(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
// Streaming write: evict-first in L2 (the output is not re-read by this kernel).
__device__ __forceinline__ void st_stream(float4 *p, float4 v)
{
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ void st_stream(uint4 *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// Release store / acquire load at GPU scope (look-back flags).
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------ operators ---
struct AddF { __device__ __forceinline__ static float id() { return 0.f; }
              __device__ __forceinline__ static float op(float a, float b) { return a + b; } };
struct MaxF { __device__ __forceinline__ static float id() { return -INFINITY; }
              __device__ __forceinline__ static float op(float a, float b) { return fmaxf(a, b); } };
// int32 (+) wraps modulo 2^32: computed on the unsigned bit pattern.
struct AddU { __device__ __forceinline__ static uint32_t id() { return 0u; }
              __device__ __forceinline__ static uint32_t op(uint32_t a, uint32_t b) { return a + b; } };
// int32 max on the unsigned bit pattern, compared as signed.
struct MaxI { __device__ __forceinline__ static uint32_t id() { return 0x80000000u; }
              __device__ __forceinline__ static uint32_t op(uint32_t a, uint32_t b) {
                  return (int32_t)a > (int32_t)b ? a : b; } };

template <class Op, class T>
__device__ __forceinline__ T warp_reduce(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Op::op(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction; result valid in every thread.  smem: >= 32 entries.
template <class Op, class T, int BLOCK>
__device__ __forceinline__ T block_reduce(T v, T *smem)
{
    constexpr int NW = BLOCK / kWarp;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_reduce<Op>(v);
    if (lane == 0) smem[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < NW ? smem[lane] : Op::id();
        t = warp_reduce<Op>(t);
        if (lane == 0) smem[0] = t;
    }
    __syncthreads();
    T r = smem[0];
    __syncthreads();
    return r;
}

// Inclusive warp scan (Hillis-Steele over 32 lanes).
template <class T>
__device__ __forceinline__ T warp_incl_scan_add(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = v + t;
    }
    return v;
}

// ----------------------------------------------------------- map functors --
// out = f(x, y; a), one instantiation per skel_fn (the compiled-in user
// functions of the map skeleton).
template <int FN> struct MapF;
template <> struct MapF<SKEL_FN_ADD>   { static constexpr int nin = 2; __device__ __forceinline__ static float f(float x, float y, float) { return x + y; } };
template <> struct MapF<SKEL_FN_SUB>   { static constexpr int nin = 2; __device__ __forceinline__ static float f(float x, float y, float) { return x - y; } };
template <> struct MapF<SKEL_FN_MUL>   { static constexpr int nin = 2; __device__ __forceinline__ static float f(float x, float y, float) { return x * y; } };
template <> struct MapF<SKEL_FN_MAX>   { static constexpr int nin = 2; __device__ __forceinline__ static float f(float x, float y, float) { return fmaxf(x, y); } };
template <> struct MapF<SKEL_FN_AXPY>  { static constexpr int nin = 2; __device__ __forceinline__ static float f(float x, float y, float a) { return fmaf(a, x, y); } };
template <> struct MapF<SKEL_FN_TANH>  { static constexpr int nin = 1; __device__ __forceinline__ static float f(float x, float, float) { return tanhf(x); } };
template <> struct MapF<SKEL_FN_SQ>    { static constexpr int nin = 1; __device__ __forceinline__ static float f(float x, float, float) { return x * x; } };
template <> struct MapF<SKEL_FN_SCALE> { static constexpr int nin = 1; __device__ __forceinline__ static float f(float x, float, float a) { return a * x; } };
template <> struct MapF<SKEL_FN_COPY>  { static constexpr int nin = 1; __device__ __forceinline__ static float f(float x, float, float) { return x; } };

__device__ __forceinline__ float4 map4_apply(float4 x, float4 y, float a,
                                             float (*fn)(float, float, float))
{
    return make_float4(fn(x.x, y.x, a), fn(x.y, y.y, a), fn(x.z, y.z, a), fn(x.w, y.w, a));
}

}  // namespace dev

// Host helpers ------------------------------------------------------------
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Every kernel of the library is launched through this wrapper, which
// counts launches (skel_launch_count).
template <class... KArgs, class... Args>
inline void launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args &&...args)
{
    kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
    note_launch();
}
inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace skel
