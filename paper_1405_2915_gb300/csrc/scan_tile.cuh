// Tile-level building blocks of the scan kernels (single scans, row-wise
// scans, reverse scans and the batched instances all use them).
//
// A tile is BLOCK threads x 4V elements.  Warp w owns the contiguous logical
// range [w*32*4V, (w+1)*32*4V) of the tile; inside it, step k of lane l holds
// the 4 consecutive elements at k*128 + l*4 + j (j = 0..3), so each step is one
// fully coalesced 128-bit access per lane.  The scan runs in that order:
// per-thread over j, a warp scan over lanes, a carry over steps k, then the
// warps' aggregates, then the tile prefix (look-back or a carried prefix).
#pragma once

#include "common.cuh"

namespace skel {
namespace dev {

template <class T> struct ScanTypes;
// float32 elements: element arithmetic in float32, carry between tiles in float64
template <> struct ScanTypes<float> { using V4 = float4; using CT = double; };
// int32 elements as uint32 bit patterns: (+) modulo 2^32, exact in any order
template <> struct ScanTypes<uint32_t> { using V4 = uint4; using CT = uint32_t; };

template <class T> __device__ __forceinline__ T to_elem(typename ScanTypes<T>::CT v);
template <> __device__ __forceinline__ float to_elem<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ uint32_t to_elem<uint32_t>(uint32_t v) { return v; }

// Where the tile's logical element e lives: phys = rev ? base - e : base + e.
struct TileMap {
    int64_t base;
    int64_t len;   // valid logical elements in this tile (<= TILE)
    bool rev;
    bool vec;      // 16-byte accesses allowed (full, aligned tile)
};

template <class T, int BLOCK, int V>
__device__ __forceinline__ void tile_load(const T *__restrict__ in, const TileMap &m, T (&v)[V][4])
{
    using V4 = typename ScanTypes<T>::V4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)w * 128 * V;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int64_t e = wbase + k * 128 + lane * 4;
        if (m.vec) {
            if (!m.rev) {
                V4 q = ld_stream(reinterpret_cast<const V4 *>(in + m.base + e));
                v[k][0] = q.x; v[k][1] = q.y; v[k][2] = q.z; v[k][3] = q.w;
            } else {
                V4 q = ld_stream(reinterpret_cast<const V4 *>(in + m.base - e - 3));
                v[k][0] = q.w; v[k][1] = q.z; v[k][2] = q.y; v[k][3] = q.x;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t ej = e + j;
                v[k][j] = ej < m.len ? in[m.rev ? m.base - ej : m.base + ej] : T(0);
            }
        }
    }
}

template <class T, int BLOCK, int V>
__device__ __forceinline__ void tile_store(T *__restrict__ out, const TileMap &m, const T (&v)[V][4])
{
    using V4 = typename ScanTypes<T>::V4;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)w * 128 * V;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int64_t e = wbase + k * 128 + lane * 4;
        if (m.vec) {
            if (!m.rev) {
                V4 q; q.x = v[k][0]; q.y = v[k][1]; q.z = v[k][2]; q.w = v[k][3];
                st_stream(reinterpret_cast<V4 *>(out + m.base + e), q);
            } else {
                V4 q; q.x = v[k][3]; q.y = v[k][2]; q.z = v[k][1]; q.w = v[k][0];
                st_stream(reinterpret_cast<V4 *>(out + m.base - e - 3), q);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t ej = e + j;
                if (ej < m.len) out[m.rev ? m.base - ej : m.base + ej] = v[k][j];
            }
        }
    }
}

// Scans the tile held in v in place (tile-local inclusive or exclusive
// prefix, without the tile prefix).  Returns the tile aggregate in every
// thread.  smem: >= BLOCK/32 + 1 entries of T.
template <class T, bool INCL, int BLOCK, int V>
__device__ __forceinline__ T tile_scan_local(T (&v)[V][4], T *smem)
{
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T base[V];
    T carry = T(0);
#pragma unroll
    for (int k = 0; k < V; ++k) {
        T s0 = v[k][0], s1 = s0 + v[k][1], s2 = s1 + v[k][2], s3 = s2 + v[k][3];
        T wi = warp_incl_scan_add(s3);
        T lex = __shfl_up_sync(0xffffffffu, wi, 1);
        if (lane == 0) lex = T(0);
        T wtot = __shfl_sync(0xffffffffu, wi, 31);
        base[k] = carry + lex;
        carry = carry + wtot;
        if (INCL) { v[k][0] = s0; v[k][1] = s1; v[k][2] = s2; v[k][3] = s3; }
        else      { v[k][0] = T(0); v[k][1] = s0; v[k][2] = s1; v[k][3] = s2; }
    }
    if (lane == 0) smem[w] = carry;
    __syncthreads();
    if (w == 0) {
        T a = lane < NW ? smem[lane] : T(0);
        T ai = warp_incl_scan_add(a);
        T ax = __shfl_up_sync(0xffffffffu, ai, 1);
        if (lane == 0) ax = T(0);
        if (lane < NW) smem[lane] = ax;
        if (lane == NW - 1) smem[NW] = ai;
    }
    __syncthreads();
    const T wex = smem[w];
    const T agg = smem[NW];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const T b = wex + base[k];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[k][j] = b + v[k][j];
    }
    __syncthreads();   // smem reused by the caller
    return agg;
}

// Adds the tile prefix to every element.
template <class T, int V>
__device__ __forceinline__ void tile_add_prefix(T (&v)[V][4], T p)
{
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) v[k][j] = p + v[k][j];
}

}  // namespace dev
}  // namespace skel

#include "lookback.cuh"
