// Shared pieces of the flat segmented batched variants (k_batched_seg.cu,
// k_batched_rr.cu): the instances lie end to end in `values`, so the call is
// one scan of the whole array that restarts at every instance start, plus a
// segmented sum of squares read at every instance's last element.
#pragma once

#include "scan_tile.cuh"

namespace skel {
namespace {

using dev::Pair;
constexpr int kBlock = 256;
constexpr int kSubTile = 4096;   // elements of a 16 KiB sub-tile

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// (sum, sum of squares, has-head) triples; combined in order by
// (a, b) -> b.head ? b : (a.s + b.s, a.q + b.q, a.head).
struct Seg {
    float s, q;
    int h;
};
__device__ __forceinline__ Seg seg_add(const Seg &a, const Seg &b)
{
    return b.h ? b : Seg{a.s + b.s, a.q + b.q, a.h};
}
// Inclusive segmented scan over the lanes of a warp.
__device__ __forceinline__ Seg warp_seg_scan(Seg v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float s = __shfl_up_sync(0xffffffffu, v.s, o);
        const float q = __shfl_up_sync(0xffffffffu, v.q, o);
        const int h = __shfl_up_sync(0xffffffffu, v.h, o);
        if (lane >= o && !v.h) {
            v.s += s;
            v.q += q;
            v.h = h;
        }
    }
    return v;
}


}  // namespace
}  // namespace skel
