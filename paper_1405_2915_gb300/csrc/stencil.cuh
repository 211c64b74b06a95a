// Building blocks of the 2D MapOverlap kernels shared by the stencil
// skeleton (k_stencil.cu) and the composed Map -> MapOverlap -> MapReduce
// chain (k_compose.cu): the boundary map of an axis and the 3x3 weighted sum
// in its fixed tap order, so that both evaluate a stencil output with the
// same operations.
#pragma once

#include "common.cuh"

namespace skel {

struct W9 { float w[9]; };
struct W33 { float w[33]; };

// Source index of logical index k on an axis of length n, or -1 (read as 0).
__device__ __forceinline__ int64_t bmap(int64_t k, int64_t n, int b)
{
    if (k >= 0 && k < n) return k;
    if (b == SKEL_CLAMP) return k < 0 ? 0 : n - 1;
    if (b == SKEL_PERIODIC) { int64_t m = k % n; return m < 0 ? m + n : m; }
    return -1;
}

__device__ __forceinline__ float at2(const float *__restrict__ in, int64_t r, int64_t c, int64_t rows,
                                     int64_t cols, int b)
{
    const int64_t sr = bmap(r, rows, b), sc = bmap(c, cols, b);
    return (sr < 0 || sc < 0) ? 0.f : __ldg(in + sr * cols + sc);
}

// The 3x3 weighted sum in a fixed tap order (row-major over di, dj).
template <bool TAPS5>
__device__ __forceinline__ float stencil9(const W9 &w, float a0, float a1, float a2, float b0, float b1,
                                          float b2, float c0, float c1, float c2)
{
    float acc = 0.f;
    if (!TAPS5) acc = fmaf(w.w[0], a0, acc);
    acc = fmaf(w.w[1], a1, acc);
    if (!TAPS5) acc = fmaf(w.w[2], a2, acc);
    acc = fmaf(w.w[3], b0, acc);
    acc = fmaf(w.w[4], b1, acc);
    acc = fmaf(w.w[5], b2, acc);
    if (!TAPS5) acc = fmaf(w.w[6], c0, acc);
    acc = fmaf(w.w[7], c1, acc);
    if (!TAPS5) acc = fmaf(w.w[8], c2, acc);
    return acc;
}

}  // namespace skel
