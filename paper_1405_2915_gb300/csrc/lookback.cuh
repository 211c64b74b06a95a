// Decoupled look-back between tiles (single-pass scans and the batched
// instances).
//
// Every tile publishes its aggregate, later its inclusive prefix, each as
// self-validating 64-bit words: the value and the call's tag travel in one
// word, written and read with relaxed GPU-scope accesses (an aligned 64-bit
// access is single-copy atomic).  One load therefore tells both whether the
// value is there and what it is -- no flag-then-value round trips and no
// acquire fences.  Encodings (the tag (epoch << 2) | 1 sits in the low 10
// bits of every word and is never 0, so zeroed memory reads as "not
// published"; an epoch is in 1..255 and the host clears the word region when
// its epoch counter wraps):
//   uint32 carry (int32 scans):  high 32 bits = value, low 32 = tag
//   float64 carry:               low 10 bits = tag, the rest are the value's
//                                top 54 bits (sign, exponent and 42 mantissa
//                                bits: truncation error 2^-42 relative per
//                                published value)
//   Pair (batched):              two float64 words (scan carry, sum of squares)
#pragma once

#include "common.cuh"

namespace skel {
namespace dev {

__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Two float64 running values carried together (batched instances: the
// scan carry and the sum of squares).
struct Pair {
    double s, q;
    Pair() = default;   // trivial, so a __shared__ Pair needs no initialisation
    __device__ __forceinline__ Pair(double v) : s(v), q(v) {}
    __device__ __forceinline__ Pair(double a, double b) : s(a), q(b) {}
};
__device__ __forceinline__ Pair operator+(const Pair &a, const Pair &b) { return Pair(a.s + b.s, a.q + b.q); }

template <class CT> __device__ __forceinline__ CT shfl_xor_ct(CT v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <class CT> __device__ __forceinline__ CT shfl_ct(CT v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <> __device__ __forceinline__ Pair shfl_xor_ct<Pair>(Pair v, int o)
{
    return Pair(__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.q, o));
}
template <> __device__ __forceinline__ Pair shfl_ct<Pair>(Pair v, int src)
{
    return Pair(__shfl_sync(0xffffffffu, v.s, src), __shfl_sync(0xffffffffu, v.q, src));
}

template <class CT> struct Codec;

// Every codec keeps the tag in the same low 10 bits: the word region is
// shared by calls of different element types, and a stale word of one type
// must never look valid to a reader of another (a value in the low bits
// would match a tag about once in 1024 words).
__device__ __forceinline__ uint64_t tag10(uint32_t epoch) { return (uint64_t)((epoch << 2) | 1u); }

template <> struct Codec<uint32_t> {
    static constexpr int W = 1;
    __device__ __forceinline__ static void put(uint64_t *w, uint32_t v, uint32_t epoch)
    {
        st_relaxed64(w, ((uint64_t)v << 32) | tag10(epoch));
    }
    __device__ __forceinline__ static bool get(const uint64_t *w, uint32_t epoch, uint32_t &v)
    {
        const uint64_t x = ld_relaxed64(w);
        v = (uint32_t)(x >> 32);
        return (x & 0xFFFFFFFFull) == tag10(epoch);
    }
};

__device__ __forceinline__ uint64_t enc_f64(double v, uint32_t epoch)
{
    return ((uint64_t)__double_as_longlong(v) & ~(uint64_t)0x3FF) | tag10(epoch);
}
__device__ __forceinline__ bool dec_f64(uint64_t x, uint32_t epoch, double &v)
{
    v = __longlong_as_double((long long)(x & ~(uint64_t)0x3FF));
    return (x & 0x3FF) == tag10(epoch);
}

template <> struct Codec<double> {
    static constexpr int W = 1;
    __device__ __forceinline__ static void put(uint64_t *w, double v, uint32_t epoch) { st_relaxed64(w, enc_f64(v, epoch)); }
    __device__ __forceinline__ static bool get(const uint64_t *w, uint32_t epoch, double &v)
    {
        return dec_f64(ld_relaxed64(w), epoch, v);
    }
};

template <> struct Codec<Pair> {
    static constexpr int W = 2;
    __device__ __forceinline__ static void put(uint64_t *w, const Pair &v, uint32_t epoch)
    {
        st_relaxed64(w, enc_f64(v.s, epoch));
        st_relaxed64(w + 1, enc_f64(v.q, epoch));
    }
    __device__ __forceinline__ static bool get(const uint64_t *w, uint32_t epoch, Pair &v)
    {
        const uint64_t a = ld_relaxed64(w), b = ld_relaxed64(w + 1);
        const bool ok_a = dec_f64(a, epoch, v.s), ok_b = dec_f64(b, epoch, v.q);
        return ok_a && ok_b;   // both halves of this publication are visible
    }
};

// Descriptor words of one call: aggregates and inclusive prefixes, W words
// per tile each.
struct LookbackDesc {
    uint64_t *agg;
    uint64_t *incl;
};

constexpr uint32_t kStAgg = 1u, kStIncl = 2u;

// Reads predecessor p's published state: status 2 (inclusive prefix), 1
// (aggregate only) or 0 (nothing yet), with the value.
template <class CT>
__device__ __forceinline__ uint32_t peek(const LookbackDesc &d, int64_t p, uint32_t epoch, CT &val)
{
    constexpr int W = Codec<CT>::W;
    CT vi, va;
    const bool hi = Codec<CT>::get(d.incl + p * W, epoch, vi);
    const bool ha = Codec<CT>::get(d.agg + p * W, epoch, va);
    val = hi ? vi : (ha ? va : CT(0));
    return hi ? kStIncl : (ha ? kStAgg : 0u);
}

// Run by all 32 lanes of one warp.  Publishes this tile's aggregate, walks
// back over the predecessors of the same segment (tiles >= first) in windows
// of 32 until it meets a published inclusive prefix, publishes this tile's
// inclusive prefix and returns the exclusive prefix (all lanes).  The wait is
// bounded by limit_ns (global timer) and by the shared abort word; on expiry
// it records kErrTimeout, sets abort to this call's epoch (so the other
// waiters of the same call stop at once, and a later call is unaffected) and
// counts unpublished tiles as 0.
template <class CT>
__device__ __forceinline__ CT lookback(int64_t tile, int64_t first, CT agg, LookbackDesc d, uint32_t epoch,
                                       Control *ctl, uint64_t limit_ns, bool publish)
{
    constexpr int W = Codec<CT>::W;
    const int lane = threadIdx.x & 31;
    if (tile == first) {
        if (publish && lane == 0) Codec<CT>::put(d.incl + tile * W, agg, epoch);
        return CT(0);
    }
    if (publish && lane == 0) Codec<CT>::put(d.agg + tile * W, agg, epoch);
    CT excl = CT(0);
    int64_t pred = tile - 1;
    uint64_t t0 = 0;
    bool gave_up = false;
    while (true) {
        const int64_t p = pred - lane;
        const bool inseg = p >= first;
        uint32_t status = 0;
        unsigned incl_mask = 0;
        CT val = CT(0);
        while (true) {
            if (inseg) status = peek<CT>(d, p, epoch, val);
            else { status = kStIncl; val = CT(0); }   // before the segment start: prefix 0
            const unsigned ready_mask = __ballot_sync(0xffffffffu, status != 0);
            incl_mask = __ballot_sync(0xffffffffu, status == kStIncl);
            const unsigned need = incl_mask ? (((incl_mask & (0u - incl_mask)) << 1) - 1u) : 0xffffffffu;
            if ((ready_mask & need) == need || gave_up) break;
            if (t0 == 0) t0 = globaltimer();
            bool expired = (globaltimer() - t0 > limit_ns) || ld_volatile(&ctl->abort) == epoch;
            expired = __any_sync(0xffffffffu, expired);
            if (expired) {
                if (lane == 0) {
                    atomicOr(&ctl->error, kErrTimeout);
                    atomicExch(&ctl->abort, epoch);
                }
                gave_up = true;
            }
        }
        const unsigned lim = incl_mask ? (((incl_mask & (0u - incl_mask)) << 1) - 1u) : 0xffffffffu;
        if (!((lim >> lane) & 1u) || status == 0) val = CT(0);
        if (sizeof(CT) == 4) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) val = val + shfl_xor_ct(val, o);
        } else {
            // float64 carries: a butterfly over the lanes up to the nearest
            // prefix only (usually a few; float64 adds are slow on this GPU),
            // then lane 0's sum to all lanes
            const int span = 32 - __clz(lim);   // lanes 0..span-1 take part
            for (int o = 16; o > 0; o >>= 1)
                if (o < span) val = val + shfl_xor_ct(val, o);   // warp-uniform
            val = shfl_ct(val, 0);
        }
        excl = excl + val;
        if (incl_mask) break;
        pred -= 32;
    }
    if (publish && lane == 0) Codec<CT>::put(d.incl + tile * W, excl + agg, epoch);
    return excl;
}

// Block-wide variant: all BLOCK threads take part, one predecessor each, so
// one round covers BLOCK predecessors.  Returns the exclusive prefix in every
// thread.
template <class CT, int BLOCK>
struct BlockLookbackSmem {
    CT part[BLOCK / 32];
    int incl_first[BLOCK / 32];
    int not_ready[BLOCK / 32];
    int expired;
};

template <class CT, int BLOCK>
__device__ __forceinline__ CT block_lookback(int64_t tile, int64_t first, CT agg, LookbackDesc d, uint32_t epoch,
                                             Control *ctl, uint64_t limit_ns, bool publish,
                                             BlockLookbackSmem<CT, BLOCK> &sm)
{
    constexpr int NW = BLOCK / 32, W = Codec<CT>::W;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tile == first) {
        if (publish && tid == 0) Codec<CT>::put(d.incl + tile * W, agg, epoch);
        return CT(0);
    }
    if (publish && tid == 0) Codec<CT>::put(d.agg + tile * W, agg, epoch);
    CT excl = CT(0);
    int64_t pred = tile - 1;
    uint64_t t0 = 0;
    bool gave_up = false;
    while (true) {
        const int64_t p = pred - tid;
        const bool inseg = p >= first;
        uint32_t status;
        CT val = CT(0);
        int lim;                // threads 0..lim take part in this round's sum
        int fi_round = BLOCK;   // thread of the nearest inclusive prefix (BLOCK: none)
        while (true) {
            if (inseg) status = peek<CT>(d, p, epoch, val);
            else { status = kStIncl; val = CT(0); }
            const unsigned im = __ballot_sync(0xffffffffu, status == kStIncl);
            if (lane == 0) sm.incl_first[w] = im ? w * 32 + __ffs(im) - 1 : BLOCK;
            __syncthreads();
            int fi = BLOCK;
#pragma unroll
            for (int k = 0; k < NW; ++k) fi = min(fi, sm.incl_first[k]);
            fi_round = fi;
            lim = fi < BLOCK ? fi : BLOCK - 1;
            const unsigned nr = __ballot_sync(0xffffffffu, status == 0u && tid <= lim);
            if (lane == 0) sm.not_ready[w] = nr != 0u;
            if (tid == 0) {
                bool exp = false;
                if (!gave_up) {
                    if (t0 == 0) t0 = globaltimer();
                    exp = (globaltimer() - t0 > limit_ns) || ld_volatile(&ctl->abort) == epoch;
                }
                sm.expired = exp;
            }
            __syncthreads();
            int any_nr = 0;
#pragma unroll
            for (int k = 0; k < NW; ++k) any_nr |= sm.not_ready[k];
            const int exp = sm.expired;
            __syncthreads();   // smem is rewritten by the next poll
            if (!any_nr || gave_up) break;
            if (exp) {
                if (tid == 0) {
                    atomicOr(&ctl->error, kErrTimeout);
                    atomicExch(&ctl->abort, epoch);
                }
                gave_up = true;
                break;
            }
        }
        if (tid > lim || status == 0) val = CT(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val = val + shfl_xor_ct(val, o);
        if (lane == 0) sm.part[w] = val;
        __syncthreads();
        CT s = CT(0);
#pragma unroll
        for (int k = 0; k < NW; ++k) s = s + sm.part[k];
        excl = excl + s;
        __syncthreads();   // sm.part is rewritten by the next round
        if (fi_round < BLOCK) break;
        pred -= BLOCK;
    }
    if (publish && tid == 0) Codec<CT>::put(d.incl + tile * W, excl + agg, epoch);
    return excl;
}

// Wide variant: each of the NW warps polls its own window of 32 predecessors
// (warp w: pred - 32w - lane) until the window is ready up to its nearest
// published prefix, so one round reads 32*NW predecessors with one barrier.
// Warps farther back wait on older tiles, which are the likeliest to be
// ready.  Returns the exclusive prefix in every thread.
template <class CT, int NW>
struct WideLookbackSmem {
    CT vals[32 * NW];   // each lane's predecessor value of the round (0 past a published prefix)
    int incl[NW];       // 1 if the warp's window holds a published prefix
    CT total;           // the running exclusive prefix after a round
    int found;          // the round reached a published prefix
};

// pub_agg: publish the aggregate first (false when the caller already has);
// pub_incl: publish the inclusive prefix at the end (for the segment's first
// tile: at once, unless the caller already has).
template <class CT, int NW>
__device__ __forceinline__ CT wide_lookback(int64_t tile, int64_t first, CT agg, LookbackDesc d, uint32_t epoch,
                                            Control *ctl, uint64_t limit_ns, bool pub_agg, bool pub_incl,
                                            WideLookbackSmem<CT, NW> &sm)
{
    constexpr int W = Codec<CT>::W;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (tile == first) {
        if (pub_incl && threadIdx.x == 0) Codec<CT>::put(d.incl + tile * W, agg, epoch);
        return CT(0);
    }
    if (pub_agg && threadIdx.x == 0) Codec<CT>::put(d.agg + tile * W, agg, epoch);
    const bool publish = pub_incl;
    CT excl = CT(0);
    int64_t pred = tile - 1;
    uint64_t t0 = 0;
    bool gave_up = false;
    while (true) {
        const int64_t p = pred - 32 * w - lane;
        const bool inseg = p >= first;
        uint32_t status = 0;
        unsigned incl_mask = 0;
        CT val = CT(0);
        while (true) {
            if (inseg) status = peek<CT>(d, p, epoch, val);
            else { status = kStIncl; val = CT(0); }
            const unsigned ready_mask = __ballot_sync(0xffffffffu, status != 0);
            incl_mask = __ballot_sync(0xffffffffu, status == kStIncl);
            const unsigned need = incl_mask ? (((incl_mask & (0u - incl_mask)) << 1) - 1u) : 0xffffffffu;
            if ((ready_mask & need) == need || gave_up) break;
            if (t0 == 0) t0 = globaltimer();
            bool expired = (globaltimer() - t0 > limit_ns) || ld_volatile(&ctl->abort) == epoch;
            expired = __any_sync(0xffffffffu, expired);
            if (expired) {
                if (lane == 0) {
                    atomicOr(&ctl->error, kErrTimeout);
                    atomicExch(&ctl->abort, epoch);
                }
                gave_up = true;
            }
        }
        const unsigned lim = incl_mask ? (((incl_mask & (0u - incl_mask)) << 1) - 1u) : 0xffffffffu;
        if (!((lim >> lane) & 1u) || status == 0) val = CT(0);
        sm.vals[w * 32 + lane] = val;
        if (lane == 0) sm.incl[w] = incl_mask != 0u;
        __syncthreads();
        // Warp 0 adds the windows up to the nearest one holding a published
        // prefix: lane l sums entry l of each of those windows, then one tree
        // over the lanes.  (float64 is a slow pipe on this part: this takes
        // k + 5 warp-wide adds for k windows, not 5 in every warp.)
        if (w == 0) {
            int kmax = NW - 1;
            bool found_any = false;
#pragma unroll
            for (int k = NW - 1; k >= 0; --k)
                if (sm.incl[k]) { kmax = k; found_any = true; }
            CT acc = CT(0);
            for (int k = 0; k <= kmax; ++k) acc = acc + sm.vals[k * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = acc + shfl_xor_ct(acc, o);
            if (lane == 0) {
                sm.total = excl + acc;
                sm.found = found_any;
            }
        }
        __syncthreads();
        excl = sm.total;
        const bool found = sm.found;
        __syncthreads();   // sm is rewritten by the next round
        if (found) break;
        pred -= 32 * NW;
    }
    if (publish && threadIdx.x == 0) Codec<CT>::put(d.incl + tile * W, excl + agg, epoch);
    return excl;
}

}  // namespace dev
}  // namespace skel
