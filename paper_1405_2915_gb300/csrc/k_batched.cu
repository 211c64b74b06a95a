// Batched uneven instances in one persistent launch: for every instance b
// (values[offsets[b] .. offsets[b+1])) the MapReduce sum of squares and the
// scan (+), fused so that each element is read once (8 bytes per element
// with both outputs, 4 with the sum only).
//
// Launch sequence (also the body of the captured CUDA graph):
//   prep    one block: validates the offsets, gives every instance
//           ceil((hi - (lo & ~3)) / TILE) tiles on a 16-byte aligned frame,
//           scans the tile counts into tile_start[], fills tile_inst[] and
//           writes 0 as the result of empty instances.
//   main    a grid of resident blocks; each takes tiles in increasing order
//           from an atomic queue, so a tile only waits on tiles that running
//           blocks already hold.  A tile loads its elements (elements of the
//           aligned frame outside the instance count as 0 and are not stored),
//           scans them, sums their squares, and finds both prefixes with a
//           look-back over the earlier tiles of its instance, carrying the
//           pair in float64.  The last tile of an instance writes its sum.
// Variants: 0 persistent (grid = SMs x resident blocks per SM); the tile's
//             aggregate is published right after its load, and all warps
//             walk the look-back in parallel windows;
//           1 one_per_tile (grid = the tile bound; surplus blocks exit),
//             otherwise as 0;
//           2 persistent with the whole block walking the look-back, one
//             predecessor per thread;
//           3 big_tile: 64 KiB frames staged by bulk copies, aggregates
//             published before the scans, all warps walking the look-back;
//           4 persistent with warp 0 alone walking the look-back;
//           5 reduce_then_scan: tile sums, per-instance prefixes, tile scans
//             (no look-back; the values are read twice);
//           6 flat_segmented: the instances as one flat array, scanned in
//             tiles of 128 KiB (96 KiB staged, 32 KiB in registers) that
//             restart at instance starts; a tile holding a start publishes
//             its tail at once, so look-back walks stop there (one read).
#include "scan_tile.cuh"

namespace skel {
namespace {

using dev::Pair;
constexpr int kBlock = 256;

struct Layout {
    int64_t *tile_start;   // B + 1
    int32_t *tile_inst;    // max_tiles
    int64_t *total_tiles;  // 1
};

size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t max_tiles(const BatchedLaunch &b, int tile)
{
    return (b.total + 3 * b.B) / tile + b.B + 1;
}

Layout layout(unsigned char *data, const BatchedLaunch &b, int tile)
{
    const int64_t mt = max_tiles(b, tile);
    Layout L;
    size_t off = 0;
    L.tile_start = reinterpret_cast<int64_t *>(data + off); off += r256((b.B + 1) * 8);
    L.tile_inst = reinterpret_cast<int32_t *>(data + off);  off += r256(mt * 4);
    L.total_tiles = reinterpret_cast<int64_t *>(data + off);
    return L;
}

size_t layout_bytes(const BatchedLaunch &b, int tile)
{
    const int64_t mt = max_tiles(b, tile);
    return r256((b.B + 1) * 8) + r256(mt * 4) + 256;
}

__device__ __forceinline__ int64_t ntiles_of(int64_t lo, int64_t hi, int tile)
{
    return hi > lo ? (hi - (lo & ~(int64_t)3) + tile - 1) / tile : 0;
}

__global__ void __launch_bounds__(1024)
batched_prep(const int64_t *__restrict__ off, int64_t B, int64_t total, int tile, Layout L,
             float *__restrict__ results, Control *ctl, int64_t max_t)
{
    constexpr int IPT = 4;
    __shared__ int64_t smem[33];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = (off[0] != 0 || off[B] != total) ? 1 : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < B; c0 += 1024 * IPT) {
        int64_t cnt[IPT];
        int64_t t = 0;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int64_t b = c0 + (int64_t)threadIdx.x * IPT + i;
            cnt[i] = 0;
            if (b < B) {
                const int64_t lo = off[b], hi = off[b + 1];
                if (hi < lo) bad = 1;
                else cnt[i] = ntiles_of(lo, hi, tile);
                if (hi <= lo && results) results[b] = 0.f;
            }
            t += cnt[i];
        }
        int64_t wi = dev::warp_incl_scan_add(t);
        if (lane == 31) smem[w] = wi;
        __syncthreads();
        if (w == 0) {
            const int64_t a = smem[lane];
            const int64_t ai = dev::warp_incl_scan_add(a);
            smem[lane] = ai - a;
            if (lane == 31) smem[32] = ai;
        }
        __syncthreads();
        int64_t run = carry + smem[w] + (wi - t);
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int64_t b = c0 + (int64_t)threadIdx.x * IPT + i;
            if (b < B) L.tile_start[b] = run;
            run += cnt[i];
        }
        carry += smem[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        L.tile_start[B] = carry;
        const bool ok = !bad && carry <= max_t;
        *L.total_tiles = ok ? carry : 0;
        if (!ok) atomicOr(&ctl->error, kErrInput);
    }
    __syncthreads();   // tile_start is complete (global writes of this block)
    // tile -> instance map: warp w fills the tiles of instances w, w+32, ...,
    // its lanes writing consecutive entries
    for (int64_t b = w; b < B; b += 32) {
        const int64_t s0 = L.tile_start[b], s1 = L.tile_start[b + 1];
        for (int64_t k = s0 + lane; k < s1 && k < max_t; k += 32) L.tile_inst[k] = (int32_t)b;
    }
}

// Loads the tile's elements [fbase, fbase + TILE) of the aligned frame; only
// positions in [lo, hi) are real (others read as 0).
template <int V>
__device__ __forceinline__ void load_masked(const float *__restrict__ in, int64_t fbase, int64_t lo, int64_t hi,
                                            float (&v)[V][4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int64_t p = fbase + (int64_t)w * 128 * V + k * 128 + lane * 4;
        if (p >= lo && p + 3 < hi) {
            const float4 q = dev::ld_stream(reinterpret_cast<const float4 *>(in + p));
            v[k][0] = q.x; v[k][1] = q.y; v[k][2] = q.z; v[k][3] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[k][j] = (p + j >= lo && p + j < hi) ? in[p + j] : 0.f;
        }
    }
}

template <int V>
__device__ __forceinline__ void store_masked(float *__restrict__ out, int64_t fbase, int64_t lo, int64_t hi,
                                             const float (&v)[V][4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int64_t p = fbase + (int64_t)w * 128 * V + k * 128 + lane * 4;
        if (p >= lo && p + 3 < hi) {
            dev::st_stream(reinterpret_cast<float4 *>(out + p), make_float4(v[k][0], v[k][1], v[k][2], v[k][3]));
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (p + j >= lo && p + j < hi) out[p + j] = v[k][j];
        }
    }
}

// ----------------------------------------------- variant 3: big tiles ----
// One block per 64 KiB frame of an instance (four 4096-element sub-tiles),
// drawn in ticket order: the frame [fbase, fbase + 16384) arrives by bulk
// copies into shared memory (clipped to the values array), the (scan, sum of
// squares) aggregate is published first, the sub-tiles are scanned in place,
// all warps walk the look-back over the instance's earlier tiles, and the
// prefix is added while the instance's elements are stored.
constexpr int kBigV = 4;
constexpr int kBigSub = 4;
constexpr int kSubTile = kBlock * 4 * kBigV;            // 4096
constexpr int kBigTile = kBigSub * kSubTile;            // 16384 elements

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <bool SCAN, bool RED, bool INCL>
__global__ void __launch_bounds__(kBlock, 3)
batched_big(const float *__restrict__ values, const int64_t *__restrict__ off, float *__restrict__ results,
            float *__restrict__ scan_out, Layout L, uint64_t *words, int64_t max_t, int64_t total_elems, Control *ctl,
            uint32_t epoch, uint64_t limit_ns)
{
    extern __shared__ __align__(1024) unsigned char dyn[];   // kBigTile floats
    float *buf = reinterpret_cast<float *>(dyn);
    __shared__ __align__(8) uint64_t bars[kBigSub];   // one per 16 KiB chunk (= sub-tile)
    __shared__ int64_t s_meta[5];   // tile, instance, lo, hi, first
    __shared__ int64_t s_last;
    __shared__ float smem[kBlock / 32 + 1];
    __shared__ float red[32];
    __shared__ dev::WideLookbackSmem<Pair, kBlock / 32> lbs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const dev::LookbackDesc d{words, words + 2 * max_t};
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(&ctl->queue, 1u);
        if ((int64_t)t == max_t - 1) ctl->queue = 0u;       // every block of the grid has drawn
        const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
        s_meta[0] = t;
        if ((int64_t)t < total) {
            const int64_t b = L.tile_inst[t];
            const int64_t lo = off[b], hi = off[b + 1], first = L.tile_start[b];
            s_meta[1] = b; s_meta[2] = lo; s_meta[3] = hi; s_meta[4] = first;
            s_last = L.tile_start[b + 1] - 1;
            const int64_t fbase = (lo & ~(int64_t)3) + ((int64_t)t - first) * kBigTile;
            int64_t end = fbase + kBigTile < hi ? fbase + kBigTile : hi;
            end = (end + 3) & ~(int64_t)3;                      // whole 16-byte groups ...
            if (end > (total_elems & ~(int64_t)3)) end = total_elems & ~(int64_t)3;   // ... inside the array
            const uint32_t bytes = end > fbase ? (uint32_t)((end - fbase) * 4) : 0u;
#pragma unroll
            for (int c = 0; c < kBigSub; ++c)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[c])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
            for (int c = 0; c < kBigSub; ++c) {
                const uint32_t bb = smem_u32(&bars[c]), o = (uint32_t)c * 16384u;
                if (o >= bytes) {   // nothing staged in this chunk: complete its phase at once
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bb) : "memory");
                    continue;
                }
                const uint32_t sz = bytes - o < 16384u ? bytes - o : 16384u;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bb), "r"(sz) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(smem_u32(dyn + o)),
                                "l"(reinterpret_cast<const unsigned char *>(values + fbase) + o), "r"(sz), "r"(bb)
                             : "memory");
            }
        }
    }
    __syncthreads();
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    const int64_t t = s_meta[0];
    if (t >= total) return;                                    // block-uniform: a surplus block
    const int64_t b = s_meta[1], lo = s_meta[2], hi = s_meta[3], first = s_meta[4], last = s_last;
    const int64_t fbase = (lo & ~(int64_t)3) + (t - first) * kBigTile;
    int64_t fend = fbase + kBigTile < hi ? fbase + kBigTile : hi;
    fend = (fend + 3) & ~(int64_t)3;
    if (fend > (total_elems & ~(int64_t)3)) fend = total_elems & ~(int64_t)3;   // staged: [fbase, fend)
    // Bounded wait for chunk c; block-uniform result.  On failure the block
    // records the timeout, waits (bounded) for every copy still landing in
    // its shared memory and leaves without publishing.
    auto wait_chunk = [&](int c) -> bool {
        uint32_t done = 0;
        for (uint32_t k = 0; k < (1u << 22) && !done; ++k)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done) : "r"(smem_u32(&bars[c])) : "memory");
        if (__syncthreads_and(done)) return true;
        if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
        for (int cc = 0; cc < kBigSub; ++cc) {
            uint32_t ok = 0;
            for (uint32_t k = 0; k < (1u << 22) && !ok; ++k)
                asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                             : "=r"(ok) : "r"(smem_u32(&bars[cc])) : "memory");
        }
        return false;
    };
    // element e of the frame: staged if fbase + e < fend, else read directly;
    // positions outside [lo, hi) count as 0
    auto at = [&](int64_t e) -> float {
        const int64_t p = fbase + e;
        if (p < lo || p >= hi) return 0.f;
        return p < fend ? buf[e] : values[p];
    };
    // early aggregates, each sub-tile as soon as its chunk has landed:
    // pairwise per thread (rounding depth 6), then the block trees
    float ps[kBigSub], pq[kBigSub];
#pragma unroll
    for (int j = 0; j < kBigSub; ++j) {
        if (!wait_chunk(j)) return;                             // block-uniform
        float gs[kBigV], gq[kBigV];
#pragma unroll
        for (int k = 0; k < kBigV; ++k) {
            const int64_t e = (int64_t)j * kSubTile + w * 128 * kBigV + k * 128 + lane * 4;
            float a[4];
            if (fbase + e >= lo && fbase + e + 3 < hi && fbase + e + 3 < fend) {
                const float4 q = *reinterpret_cast<const float4 *>(buf + e);
                a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = at(e + i);
            }
            gs[k] = (a[0] + a[1]) + (a[2] + a[3]);
            gq[k] = fmaf(a[0], a[0], a[1] * a[1]) + fmaf(a[2], a[2], a[3] * a[3]);
        }
        ps[j] = (gs[0] + gs[1]) + (gs[2] + gs[3]);
        pq[j] = (gq[0] + gq[1]) + (gq[2] + gq[3]);
    }
    const float agg_s = SCAN ? dev::block_reduce<dev::AddF, float, kBlock>((ps[0] + ps[1]) + (ps[2] + ps[3]), red)
                             : 0.f;
    const float agg_q = RED ? dev::block_reduce<dev::AddF, float, kBlock>((pq[0] + pq[1]) + (pq[2] + pq[3]), red)
                            : 0.f;
    const Pair agg((double)agg_s, (double)agg_q);
    const bool multi = first != last;
    if (multi && threadIdx.x == 0) {
        if (t == first) dev::Codec<Pair>::put(d.incl + t * 2, agg, epoch);
        else dev::Codec<Pair>::put(d.agg + t * 2, agg, epoch);
    }
    // pass A: scan the sub-tiles in place.  The carries into the sub-tiles
    // are block-uniform: kept in shared memory (written before the barriers
    // of the sub-tile's scan, read after them) rather than in registers.
    __shared__ double s_carry[kBigSub];
    double run = 0.0;
    if (SCAN) {
#pragma unroll
        for (int j = 0; j < kBigSub; ++j) {
            if (threadIdx.x == 0) s_carry[j] = run;
            const int64_t o = (int64_t)j * kSubTile;
            if (fbase + o >= hi) continue;                      // block-uniform
            float v[kBigV][4];
#pragma unroll
            for (int k = 0; k < kBigV; ++k) {
                const int64_t e = o + w * 128 * kBigV + k * 128 + lane * 4;
                if (fbase + e >= lo && fbase + e + 3 < hi && fbase + e + 3 < fend) {
                    const float4 q = *reinterpret_cast<const float4 *>(buf + e);
                    v[k][0] = q.x; v[k][1] = q.y; v[k][2] = q.z; v[k][3] = q.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[k][i] = at(e + i);
                }
            }
            const float sub = dev::tile_scan_local<float, INCL, kBlock, kBigV>(v, smem);
#pragma unroll
            for (int k = 0; k < kBigV; ++k) {
                const int64_t e = o + w * 128 * kBigV + k * 128 + lane * 4;
                *reinterpret_cast<float4 *>(buf + e) = make_float4(v[k][0], v[k][1], v[k][2], v[k][3]);
            }
            run += (double)sub;
        }
    }
    Pair p(0.0);
    if (multi)
        p = dev::wide_lookback<Pair, kBlock / 32>(t, first, agg, d, epoch, ctl, limit_ns, false, t != first, lbs);
    if (RED && t == last && threadIdx.x == 0) results[b] = (float)(p.q + agg.q);
    if (SCAN) {
        // pass B: add the prefix and store the instance's elements
#pragma unroll
        for (int j = 0; j < kBigSub; ++j) {
            const int64_t o = (int64_t)j * kSubTile;
            if (fbase + o >= hi) continue;
            const float pre = (float)(p.s + s_carry[j]);
#pragma unroll
            for (int k = 0; k < kBigV; ++k) {
                const int64_t e = o + w * 128 * kBigV + k * 128 + lane * 4;
                const float4 q = *reinterpret_cast<const float4 *>(buf + e);
                const float r[4] = {pre + q.x, pre + q.y, pre + q.z, pre + q.w};
                const int64_t pp = fbase + e;
                if (pp >= lo && pp + 3 < hi) {
                    dev::st_stream(reinterpret_cast<float4 *>(scan_out + pp), make_float4(r[0], r[1], r[2], r[3]));
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (pp + i >= lo && pp + i < hi) scan_out[pp + i] = r[i];
                }
            }
        }
    }
}

// ---------------------------------------- variant 6: flat segmented ----
// The instances lie end to end in `values`, so the batched call is one scan
// of the whole array that restarts at every instance start (a segmented
// scan), plus a segmented sum of squares read at every instance's last
// element.  Tiles of the flat array (every tile but the last is whole and
// 16-byte aligned, unlike per-instance frames, so short instances share a
// tile instead of each taking one), staged partly in shared memory and
// partly in registers as in scan variant 7, drawn in ticket order:
//   heads:  the instance starts inside the tile (a binary search of the
//           offsets), as a bitmap in shared memory;
//   pass 1: each warp's (sum, sum of squares) since the last head of its
//           range, and whether the range holds a head; one warp combines
//           them in tile order, which gives every warp its carry and the
//           tile's tail (the sums of the instance running at its end);
//   publish: a tile holding a head publishes its tail at once as an
//           inclusive prefix (it depends on no earlier tile), one without
//           publishes its sums as an aggregate;
//   look-back: only a tile whose first element is not a head walks back,
//           adding aggregates up to an inclusive prefix (then a tile without
//           heads publishes its own);
//   pass 2: each warp scans its elements (restarting at heads), stores them,
//           and the last element of each instance writes its sum of squares.
// The combine of (sum, sum of squares, has-head) triples in order is
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

// Offsets of a tile's instances kept in shared memory by the flat variant.
constexpr int kSegOffCap = 512;

// Offsets check for the flat variant: offsets[0] = 0, offsets[B] = total,
// non-decreasing; empty instances get 0 as their sum of squares.  *ok = 1 if
// valid (the main kernels do nothing otherwise).  tile_inst[t] = the
// instance holding the first element of tile t (each tile start lies in
// exactly one non-empty instance), so that a tile finds its instances with
// one load instead of a binary search on its critical path.
__global__ void __launch_bounds__(1024)
batched_seg_prep(const int64_t *__restrict__ off, int64_t B, int64_t total, int tile, float *__restrict__ results,
                 int *__restrict__ ok, int64_t *__restrict__ tile_inst, Control *ctl)
{
    __shared__ int bad;
    if (threadIdx.x == 0) bad = (off[0] != 0 || off[B] != total) ? 1 : 0;
    __syncthreads();
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const int64_t lo = off[b], hi = off[b + 1];
        if (hi < lo) bad = 1;
        else if (hi == lo && results) results[b] = 0.f;
    }
    __syncthreads();
    if (!bad)
        for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
            const int64_t lo = off[b], hi = off[b + 1];
            if (hi <= lo) continue;
            for (int64_t t = (lo + tile - 1) / tile; t <= (hi - 1) / tile; ++t) tile_inst[t] = b;
        }
    if (threadIdx.x == 0) {
        *ok = bad ? 0 : 1;
        if (bad) atomicOr(&ctl->error, kErrInput);
    }
}

template <bool SCAN, bool RED, bool INCL, int SUBS, int SUBR, int MINB, bool PART>
__global__ void __launch_bounds__(kBlock, MINB)
batched_seg(const float *__restrict__ values, const int64_t *__restrict__ off, int64_t B, int64_t total,
            float *__restrict__ results, float *__restrict__ scan_out, const int *__restrict__ ok,
            const int64_t *__restrict__ tile_inst, uint64_t *words, int64_t ntiles, Control *ctl, uint32_t epoch,
            uint64_t limit_ns)
{
    constexpr int NW = kBlock / 32, NS = SUBS + SUBR, TILE = NS * kSubTile, SLEN = SUBS * kSubTile;
    constexpr int PER = (NS * NW + 31) / 32;   // warp ranges per lane in the tile's combine
    extern __shared__ __align__(1024) unsigned char dyn[];   // SUBS x 16 KiB
    const float *buf = reinterpret_cast<const float *>(dyn);
    __shared__ __align__(8) uint64_t bars[SUBS];
    __shared__ uint32_t heads[TILE / 32 + 1];   // bit e: an instance starts at tile element e (e <= TILE)
    __shared__ int64_t s_tile;
    __shared__ int32_t toff[kSegOffCap];   // offsets of instances b0+1.. relative to the tile (the first kSegOffCap)
    __shared__ int s_cnt;                  // instances after b0 that start inside the tile (or right after it)
    __shared__ Seg wseg[NS * NW], wcarry[NS * NW];
    __shared__ Seg s_tail;
    __shared__ dev::WideLookbackSmem<Pair, NW> lbs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const dev::LookbackDesc d{words, words + 2 * ntiles};
    if (!*ok) return;   // rejected offsets (reported by the prep kernel)
    if (threadIdx.x == 0) {
        int64_t t;
        if (PART) t = ntiles - 1;
        else {
            t = atomicAdd(&ctl->ticket, 1u);
            if (t == (int64_t)gridDim.x - 1) ctl->ticket = 0u;   // the last ticket: every block has drawn
        }
        s_tile = t;
        const int64_t t0 = t * TILE;
        const int len0 = PART ? (int)(total - t0) : TILE;
        const int slen0 = len0 < SLEN ? len0 : SLEN;
        const uint32_t bytes = (uint32_t)(slen0 * 4) & ~15u;
#pragma unroll
        for (int c = 0; c < SUBS; ++c)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bars[c])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int c = 0; c < SUBS; ++c) {
            const uint32_t bb = smem_u32(&bars[c]), o = (uint32_t)c * 16384u;
            if (o >= bytes) {   // nothing staged in this chunk: complete its phase at once
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bb) : "memory");
                continue;
            }
            const uint32_t sz = bytes - o < 16384u ? bytes - o : 16384u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bb), "r"(sz) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(dyn + o)), "l"(reinterpret_cast<const unsigned char *>(values + t0) + o),
                            "r"(sz), "r"(bb)
                         : "memory");
        }
    }
    for (int i = threadIdx.x; i < TILE / 32 + 1; i += kBlock) heads[i] = 0u;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int64_t t = s_tile, t0 = t * TILE;
    const int64_t b0 = __ldg(tile_inst + t);
    const int len = PART ? (int)(total - t0) : TILE;
    const int slen = len < SLEN ? len : SLEN;
    const int whole = slen & ~3;
    const float *src = values + t0;
    // the register part first: its loads fly while the heads are laid out
    auto load4 = [&](int e) -> float4 {
        if (!PART || e + 3 < len) return dev::ld_stream(reinterpret_cast<const float4 *>(src + e));
        return make_float4(e < len ? src[e] : 0.f, e + 1 < len ? src[e + 1] : 0.f, e + 2 < len ? src[e + 2] : 0.f, 0.f);
    };
    float4 rv[SUBR][4];
#pragma unroll
    for (int r = 0; r < SUBR; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) rv[r][k] = load4(SLEN + r * kSubTile + w * 512 + k * 128 + lane * 4);
    // heads: the starts of the instances after b0 that begin inside the
    // tile, the start at element 0 if an instance begins there, and bit
    // `len` if an instance begins right after the tile (its last element
    // then ends an instance)
    {
        if (threadIdx.x == 0 && __ldg(off + b0) == t0) atomicOr(&heads[0], 1u);
        for (int64_t b = b0 + 1 + threadIdx.x; b <= B; b += kBlock) {
            const int64_t pos = __ldg(off + b) - t0;   // off[B] = total marks the array's end
            if (pos > len) break;                      // offsets are sorted: no later start lies in the tile
            atomicOr(&heads[pos >> 5], 1u << (pos & 31));
            if (RED) {
                const int64_t k = b - b0 - 1;
                if (k < kSegOffCap) toff[k] = (int32_t)pos;
                atomicMax(&s_cnt, (int)(k < kSegOffCap ? k + 1 : kSegOffCap + 1));
            }
        }
    }
    // the instance holding tile element e: b0 + the number of listed offsets
    // at or before e (a search in shared memory; beyond the list's capacity
    // a search of the offsets array from b0)
    auto inst_at = [&](int e) -> int64_t {
        const int cnt = s_cnt;
        if (cnt <= kSegOffCap) {
            int lo = 0, hi = cnt;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (toff[mid] <= e) lo = mid + 1;
                else hi = mid;
            }
            return b0 + lo;
        }
        int64_t lo = b0, hi = B - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(off + mid) <= t0 + e) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    auto head4 = [&](int e) -> uint32_t {   // head bits of elements e..e+4 (bit 4: the element after)
        const uint32_t w0 = heads[e >> 5], sh = e & 31;
        uint32_t v = w0 >> sh;
        if (sh > 27) v |= heads[(e >> 5) + 1] << (32 - sh);
        return v & 31u;
    };
    auto src4 = [&](int e) -> float4 {
        if (!PART || e + 3 < whole) return *reinterpret_cast<const float4 *>(buf + e);
        if (e >= slen) return make_float4(0.f, 0.f, 0.f, 0.f);
        return load4(e);   // the unstaged tail (fewer than 4 elements) is read directly
    };
    auto wait_chunk = [&](int c) -> bool {
        uint32_t done = 0;
        for (uint32_t k = 0; k < (1u << 22) && !done; ++k)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done) : "r"(smem_u32(&bars[c])) : "memory");
        if (__syncthreads_and(done)) return true;
        if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
        for (int cc = 0; cc < SUBS; ++cc) {
            uint32_t okk = 0;
            for (uint32_t k = 0; k < (1u << 22) && !okk; ++k)
                asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                             : "=r"(okk) : "r"(smem_u32(&bars[cc])) : "memory");
        }
        return false;
    };
    // one lane's four elements: their sums since the last head among them
    auto lane_seg = [&](const float4 &v, uint32_t hb) -> Seg {
        const float x[4] = {v.x, v.y, v.z, v.w};
        Seg a{0.f, 0.f, 0};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if ((hb >> i) & 1u) a = Seg{0.f, 0.f, 1};
            a.s += x[i];
            a.q = fmaf(x[i], x[i], a.q);
        }
        return a;
    };
    // A warp range holds no head and ends no instance (no head bit from its
    // first element through the element after its last): it is scanned as
    // a plain range, without per-element head tests.  Warp-uniform.
    auto head_free = [&](int j) -> bool {
        const int wb = (j * kSubTile + w * 512) >> 5;   // 16 words and one bit
        const uint32_t h = lane < 16 ? heads[wb + lane] : (lane == 16 ? heads[wb + 16] & 1u : 0u);
        return !__any_sync(0xffffffffu, h != 0u);
    };
    // pass 1: each warp range's segmented sums, in tile order
    auto range_seg = [&](int j, const float4 (&v)[4]) {
        if (head_free(j)) {
            float s = 0.f, q = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s += (v[k].x + v[k].y) + (v[k].z + v[k].w);
                if (RED) q = fmaf(v[k].x, v[k].x, fmaf(v[k].y, v[k].y, fmaf(v[k].z, v[k].z, fmaf(v[k].w, v[k].w, q))));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                if (RED) q += __shfl_xor_sync(0xffffffffu, q, o);
            }
            if (lane == 0) wseg[j * NW + w] = Seg{s, q, 0};
            return;
        }
        Seg c{0.f, 0.f, 0};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = j * kSubTile + w * 512 + k * 128 + lane * 4;
            const uint32_t hb = head4(e);
            if (!__any_sync(0xffffffffu, hb & 15u)) {   // no head among these 128 elements: plain sums
                float s = (v[k].x + v[k].y) + (v[k].z + v[k].w), q = 0.f;
                if (RED) q = fmaf(v[k].x, v[k].x, fmaf(v[k].y, v[k].y, fmaf(v[k].z, v[k].z, v[k].w * v[k].w)));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (RED) q += __shfl_xor_sync(0xffffffffu, q, o);
                }
                c.s += s;
                c.q += q;
                continue;
            }
            const Seg tot = warp_seg_scan(lane_seg(v[k], hb));
            const Seg last{__shfl_sync(0xffffffffu, tot.s, 31), __shfl_sync(0xffffffffu, tot.q, 31),
                           __shfl_sync(0xffffffffu, tot.h, 31)};
            c = seg_add(c, last);
        }
        if (lane == 0) wseg[j * NW + w] = c;
    };
    __syncthreads();   // the heads bitmap is complete
#pragma unroll
    for (int j = 0; j < SUBS; ++j) {
        if (!wait_chunk(j)) return;                             // block-uniform
        float4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = src4(j * kSubTile + w * 512 + k * 128 + lane * 4);
        range_seg(j, v);
    }
#pragma unroll
    for (int r = 0; r < SUBR; ++r) range_seg(SUBS + r, rv[r]);
    __syncthreads();
    if (w == 0) {   // exclusive segmented combine of the warp ranges in tile order, PER consecutive ones per lane
        Seg a[PER], tot{0.f, 0.f, 0};
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            a[i] = lane * PER + i < NS * NW ? wseg[lane * PER + i] : Seg{0.f, 0.f, 0};
            tot = seg_add(tot, a[i]);
        }
        const Seg inc = warp_seg_scan(tot);
        Seg ex{__shfl_up_sync(0xffffffffu, inc.s, 1), __shfl_up_sync(0xffffffffu, inc.q, 1),
               __shfl_up_sync(0xffffffffu, inc.h, 1)};
        if (lane == 0) ex = Seg{0.f, 0.f, 0};
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (lane * PER + i < NS * NW) wcarry[lane * PER + i] = ex;
            ex = seg_add(ex, a[i]);
        }
        if (lane == 31) s_tail = inc;
    }
    __syncthreads();
    const Seg tail = s_tail;
    const Pair tp((double)tail.s, (double)tail.q);
    const bool start_head = heads[0] & 1u;
    if (threadIdx.x == 0) {
        if (tail.h) dev::Codec<Pair>::put(d.incl + t * 2, tp, epoch);   // depends on no earlier tile
        else dev::Codec<Pair>::put(d.agg + t * 2, tp, epoch);
    }
    Pair p(0.0);
    if (!start_head) p = dev::wide_lookback<Pair, NW>(t, 0, tp, d, epoch, ctl, limit_ns, false, !tail.h, lbs);
    // pass 2
    auto scan_store = [&](int j, const float4 (&v)[4]) {
        Seg c = wcarry[j * NW + w];
        if (!c.h) {   // no head before this range in the tile: the running instance began in an earlier tile
            c.s = (float)(p.s + (double)c.s);
            c.q = (float)(p.q + (double)c.q);
        }
        if (head_free(j)) {   // a plain scan of the sums; no instance ends here, so no squares are needed
            if (!SCAN) return;
            // the four 128-element blocks' warp scans interleaved, then their carries chained
            float a[4], ab[4], abc[4], mine[4], inc[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = v[k].x;
                ab[k] = a[k] + v[k].y;
                abc[k] = ab[k] + v[k].z;
                mine[k] = abc[k] + v[k].w;
                inc[k] = mine[k];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float u = __shfl_up_sync(0xffffffffu, inc[k], o);
                    if (lane >= o) inc[k] += u;
                }
            }
            float base[4];
            base[0] = c.s;
#pragma unroll
            for (int k = 1; k < 4; ++k) base[k] = base[k - 1] + __shfl_sync(0xffffffffu, inc[k - 1], 31);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = j * kSubTile + w * 512 + k * 128 + lane * 4;
                const float run = base[k] + (inc[k] - mine[k]);
                const float4 o4 = INCL ? make_float4(run + a[k], run + ab[k], run + abc[k], run + mine[k])
                                       : make_float4(run, run + a[k], run + ab[k], run + abc[k]);
                if (!PART || e + 3 < len) {
                    dev::st_stream(reinterpret_cast<float4 *>(scan_out + t0 + e), o4);
                } else {
                    const float o[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (e + i < len) scan_out[t0 + e + i] = o[i];
                }
            }
            return;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = j * kSubTile + w * 512 + k * 128 + lane * 4;
            const uint32_t hb = head4(e);
            if (!__any_sync(0xffffffffu, hb)) {   // no head and no instance end among these 128: a plain scan
                if (SCAN) {
                    const float a = v[k].x, ab = a + v[k].y, abc = ab + v[k].z, mine = abc + v[k].w;
                    float inc = mine;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const float u = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += u;
                    }
                    const float run = c.s + (inc - mine);
                    const float4 o4 = INCL ? make_float4(run + a, run + ab, run + abc, run + mine)
                                           : make_float4(run, run + a, run + ab, run + abc);
                    if (!PART || e + 3 < len) {
                        dev::st_stream(reinterpret_cast<float4 *>(scan_out + t0 + e), o4);
                    } else {
                        const float o[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (e + i < len) scan_out[t0 + e + i] = o[i];
                    }
                    c.s += __shfl_sync(0xffffffffu, inc, 31);
                }
                if (RED) {   // the squares run on to an instance end later in the range
                    float q = fmaf(v[k].x, v[k].x, fmaf(v[k].y, v[k].y, fmaf(v[k].z, v[k].z, v[k].w * v[k].w)));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
                    c.q += q;
                }
                continue;
            }
            const Seg mine = lane_seg(v[k], hb);
            const Seg inc = warp_seg_scan(mine);
            Seg ex{__shfl_up_sync(0xffffffffu, inc.s, 1), __shfl_up_sync(0xffffffffu, inc.q, 1),
                   __shfl_up_sync(0xffffffffu, inc.h, 1)};
            if (lane == 0) ex = Seg{0.f, 0.f, 0};
            Seg run = seg_add(c, ex);   // the sums since the last head before this lane's elements
            const float x[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if ((hb >> i) & 1u) run = Seg{0.f, 0.f, 1};
                const float before = run.s;
                run.s += x[i];
                run.q = fmaf(x[i], x[i], run.q);
                o[i] = INCL ? run.s : before;
                // the last element of an instance: the next element starts one,
                // or the array ends here
                if (RED && e + i < len && (((hb >> (i + 1)) & 1u) || t0 + e + i == total - 1))
                    results[inst_at(e + i)] = run.q;
            }
            if (SCAN) {
                if (!PART || e + 3 < len) {
                    dev::st_stream(reinterpret_cast<float4 *>(scan_out + t0 + e), make_float4(o[0], o[1], o[2], o[3]));
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (e + i < len) scan_out[t0 + e + i] = o[i];
                }
            }
            const Seg last{__shfl_sync(0xffffffffu, inc.s, 31), __shfl_sync(0xffffffffu, inc.q, 31),
                           __shfl_sync(0xffffffffu, inc.h, 31)};
            c = seg_add(c, last);
        }
    };
#pragma unroll
    for (int j = 0; j < SUBS; ++j) {
        if (PART && j * kSubTile >= len) break;                 // block-uniform
        float4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = src4(j * kSubTile + w * 512 + k * 128 + lane * 4);
        scan_store(j, v);
    }
#pragma unroll
    for (int r = 0; r < SUBR; ++r) {
        if (PART && SLEN + r * kSubTile >= len) break;          // block-uniform
        scan_store(SUBS + r, rv[r]);
    }
}

// LB: how the look-back is walked -- 0 by warp 0 alone (variant 4), 1 by
// the whole block one predecessor per thread (variant 2), 2 by all warps in
// parallel windows after publishing the tile's aggregate early, from a
// pairwise sum taken right after the load (variants 0 and 1).
// words: 2 * max_t aggregate words, then 2 * max_t prefix words.
// Where tile t lives: its instance b = [lo, hi), the instance's first and
// last tiles, and the 16-byte aligned frame start.  t >= total: no tile.
struct TileInfo {
    int64_t t, b, lo, hi, first, last, fbase;
};

template <int TILE>
__device__ __forceinline__ TileInfo tile_info(int64_t t, int64_t total, const Layout &L,
                                              const int64_t *__restrict__ off)
{
    TileInfo x{t, 0, 0, 0, 0, 0, 0};
    if (t >= total) return x;
    x.b = L.tile_inst[t];
    x.lo = off[x.b];
    x.hi = off[x.b + 1];
    x.first = L.tile_start[x.b];
    x.last = L.tile_start[x.b + 1] - 1;
    x.fbase = (x.lo & ~(int64_t)3) + (t - x.first) * TILE;
    return x;
}

template <bool SCAN, bool RED, bool INCL, int V, int LB>
__global__ void __launch_bounds__(kBlock)
batched_main(const float *__restrict__ values, const int64_t *__restrict__ off, float *__restrict__ results,
             float *__restrict__ scan_out, Layout L, uint64_t *words, int64_t max_t, Control *ctl, uint32_t epoch,
             uint64_t limit_ns)
{
    constexpr int TILE = kBlock * 4 * V;
    __shared__ float smem[kBlock / 32 + 1];
    __shared__ float red_smem[32];
    __shared__ int64_t s_tile;
    __shared__ Pair s_prefix;
    __shared__ dev::BlockLookbackSmem<Pair, kBlock> lbs;
    __shared__ dev::WideLookbackSmem<Pair, kBlock / 32> wls;
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    const dev::LookbackDesc d{words, words + 2 * max_t};
    // A block draws its next ticket only when it is ready to work on it: a
    // ticket held while an earlier one is still processed would not publish
    // its aggregate in time, and the look-back walks of the tiles after it
    // would line up behind that block one after the other.
    while (true) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(&ctl->queue, 1u);
        __syncthreads();
        const TileInfo cur = tile_info<TILE>(s_tile, total, L, off);
        if (cur.t >= total) break;
        const int64_t t = cur.t, b = cur.b, lo = cur.lo, hi = cur.hi, first = cur.first, last = cur.last;
        const int64_t fbase = cur.fbase;
        const bool multi = first != last;   // block-uniform
        float v[V][4];
        load_masked<V>(values, fbase, lo, hi, v);
        Pair agg(0.0);
        if (LB == 2) {
            // pairwise per thread (rounding depth 2 + log2 V), then the block trees
            float ps[V], pq[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                ps[k] = (v[k][0] + v[k][1]) + (v[k][2] + v[k][3]);
                pq[k] = fmaf(v[k][0], v[k][0], v[k][1] * v[k][1]) + fmaf(v[k][2], v[k][2], v[k][3] * v[k][3]);
            }
#pragma unroll
            for (int st = 1; st < V; st *= 2)
#pragma unroll
                for (int i = 0; i + st < V; i += 2 * st) { ps[i] = ps[i] + ps[i + st]; pq[i] = pq[i] + pq[i + st]; }
            const float as = SCAN ? dev::block_reduce<dev::AddF, float, kBlock>(ps[0], red_smem) : 0.f;
            const float aq = RED ? dev::block_reduce<dev::AddF, float, kBlock>(pq[0], red_smem) : 0.f;
            agg = Pair((double)as, (double)aq);
            if (multi && threadIdx.x == 0) {
                if (t == first) dev::Codec<Pair>::put(d.incl + t * 2, agg, epoch);
                else dev::Codec<Pair>::put(d.agg + t * 2, agg, epoch);
            }
            if (SCAN) dev::tile_scan_local<float, INCL, kBlock, V>(v, smem);
        } else {
            float q = 0.f;
            if (RED) {
#pragma unroll
                for (int k = 0; k < V; ++k)
#pragma unroll
                    for (int j = 0; j < 4; ++j) q = fmaf(v[k][j], v[k][j], q);
                q = dev::block_reduce<dev::AddF, float, kBlock>(q, red_smem);
            }
            float sagg = 0.f;
            if (SCAN) sagg = dev::tile_scan_local<float, INCL, kBlock, V>(v, smem);
            agg = Pair((double)sagg, (double)q);
        }
        Pair p(0.0);
        if (multi) {
            if (LB == 2) {
                p = dev::wide_lookback<Pair, kBlock / 32>(t, first, agg, d, epoch, ctl, limit_ns, false, t != first, wls);
            } else if (LB == 1) {
                p = dev::block_lookback<Pair, kBlock>(t, first, agg, d, epoch, ctl, limit_ns, true, lbs);
            } else {
                if (threadIdx.x < 32) {
                    const Pair w = dev::lookback<Pair>(t, first, agg, d, epoch, ctl, limit_ns, true);
                    if (threadIdx.x == 0) s_prefix = w;
                }
                __syncthreads();
                p = s_prefix;
            }
        }
        if (RED && t == last && threadIdx.x == 0) results[b] = (float)(p.q + agg.q);
        if (SCAN) {
            dev::tile_add_prefix<float, V>(v, (float)p.s);
            store_masked<V>(scan_out, fbase, lo, hi, v);
        }
        __syncthreads();   // s_tile / s_prefix are rewritten by the next iteration
    }
    if (threadIdx.x == 0) {
        const uint32_t prev = atomicAdd(&ctl->exited, 1u);
        if (prev == gridDim.x - 1) {   // every block has drawn its last ticket
            ctl->queue = 0u;
            ctl->exited = 0u;
        }
    }
}

template <bool SCAN, bool RED, bool INCL, int V>
int run_main(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, const Layout &L,
             uint32_t epoch, int64_t max_t, cudaStream_t s)
{
    auto kern = c.variant == 2   ? batched_main<SCAN, RED, INCL, V, 1>
                : c.variant == 4 ? batched_main<SCAN, RED, INCL, V, 0>
                                 : batched_main<SCAN, RED, INCL, V, 2>;
    int64_t grid;
    if (c.variant == 1) {
        grid = max_t;
    } else {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, 0);
        if (occ < 1) occ = 1;
        grid = (int64_t)device_info().sms * occ;
        if (grid > max_t) grid = max_t;
    }
    if (grid < 1) grid = 1;
    if (grid > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many tiles");
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)grid, kBlock, 0, s, b.values, b.offsets, b.results, b.scan_out, L, words, max_t, ctl,
                  epoch, k.wait_limit_ns);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "batched launch");
}

template <int V>
int run_v(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
          uint32_t epoch, cudaStream_t s)
{
    constexpr int TILE = kBlock * 4 * V;
    const Layout L = layout(data, b, TILE);
    const int64_t mt = max_tiles(b, TILE);
    if (mt > 0x7fffffffLL || b.B > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many instances or tiles");
    launch_kernel(batched_prep, 1, 1024, 0, s, b.offsets, b.B, b.total, TILE, L, b.results, ctl, mt);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched prep launch");
    if (b.want_scan && b.want_reduce)
        return b.inclusive ? run_main<true, true, true, V>(b, c, ctl, words, L, epoch, mt, s)
                           : run_main<true, true, false, V>(b, c, ctl, words, L, epoch, mt, s);
    if (b.want_scan)
        return b.inclusive ? run_main<true, false, true, V>(b, c, ctl, words, L, epoch, mt, s)
                           : run_main<true, false, false, V>(b, c, ctl, words, L, epoch, mt, s);
    return run_main<false, true, true, V>(b, c, ctl, words, L, epoch, mt, s);
}

// variant 6 tile shapes (the config's tile index): sub-tiles staged in
// shared memory, sub-tiles held in registers, blocks per SM
constexpr int kSegShape[4][3] = {{6, 2, 2}, {6, 3, 2}, {6, 4, 2}, {4, 2, 3}};
constexpr int seg_tile(int shape) { return (kSegShape[shape][0] + kSegShape[shape][1]) * kSubTile; }

int tile_of(const Choice &c)
{
    if (c.variant == 3) return kBigTile;
    if (c.variant == 6) return seg_tile(c.tile >= 0 && c.tile < 4 ? c.tile : 0);
    if (c.variant == 7) return 4096;   // kBrTE
    return kBlock * 4 * (c.ept > 0 ? c.ept : 4);
}

template <bool SCAN, bool RED, bool INCL, int SH>
int run_seg_k(const BatchedLaunch &b, Control *ctl, uint64_t *words, const int *ok, const int64_t *tile_inst,
              uint32_t epoch, cudaStream_t s)
{
    constexpr int SUBS = kSegShape[SH][0], SUBR = kSegShape[SH][1], MINB = kSegShape[SH][2], TILE = seg_tile(SH);
    auto kfull = batched_seg<SCAN, RED, INCL, SUBS, SUBR, MINB, false>;
    auto kpart = batched_seg<SCAN, RED, INCL, SUBS, SUBR, MINB, true>;
    const int dyn = SUBS * kSubTile * (int)sizeof(float);
    cudaError_t ea = cudaFuncSetAttribute(kfull, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea == cudaSuccess) ea = cudaFuncSetAttribute(kpart, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea != cudaSuccess) return fail_cuda(ea, "batched segmented: shared memory opt-in");
    const int64_t ntiles = ceil_div(b.total, TILE), nfull = b.total / TILE;
    const DebugKnobs k = debug_knobs();
    if (nfull > 0)
        launch_kernel(kfull, (unsigned)nfull, kBlock, (size_t)dyn, s, b.values, b.offsets, b.B, b.total, b.results,
                      b.scan_out, ok, tile_inst, words, ntiles, ctl, epoch, k.wait_limit_ns);
    if (ntiles > nfull)   // the array's last, partial tile, after the whole ones
        launch_kernel(kpart, 1u, kBlock, (size_t)dyn, s, b.values, b.offsets, b.B, b.total, b.results, b.scan_out,
                      ok, tile_inst, words, ntiles, ctl, epoch, k.wait_limit_ns);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "batched segmented launch");
}

template <int SH>
int run_seg_shape(const BatchedLaunch &b, Control *ctl, uint64_t *words, const int *ok, const int64_t *tile_inst,
                  uint32_t epoch, cudaStream_t s)
{
    if (b.want_scan && b.want_reduce)
        return b.inclusive ? run_seg_k<true, true, true, SH>(b, ctl, words, ok, tile_inst, epoch, s)
                           : run_seg_k<true, true, false, SH>(b, ctl, words, ok, tile_inst, epoch, s);
    if (b.want_scan)
        return b.inclusive ? run_seg_k<true, false, true, SH>(b, ctl, words, ok, tile_inst, epoch, s)
                           : run_seg_k<true, false, false, SH>(b, ctl, words, ok, tile_inst, epoch, s);
    return run_seg_k<false, true, true, SH>(b, ctl, words, ok, tile_inst, epoch, s);
}

int run_seg(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
            uint32_t epoch, cudaStream_t s)
{
    if (c.ept > 0 && c.ept != 4) return fail(SKEL_ERR_INVALID_ARG, "batched segmented: ept must be 4");
    if (c.tile < 0 || c.tile > 3) return fail(SKEL_ERR_INVALID_ARG, "batched segmented: tile shape must be 0..3");
    const int tile = tile_of(c);
    if (ceil_div(b.total, tile) > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many tiles");
    int *ok = reinterpret_cast<int *>(data);
    int64_t *tile_inst = reinterpret_cast<int64_t *>(data + 256);
    launch_kernel(batched_seg_prep, 1, 1024, 0, s, b.offsets, b.B, b.total, tile, b.results, ok, tile_inst, ctl);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched segmented prep launch");
    if (b.total == 0) return SKEL_OK;
    switch (c.tile) {
    case 1: return run_seg_shape<1>(b, ctl, words, ok, tile_inst, epoch, s);
    case 2: return run_seg_shape<2>(b, ctl, words, ok, tile_inst, epoch, s);
    case 3: return run_seg_shape<3>(b, ctl, words, ok, tile_inst, epoch, s);
    default: return run_seg_shape<0>(b, ctl, words, ok, tile_inst, epoch, s);
    }
}

// ------------------- variant 7: flat segmented, aggregators and re-reading scanners --
// The flat segmented scan of variant 6 (one look-back pass over the
// concatenated values, restarting at instance starts) with the block layout
// of scan variant 8: one persistent block per SM whose
//   aggregator warps draw tile tickets in order, bulk-copy each 16 KiB tile
//     (and its 16-byte placement record) into a ring slot, sum the tile's
//     tail -- the elements from the start of the instance that holds its
//     last element, or the whole tile -- publish it (an inclusive prefix when
//     that instance starts inside the tile, else an aggregate), queue the
//     tile for the scanners and refill the slot at once;
//   scanner warps take one tile each, bulk-copy it again (from L2) into
//     their own buffer, mark the instance starts inside it in a bitmap, walk
//     the look-back when the tile continues an instance from an earlier
//     tile, then scan the buffer (restarting at instance starts), store it,
//     and write each instance's sum of squares at its last element.
// Each element is read from DRAM once (if the second read hits L2) and
// written once.  Progress, bounded waits and the ticket reset as in scan
// variant 8.
constexpr int kBrTE = 4096;    // elements per tile
constexpr int kBrAggW = 2;     // aggregator warps
constexpr int kBrQueue = 16;   // queue entries per block
constexpr int kBrOffCap = 64;  // instance offsets a scanner keeps per tile (more: searched in global memory)
constexpr int kBrBar = 1;      // named barrier of the aggregators
constexpr uint32_t kBrSleepNs = 20000;

struct __align__(16) BrMeta {
    int64_t b0;   // the instance holding the tile's first element
    int64_t hp;   // first element of the instance holding the tile's last element
};

__device__ __forceinline__ void br_sync(int nthreads) { asm volatile("bar.sync %0, %1;" :: "r"(kBrBar), "r"(nthreads) : "memory"); }
__device__ __forceinline__ bool br_and(int nthreads, bool p)
{
    uint32_t r;
    asm volatile("{ .reg .pred pi, po; setp.ne.u32 pi, %1, 0; bar.red.and.pred po, %2, %3, pi; selp.u32 %0, 1, 0, po; }"
                 : "=r"(r) : "r"((uint32_t)p), "r"(kBrBar), "r"(nthreads) : "memory");
    return r != 0;
}
__device__ __forceinline__ bool br_try(const uint64_t *bar, uint32_t par)
{
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(par), "r"(kBrSleepNs) : "memory");
    return done != 0;
}
__device__ __forceinline__ void br_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void br_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// A running float32 sum kept as an unevaluated pair hi + lo and advanced by
// an exact two-sum (Knuth's TwoSum): about 48 bits with float32 operations.
struct BrFF {
    float hi, lo;
    __device__ __forceinline__ float base() const { return hi + lo; }
    __device__ __forceinline__ void set(float v) { hi = v; lo = 0.f; }
    __device__ __forceinline__ void set(double v) { hi = (float)v; lo = (float)(v - (double)hi); }
    __device__ __forceinline__ void add(float v)
    {
        const float s = hi + v, bv = s - hi;
        lo += (hi - (s - bv)) + (v - bv);
        hi = s;
    }
};

// The non-empty instance holding element v: the largest b in [0, B) with
// off[b] <= v (sorted offsets; off[0] = 0 <= v < off[B]).
__device__ __forceinline__ int64_t br_instance_of(const int64_t *__restrict__ off, int64_t B, int64_t v)
{
    int64_t lo = 0, hi = B - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Each tile's placement, one thread per tile (unchecked offsets give
// placements the main kernel never reads: it stops at the check's flag).
__global__ void __launch_bounds__(256)
batched_br_meta(const int64_t *__restrict__ off, int64_t B, int64_t total, BrMeta *__restrict__ meta)
{
    const int64_t ntiles = (total + kBrTE - 1) / kBrTE;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t last = (t + 1) * kBrTE < total ? (t + 1) * kBrTE - 1 : total - 1;
        const int64_t b0 = br_instance_of(off, B, t * kBrTE), bl = br_instance_of(off, B, last);
        meta[t] = BrMeta{b0, __ldg(off + bl)};
    }
}

// Offsets check (as variant 6's).
__global__ void __launch_bounds__(1024)
batched_br_prep(const int64_t *__restrict__ off, int64_t B, int64_t total, float *__restrict__ results,
                int *__restrict__ ok, Control *ctl)
{
    __shared__ int bad;
    if (threadIdx.x == 0) bad = (off[0] != 0 || off[B] != total) ? 1 : 0;
    __syncthreads();
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const int64_t lo = off[b], hi = off[b + 1];
        if (hi < lo) bad = 1;
        else if (hi == lo && results) results[b] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *ok = bad ? 0 : 1;
        if (bad) atomicOr(&ctl->error, kErrInput);
    }
}

template <bool SCAN, bool RED, bool INCL, int R, int NC>
__global__ void __launch_bounds__((kBrAggW + NC) * 32, 1)
batched_br(const float *__restrict__ values, const int64_t *__restrict__ off, int64_t B, int64_t total,
           float *__restrict__ results, float *__restrict__ scan_out, const int *__restrict__ ok,
           const BrMeta *__restrict__ meta, dev::LookbackDesc d, Control *ctl, uint32_t epoch, int64_t skip_tile,
           uint64_t limit_ns)
{
    constexpr int TE = kBrTE, NA = kBrAggW, QC = kBrQueue, CAP = kBrOffCap;
    constexpr uint32_t TB = TE * 4;
    extern __shared__ __align__(1024) unsigned char dyn[];   // R ring slots, then one buffer per scanner warp
    __shared__ __align__(8) uint64_t ring_full[R], buf_full[NC];
    __shared__ BrMeta slot_meta[R];
    __shared__ int64_t slot_tile[R];
    __shared__ int64_t q_tile[QC], q_b0[QC];
    __shared__ Seg q_agg[QC];
    __shared__ float a_s[NA], a_q[NA];
    __shared__ uint32_t hbits[NC][TE / 32 + 1];   // per scanner: bit e = an instance starts at tile element e
    __shared__ int32_t toff[NC][CAP];             // per scanner: starts of instances b0+1.. relative to the tile
    __shared__ int q_tail, q_claim, q_read, a_done, s_stop;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t ntiles = (total + TE - 1) / TE, nfull = total / TE;
    if (!*ok) return;   // rejected offsets (reported by the prep kernel); every block leaves, no ticket drawn
    auto gave_up = [&]() { return dev::ld_volatile(&ctl->abort) == epoch; };
    auto give_up = [&]() {
        atomicOr(&ctl->error, kErrTimeout);
        atomicExch(&ctl->abort, epoch);
    };
    auto wait_phase = [&](const uint64_t *bar, uint32_t par) -> bool {
        const uint64_t t0 = dev::globaltimer();
        for (uint32_t k = 0; k < (1u << 26); ++k) {
            if (br_try(bar, par)) return true;
            if (gave_up() || dev::globaltimer() - t0 > limit_ns) return false;
        }
        return false;
    };
    if (threadIdx.x == 0) {
        q_tail = 0;
        q_claim = 0;
        q_read = 0;
        a_done = 0;
        s_stop = 0;
        for (int r = 0; r < R; ++r) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&ring_full[r])) : "memory");
        for (int r = 0; r < NC; ++r) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&buf_full[r])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (w < NA) {
        // ---------------------------------------------------------- aggregators
        auto start = [&](int slot, uint32_t t) {   // thread 0
            if (s_stop || (int64_t)t >= ntiles) {
                s_stop = 1;
                slot_tile[slot] = ntiles;
                return;
            }
            slot_tile[slot] = t;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const bool whole = (int64_t)t < nfull;   // the partial last tile is summed from global memory
            br_expect(&ring_full[slot], (whole ? TB : 0u) + (uint32_t)sizeof(BrMeta));
            br_copy(&slot_meta[slot], meta + t, (uint32_t)sizeof(BrMeta), &ring_full[slot]);
            if (whole) br_copy(dyn + slot * TB, values + t * (int64_t)TE, TB, &ring_full[slot]);
        };
        if (threadIdx.x == 0) {
            uint32_t first[R];
#pragma unroll
            for (int s = 0; s < R; ++s) first[s] = atomicAdd(&ctl->ticket, 1u);   // all in flight at once
#pragma unroll
            for (int s = 0; s < R; ++s) start(s, first[s]);
        }
        br_sync(NA * 32);
        for (int i = 0;; ++i) {
            const int slot = i % R;
            const uint32_t par = (uint32_t)(i / R) & 1u;
            const int64_t t = slot_tile[slot];
            if (t >= ntiles) break;   // uniform over the aggregators
            // the slot's next ticket, drawn now so that its round trip overlaps
            // the wait and the sum (drawn further ahead, a tile would be held
            // back while later tiles look back at it)
            uint32_t next = (uint32_t)ntiles;
            if (threadIdx.x == 0 && !s_stop) next = atomicAdd(&ctl->ticket, 1u);
            const bool done = wait_phase(&ring_full[slot], par);
            if (!br_and(NA * 32, done)) {   // a copy never landed
                if (threadIdx.x == 0) give_up();
                for (int j = 0; j < R; ++j) {   // drain every slot still waiting on a copy
                    if (slot_tile[j] >= ntiles) continue;
                    const uint32_t pj = (uint32_t)(i / R + (j < slot ? 1 : 0)) & 1u;
                    const uint64_t t0 = dev::globaltimer();
                    for (uint32_t k = 0; k < (1u << 26); ++k)
                        if (br_try(&ring_full[j], pj) || dev::globaltimer() - t0 > limit_ns) break;
                }
                break;
            }
            const int64_t t0 = t * TE;
            const BrMeta m = slot_meta[slot];
            const int hp = m.hp > t0 ? (int)(m.hp - t0) : 0;   // the tail starts here
            const bool head = m.hp >= t0;                         // ... at an instance start inside the tile
            // the tail's sums: four accumulators per thread, each over groups of four
            float as[4] = {0.f, 0.f, 0.f, 0.f}, aq[4] = {0.f, 0.f, 0.f, 0.f};
            constexpr int PER = TE / 4 / (NA * 32);   // groups of four per thread
            const float4 *src = reinterpret_cast<const float4 *>(dyn + slot * TB);
            if (t < nfull && hp == 0) {   // the whole tile (the usual case)
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const float4 v = src[k * NA * 32 + threadIdx.x];
                    as[k & 3] += (v.x + v.y) + (v.z + v.w);
                    if (RED) aq[k & 3] += fmaf(v.x, v.x, v.y * v.y) + fmaf(v.z, v.z, v.w * v.w);
                }
            } else if (t < nfull) {   // from element hp on
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int g = k * NA * 32 + threadIdx.x;
                    float4 v = src[g];
                    if (4 * g + 0 < hp) v.x = 0.f;
                    if (4 * g + 1 < hp) v.y = 0.f;
                    if (4 * g + 2 < hp) v.z = 0.f;
                    if (4 * g + 3 < hp) v.w = 0.f;
                    as[k & 3] += (v.x + v.y) + (v.z + v.w);
                    if (RED) aq[k & 3] += fmaf(v.x, v.x, v.y * v.y) + fmaf(v.z, v.z, v.w * v.w);
                }
            } else {
                const int len = (int)(total - t0);
                for (int k0 = 0; k0 * NA * 32 * 4 < len; k0 += 4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int e = ((k0 + j) * NA * 32 + threadIdx.x) * 4;
                        float x[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) x[u] = (e + u < len && e + u >= hp) ? values[t0 + e + u] : 0.f;
                        as[j] += (x[0] + x[1]) + (x[2] + x[3]);
                        if (RED) aq[j] += fmaf(x[0], x[0], x[1] * x[1]) + fmaf(x[2], x[2], x[3] * x[3]);
                    }
                }
            }
            float ss = (as[0] + as[1]) + (as[2] + as[3]), sq = (aq[0] + aq[1]) + (aq[2] + aq[3]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ss += __shfl_xor_sync(0xffffffffu, ss, o);
                if (RED) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            }
            if (lane == 0) {
                a_s[w] = ss;
                a_q[w] = sq;
            }
            br_sync(NA * 32);   // every read of the slot is done; the partial sums are visible
            if (threadIdx.x == 0) {
                float s = a_s[0], q = a_q[0];
#pragma unroll
                for (int j = 1; j < NA; ++j) {
                    s += a_s[j];
                    q += a_q[j];
                }
                const Pair tp((double)s, (double)q);
                if (t == skip_tile) {
                    // test hook: this tile never publishes
                } else if (head) dev::Codec<Pair>::put(d.incl + t * 2, tp, epoch);   // depends on no earlier tile
                else dev::Codec<Pair>::put(d.agg + t * 2, tp, epoch);
                const uint64_t w0 = dev::globaltimer();
                for (uint32_t k = 0; k < (1u << 26); ++k) {   // room in the queue (bounded)
                    if (q_tail - *(volatile int *)&q_read < QC) break;
                    if (gave_up() || dev::globaltimer() - w0 > limit_ns) break;
                    __nanosleep(64);
                }
                if (q_tail - *(volatile int *)&q_read < QC) {
                    q_tile[q_tail % QC] = t;
                    q_b0[q_tail % QC] = m.b0;
                    q_agg[q_tail % QC] = Seg{s, q, head ? 1 : 0};
                    __threadfence_block();
                    *(volatile int *)&q_tail = q_tail + 1;
                } else {
                    give_up();   // the tile is dropped; the call reports the timeout
                }
                start(slot, next);
            }
        }
        if (threadIdx.x == 0) {
            __threadfence_block();
            *(volatile int *)&a_done = 1;
            // the last block to stop drawing tickets resets the counter
            __threadfence();
            if (atomicAdd(&ctl->exited, 1u) == gridDim.x - 1) {
                ctl->ticket = 0u;
                ctl->exited = 0u;
            }
        }
        return;
    }
    // --------------------------------------------------------------- scanners
    const int cw = w - NA;
    unsigned char *buf = dyn + (R + cw) * TB;
    uint32_t *hb = hbits[cw];
    int32_t *to = toff[cw];
    uint32_t cpar = 0;
    while (true) {
        int k = 0, have = 0;
        if (lane == 0) {
            k = atomicAdd(&q_claim, 1);
            const uint64_t w0 = dev::globaltimer();
            for (uint32_t it = 0; it < (1u << 26); ++it) {
                const int dn = *(volatile int *)&a_done;
                __threadfence_block();
                if (k < *(volatile int *)&q_tail) { have = 1; break; }
                if (dn) break;
                if (dev::globaltimer() - w0 > 4 * limit_ns) { give_up(); break; }
                __nanosleep(64);
            }
        }
        if (!__shfl_sync(0xffffffffu, have, 0)) break;
        int64_t t = 0, b0 = 0;
        Seg agg{0.f, 0.f, 0};
        if (lane == 0) {
            __threadfence_block();
            t = q_tile[k % QC];
            b0 = q_b0[k % QC];
            agg = q_agg[k % QC];
            __threadfence_block();
            atomicAdd(&q_read, 1);
            if (t < nfull) {   // the tile again, into this warp's buffer
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                br_expect(&buf_full[cw], TB);
                br_copy(buf, values + t * (int64_t)TE, TB, &buf_full[cw]);
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&buf_full[cw])) : "memory");
            }
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        agg.s = __shfl_sync(0xffffffffu, agg.s, 0);
        agg.q = __shfl_sync(0xffffffffu, agg.q, 0);
        agg.h = __shfl_sync(0xffffffffu, agg.h, 0);
        const int64_t t0 = t * TE;
        const int len = (int)(total - t0 < TE ? total - t0 : TE);
        // the instance starts inside the tile (bit len: one starts right after
        // it, or the array ends there), and the first kBrOffCap of them listed
        for (int i = lane; i < TE / 32 + 1; i += 32) hb[i] = 0u;
        __syncwarp();
        const bool start_head = __ldg(off + b0) == t0;
        if (lane == 0 && start_head) atomicOr(&hb[0], 1u);
        int cnt = 0;   // instances after b0 that start in (0, len]
        for (int64_t b = b0 + 1 + lane;; b += 32) {
            const bool in = b <= B && __ldg(off + b) - t0 <= len;
            if (in) {
                const int pos = (int)(__ldg(off + b) - t0);
                atomicOr(&hb[pos >> 5], 1u << (pos & 31));
                const int64_t kk = b - b0 - 1;
                if (kk < CAP) to[kk] = pos;
                cnt = (int)(kk + 1);
            }
            if (!__any_sync(0xffffffffu, in)) break;   // offsets are sorted: the rest lie after the tile
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
        __syncwarp();
        // the prefix of the running instance: a look-back when it began in an earlier tile
        Pair p(0.0);
        if (!start_head) p = dev::lookback<Pair>(t, 0, Pair((double)agg.s, (double)agg.q), d, epoch, ctl, limit_ns, false);
        if (lane == 0 && !start_head && !agg.h && t != skip_tile)   // no instance starts here: its prefix runs on
            dev::Codec<Pair>::put(d.incl + t * 2, p + Pair((double)agg.s, (double)agg.q), epoch);
        const bool landed = __all_sync(0xffffffffu, wait_phase(&buf_full[cw], cpar));
        cpar ^= 1u;
        if (!landed) {
            if (lane == 0) give_up();
            const uint64_t w0 = dev::globaltimer();
            for (uint32_t it = 0; it < (1u << 26); ++it)
                if (br_try(&buf_full[cw], cpar ^ 1u) || dev::globaltimer() - w0 > limit_ns) break;
            break;
        }
        // the instance holding tile element e: b0 + the listed starts at or before e
        auto inst_at = [&](int e) -> int64_t {
            if (cnt <= CAP) {
                int lo = 0, hi = cnt;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (to[mid] <= e) lo = mid + 1;
                    else hi = mid;
                }
                return b0 + lo;
            }
            int64_t lo = b0, hi = B - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(off + mid) <= t0 + e) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        // does an instance end in the tile (a start in (0, len])?  Else no sum of squares is written here.
        bool ends = false;
        for (int i = lane; i < TE / 32 + 1; i += 32) ends |= (i == 0 ? (hb[0] & ~1u) : hb[i]) != 0u;
        ends = RED && __any_sync(0xffffffffu, ends);
        BrFF cs, cq;
        cs.set(p.s);
        cq.set(p.q);
        const float4 *src = reinterpret_cast<const float4 *>(buf);
        // one 128-element group, with or without instance starts and ends
        auto group = [&](int g) {
            const int e = g * 128 + 4 * lane;
            float4 v;
            if (t < nfull) v = src[g * 32 + lane];
            else {
                v.x = e < len ? values[t0 + e] : 0.f;
                v.y = e + 1 < len ? values[t0 + e + 1] : 0.f;
                v.z = e + 2 < len ? values[t0 + e + 2] : 0.f;
                v.w = e + 3 < len ? values[t0 + e + 3] : 0.f;
            }
            uint32_t h5;   // head bits of elements e..e+4
            {
                const uint32_t sh = e & 31;
                uint32_t x = hb[e >> 5] >> sh;
                if (sh > 27) x |= hb[(e >> 5) + 1] << (32 - sh);
                h5 = x & 31u;
            }
            if (!__any_sync(0xffffffffu, h5 != 0u)) {   // no start and no end among these 128: a plain scan
                const float a = v.x, ab = a + v.y, abc = ab + v.z, mine = abc + v.w;
                float inc = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float u = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += u;
                }
                if (SCAN) {
                    const float run = cs.base() + (inc - mine);
                    const float4 o4 = INCL ? make_float4(run + a, run + ab, run + abc, run + mine)
                                           : make_float4(run, run + a, run + ab, run + abc);
                    if (t < nfull) dev::st_stream(reinterpret_cast<float4 *>(scan_out + t0) + g * 32 + lane, o4);
                    else {
                        const float o[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (e + i < len) scan_out[t0 + e + i] = o[i];
                    }
                }
                cs.add(__shfl_sync(0xffffffffu, inc, 31));
                if (ends) {   // the squares run on to an instance end later in the tile
                    float q = fmaf(v.x, v.x, v.y * v.y) + fmaf(v.z, v.z, v.w * v.w);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
                    cq.add(q);
                }
                return;
            }
            // a start or an end among these 128: the segmented scan
            const float x[4] = {v.x, v.y, v.z, v.w};
            Seg mine{0.f, 0.f, 0};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if ((h5 >> i) & 1u) mine = Seg{0.f, 0.f, 1};
                mine.s += x[i];
                mine.q = fmaf(x[i], x[i], mine.q);
            }
            const Seg inc = warp_seg_scan(mine);
            Seg ex{__shfl_up_sync(0xffffffffu, inc.s, 1), __shfl_up_sync(0xffffffffu, inc.q, 1),
                   __shfl_up_sync(0xffffffffu, inc.h, 1)};
            if (lane == 0) ex = Seg{0.f, 0.f, 0};
            Seg run = seg_add(Seg{cs.base(), cq.base(), 0}, ex);   // the sums since the last start before this lane
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if ((h5 >> i) & 1u) run = Seg{0.f, 0.f, 1};
                const float before = run.s;
                run.s += x[i];
                run.q = fmaf(x[i], x[i], run.q);
                o[i] = INCL ? run.s : before;
                if (RED && e + i < len && ((h5 >> (i + 1)) & 1u)) results[inst_at(e + i)] = run.q;   // an instance's last element
            }
            if (SCAN) {
                if (t < nfull) dev::st_stream(reinterpret_cast<float4 *>(scan_out + t0) + g * 32 + lane, make_float4(o[0], o[1], o[2], o[3]));
                else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (e + i < len) scan_out[t0 + e + i] = o[i];
                }
            }
            const Seg last{__shfl_sync(0xffffffffu, inc.s, 31), __shfl_sync(0xffffffffu, inc.q, 31),
                           __shfl_sync(0xffffffffu, inc.h, 31)};
            if (last.h) {
                cs.set(last.s);
                cq.set(last.q);
            } else {
                cs.add(last.s);
                cq.add(last.q);
            }
                };
        // blocks of 512 elements: four interleaved warp scans when none of the
        // block's groups holds a start or an end, else group by group
#pragma unroll 1
        for (int g4 = 0; g4 * 512 < len; ++g4) {
            bool plain = t < nfull;
            if (plain) {
                const int w0 = (g4 * 512) >> 5;   // 16 words and the bit after the block
                const uint32_t hw = lane < 16 ? hb[w0 + lane] : (lane == 16 ? hb[w0 + 16] & 1u : 0u);
                plain = !__any_sync(0xffffffffu, hw != 0u);
            }
            if (!plain) {
                for (int g = 4 * g4; g < 4 * g4 + 4 && g * 128 < len; ++g) group(g);
                continue;
            }
            float4 v[4];
            float a[4], ab[4], abc[4], mine[4], inc[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[k] = src[(4 * g4 + k) * 32 + lane];
                a[k] = v[k].x;
                ab[k] = a[k] + v[k].y;
                abc[k] = ab[k] + v[k].z;
                mine[k] = abc[k] + v[k].w;
                inc[k] = mine[k];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float u = __shfl_up_sync(0xffffffffu, inc[k], o);
                    if (lane >= o) inc[k] += u;
                }
            const float base = cs.base();
            float loc = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (SCAN) {
                    const float run = base + (loc + (inc[k] - mine[k]));
                    const float4 o4 = INCL ? make_float4(run + a[k], run + ab[k], run + abc[k], run + mine[k])
                                           : make_float4(run, run + a[k], run + ab[k], run + abc[k]);
                    dev::st_stream(reinterpret_cast<float4 *>(scan_out + t0) + (4 * g4 + k) * 32 + lane, o4);
                }
                loc += __shfl_sync(0xffffffffu, inc[k], 31);
            }
            cs.add(loc);
            if (ends) {   // the squares run on to an instance end later in the tile
                float q = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) q += fmaf(v[k].x, v[k].x, v[k].y * v[k].y) + fmaf(v[k].z, v[k].z, v[k].w * v[k].w);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
                cq.add(q);
            }
        }
        __syncwarp();   // every read of the buffer and the bitmap is done before the next tile
    }
}

template <bool SCAN, bool RED, bool INCL, int R, int NC>
int run_br_k(const BatchedLaunch &b, Control *ctl, uint64_t *words, const int *ok, const BrMeta *meta,
             uint32_t epoch, cudaStream_t s)
{
    auto kern = batched_br<SCAN, RED, INCL, R, NC>;
    const int dyn = (R + NC) * kBrTE * 4, threads = (kBrAggW + NC) * 32;
    const int occ = kernel_occupancy(kern, threads, dyn);
    if (occ < 1) return fail(SKEL_ERR_UNSUPPORTED, "batched reread: kernel does not fit an SM");
    const int64_t ntiles = ceil_div(b.total, (int64_t)kBrTE);
    dev::LookbackDesc d{words, words + 2 * ntiles};
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)(device_info().sms * occ), threads, (size_t)dyn, s, b.values, b.offsets, b.B,
                  b.total, b.results, b.scan_out, ok, meta, d, ctl, epoch, k.scan_skip_publish_tile, k.wait_limit_ns);
    const cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "batched reread launch");
}

template <int R, int NC>
int run_br_shape(const BatchedLaunch &b, Control *ctl, uint64_t *words, const int *ok, const BrMeta *meta,
                 uint32_t epoch, cudaStream_t s)
{
    if (b.want_scan && b.want_reduce)
        return b.inclusive ? run_br_k<true, true, true, R, NC>(b, ctl, words, ok, meta, epoch, s)
                           : run_br_k<true, true, false, R, NC>(b, ctl, words, ok, meta, epoch, s);
    if (b.want_scan)
        return b.inclusive ? run_br_k<true, false, true, R, NC>(b, ctl, words, ok, meta, epoch, s)
                           : run_br_k<true, false, false, R, NC>(b, ctl, words, ok, meta, epoch, s);
    return run_br_k<false, true, true, R, NC>(b, ctl, words, ok, meta, epoch, s);
}

// tile: the ring's tiles and the scanner warps (16 KiB each): 0 = 6 + 6, 1 = 4 + 8.
int run_br(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
           uint32_t epoch, cudaStream_t s)
{
    if (c.ept > 0 && c.ept != 4) return fail(SKEL_ERR_INVALID_ARG, "batched reread: ept must be 4");
    if (c.tile < 0 || c.tile > 1) return fail(SKEL_ERR_INVALID_ARG, "batched reread: tile must be 0 or 1");
    const int64_t ntiles = ceil_div(b.total, (int64_t)kBrTE);
    if (ntiles > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many tiles");
    int *ok = reinterpret_cast<int *>(data);
    BrMeta *meta = reinterpret_cast<BrMeta *>(data + 256);
    launch_kernel(batched_br_prep, 1, 1024, 0, s, b.offsets, b.B, b.total, b.results, ok, ctl);
    if (b.total > 0) {
        const int64_t mgrid = std::min<int64_t>(ceil_div(ntiles, (int64_t)256), (int64_t)device_info().sms * 8);
        launch_kernel(batched_br_meta, (unsigned)mgrid, 256, 0, s, b.offsets, b.B, b.total, meta);
    }
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched reread prep launch");
    if (b.total == 0) return SKEL_OK;
    return c.tile ? run_br_shape<4, 8>(b, ctl, words, ok, meta, epoch, s)
                  : run_br_shape<6, 6>(b, ctl, words, ok, meta, epoch, s);
}

template <bool SCAN, bool RED, bool INCL>
int run_big_k(const BatchedLaunch &b, Control *ctl, uint64_t *words, const Layout &L, uint32_t epoch, int64_t max_t,
              cudaStream_t s)
{
    auto kern = batched_big<SCAN, RED, INCL>;
    const int dyn = kBigTile * (int)sizeof(float);
    cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea != cudaSuccess) return fail_cuda(ea, "batched big: shared memory opt-in");
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)max_t, kBlock, (size_t)dyn, s, b.values, b.offsets, b.results, b.scan_out, L, words,
                  max_t, b.total, ctl, epoch, k.wait_limit_ns);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "batched big launch");
}

int run_big(const BatchedLaunch &b, Control *ctl, uint64_t *words, unsigned char *data, uint32_t epoch,
            cudaStream_t s)
{
    const Layout L = layout(data, b, kBigTile);
    const int64_t mt = max_tiles(b, kBigTile);
    if (mt > 0x7fffffffLL || b.B > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many instances or tiles");
    launch_kernel(batched_prep, 1, 1024, 0, s, b.offsets, b.B, b.total, kBigTile, L, b.results, ctl, mt);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched prep launch");
    if (b.want_scan && b.want_reduce)
        return b.inclusive ? run_big_k<true, true, true>(b, ctl, words, L, epoch, mt, s)
                           : run_big_k<true, true, false>(b, ctl, words, L, epoch, mt, s);
    if (b.want_scan)
        return b.inclusive ? run_big_k<true, false, true>(b, ctl, words, L, epoch, mt, s)
                           : run_big_k<true, false, false>(b, ctl, words, L, epoch, mt, s);
    return run_big_k<false, true, true>(b, ctl, words, L, epoch, mt, s);
}

// ------------------------------------ variant 5: reduce-then-scan ----
// No look-back at all: (1) every tile's (sum, sum of squares), (2) per
// instance, the exclusive scan of its tile sums and the total of its sums of
// squares (one warp per instance, carried in float64), (3) every tile scanned
// locally and offset by its prefix.  The values are read twice (12 bytes per
// element with both outputs instead of 8), but no tile ever waits on another.
// Per-tile placement for the reduce-then-scan passes, computed once in
// parallel: one 32-byte load per tile there instead of three dependent ones
// (tile -> instance -> offsets), and its address is known a tile ahead.
struct __align__(16) TileMeta {
    int64_t fbase, lo, hi, pad;
};

template <int TILE>
__global__ void __launch_bounds__(kBlock)
batched_meta(const int64_t *__restrict__ off, Layout L, TileMeta *__restrict__ meta)
{
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    for (int64_t t = (int64_t)blockIdx.x * kBlock + threadIdx.x; t < total; t += (int64_t)gridDim.x * kBlock) {
        const TileInfo x = tile_info<TILE>(t, total, L, off);
        meta[t] = TileMeta{x.fbase, x.lo, x.hi, 0};
    }
}

__device__ __forceinline__ TileMeta load_meta(const TileMeta *meta, int64_t t)
{
    const longlong2 *p = reinterpret_cast<const longlong2 *>(meta + t);
    const longlong2 a = __ldg(p), b = __ldg(p + 1);
    return TileMeta{a.x, a.y, b.x, b.y};
}

template <bool SCAN, bool RED, int V>
__global__ void __launch_bounds__(kBlock)
batched_rts_sums(const float *__restrict__ values, const TileMeta *__restrict__ meta, Layout L, double *aggS,
                 double *aggQ)
{
    __shared__ float red[32];
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    TileMeta x = blockIdx.x < total ? load_meta(meta, blockIdx.x) : TileMeta{0, 0, 0, 0};
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {          // block-uniform
        const int64_t tn = t + gridDim.x;
        const TileMeta xn = tn < total ? load_meta(meta, tn) : x;       // the next tile's placement, in flight
        float v[V][4];
        load_masked<V>(values, x.fbase, x.lo, x.hi, v);
        float ps[V], pq[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            ps[k] = (v[k][0] + v[k][1]) + (v[k][2] + v[k][3]);
            pq[k] = fmaf(v[k][0], v[k][0], v[k][1] * v[k][1]) + fmaf(v[k][2], v[k][2], v[k][3] * v[k][3]);
        }
#pragma unroll
        for (int st = 1; st < V; st *= 2)
#pragma unroll
            for (int i = 0; i + st < V; i += 2 * st) { ps[i] = ps[i] + ps[i + st]; pq[i] = pq[i] + pq[i + st]; }
        const float as = SCAN ? dev::block_reduce<dev::AddF, float, kBlock>(ps[0], red) : 0.f;
        const float aq = RED ? dev::block_reduce<dev::AddF, float, kBlock>(pq[0], red) : 0.f;
        if (threadIdx.x == 0) {
            aggS[t] = (double)as;
            aggQ[t] = (double)aq;
        }
        x = xn;
    }
}

// One warp per instance: prefS[t] = sum of the instance's tile sums before
// t; results[b] = sum of its tiles' sums of squares.
__global__ void __launch_bounds__(kBlock)
batched_rts_prefix(Layout L, int64_t B, const double *__restrict__ aggS, const double *__restrict__ aggQ,
                   double *__restrict__ prefS, float *__restrict__ results, int scan, int red)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kBlock / 32);
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    if (total == 0) return;   // rejected offsets: nothing was laid out
    for (int64_t b = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); b < B; b += warps) {
        const int64_t s0 = L.tile_start[b], s1 = L.tile_start[b + 1];
        if (s1 <= s0) continue;                                   // empty: prep wrote its result
        double carry = 0.0, q = 0.0;
        for (int64_t k0 = s0; k0 < s1; k0 += 32) {
            const int64_t k = k0 + lane;
            const double a = (scan && k < s1) ? aggS[k] : 0.0;
            if (red && k < s1) q += aggQ[k];
            const double incl = dev::warp_incl_scan_add(a);
            if (scan && k < s1) prefS[k] = carry + (incl - a);
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (red) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
            if (lane == 0) results[b] = (float)q;
        }
    }
}

template <bool INCL, int V>
__global__ void __launch_bounds__(kBlock, V <= 4 ? 1 : 3)
batched_rts_apply(const float *__restrict__ values, const TileMeta *__restrict__ meta, float *__restrict__ scan_out,
                  Layout L, const double *__restrict__ prefS)
{
    __shared__ float smem[kBlock / 32 + 1];
    __shared__ float s_pre[2];
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    // last tiles first: the sums pass read the values in increasing order, so
    // its most recent tiles are still in L2 when this pass starts
    int par = 0;
    TileMeta x = blockIdx.x < total ? load_meta(meta, total - 1 - blockIdx.x) : TileMeta{0, 0, 0, 0};
    for (int64_t k = blockIdx.x; k < total; k += gridDim.x, par ^= 1) {   // block-uniform
        const int64_t t = total - 1 - k;
        const int64_t kn = k + gridDim.x;
        const TileMeta xn = kn < total ? load_meta(meta, total - 1 - kn) : x;   // next placement, in flight
        float v[V][4];
        load_masked<V>(values, x.fbase, x.lo, x.hi, v);
        // one float64 -> float32 conversion per tile, read after the scan's
        // barriers; two slots, so the next tile's write cannot overtake a read
        if (threadIdx.x == 0) s_pre[par] = (float)prefS[t];
        dev::tile_scan_local<float, INCL, kBlock, V>(v, smem);
        dev::tile_add_prefix<float, V>(v, s_pre[par]);
        store_masked<V>(scan_out, x.fbase, x.lo, x.hi, v);
        x = xn;
    }
}

template <int V>
int run_rts(const BatchedLaunch &b, Control *ctl, unsigned char *data, cudaStream_t s)
{
    constexpr int TILE = kBlock * 4 * V;
    const Layout L = layout(data, b, TILE);
    const int64_t mt = max_tiles(b, TILE);
    if (mt > 0x7fffffffLL || b.B > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many instances or tiles");
    double *aggS = reinterpret_cast<double *>(data + layout_bytes(b, TILE));
    double *aggQ = aggS + mt;
    double *prefS = aggQ + mt;
    // 16-byte loads of the placements: start them on a 256-byte boundary
    // (3 * 8 * mt bytes of float64 before them is only 8-byte aligned for odd mt)
    TileMeta *meta = reinterpret_cast<TileMeta *>(data + r256(layout_bytes(b, TILE) + 3 * 8 * (size_t)mt));
    launch_kernel(batched_prep, 1, 1024, 0, s, b.offsets, b.B, b.total, TILE, L, b.results, ctl, mt);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched prep launch");
    const int64_t mgrid = ceil_div(mt, kBlock) < 4096 ? ceil_div(mt, kBlock) : 4096;
    launch_kernel(batched_meta<TILE>, (unsigned)mgrid, kBlock, 0, s, b.offsets, L, meta);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched meta launch");
    int64_t grid = mt;
    const int64_t cap = (int64_t)device_info().sms * 64;
    if (grid > cap) grid = cap;
    const bool sc = b.want_scan, rd = b.want_reduce;
    if (sc && rd) launch_kernel(batched_rts_sums<true, true, V>, (unsigned)grid, kBlock, 0, s, b.values, meta, L, aggS, aggQ);
    else if (sc) launch_kernel(batched_rts_sums<true, false, V>, (unsigned)grid, kBlock, 0, s, b.values, meta, L, aggS, aggQ);
    else launch_kernel(batched_rts_sums<false, true, V>, (unsigned)grid, kBlock, 0, s, b.values, meta, L, aggS, aggQ);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched sums launch");
    const int64_t pgrid = ceil_div(b.B, kBlock / 32) < 4096 ? ceil_div(b.B, kBlock / 32) : 4096;
    launch_kernel(batched_rts_prefix, (unsigned)pgrid, kBlock, 0, s, L, b.B, aggS, aggQ, prefS, b.results, (int)sc,
                  (int)rd);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched prefix launch");
    if (!sc) return SKEL_OK;
    if (b.inclusive) launch_kernel(batched_rts_apply<true, V>, (unsigned)grid, kBlock, 0, s, b.values, meta, b.scan_out, L, prefS);
    else launch_kernel(batched_rts_apply<false, V>, (unsigned)grid, kBlock, 0, s, b.values, meta, b.scan_out, L, prefS);
    e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "batched apply launch");
}

}  // namespace

int batched_variant_count() { return 8; }
const char *batched_variant_name(int v)
{
    static const char *names[] = {"persistent", "one_per_tile", "persistent_block_lookback", "big_tile",
                                  "persistent_warp_lookback", "reduce_then_scan", "flat_segmented", "flat_reread"};
    return v >= 0 && v < 8 ? names[v] : "?";
}
Choice batched_default() { return Choice{5, 256, 8, 0}; }

size_t batched_data_bytes(const BatchedLaunch &b, const Choice &c)
{
    // the flat variant keeps a flag and each tile's first instance
    if (c.variant == 6) return 256 + 8 * (size_t)ceil_div(b.total, tile_of(c));
    // the re-reading variant: a flag and a 16-byte placement per tile
    if (c.variant == 7) return 256 + 16 * (size_t)ceil_div(b.total, tile_of(c));
    // reduce-then-scan also keeps three float64 values per tile and, from the
    // next 256-byte boundary, a 32-byte placement per tile
    if (c.variant != 5) return layout_bytes(b, tile_of(c));
    const size_t mt = (size_t)max_tiles(b, tile_of(c));
    return r256(layout_bytes(b, tile_of(c)) + 3 * 8 * mt) + 32 * mt;
}
// aggregate and prefix of every tile, two words (scan carry, sum of squares) each
size_t batched_word_count(const BatchedLaunch &b, const Choice &c) { return 4 * (size_t)max_tiles(b, tile_of(c)); }

int launch_batched(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
                   uint32_t epoch, cudaStream_t s)
{
    if (c.variant < 0 || c.variant > 7) return fail(SKEL_ERR_INVALID_ARG, "batched: unknown variant");
    if (c.block > 0 && c.block != kBlock) return fail(SKEL_ERR_INVALID_ARG, "batched: block must be 256");
    if (!aligned16(b.values) || (b.scan_out && !aligned16(b.scan_out)))
        return fail(SKEL_ERR_UNSUPPORTED, "batched: values and scan_out must be 16-byte aligned");
    if (b.B == 0) return SKEL_OK;
    if (c.variant == 3) {
        if (c.ept > 0 && c.ept != kBigV) return fail(SKEL_ERR_INVALID_ARG, "batched big: ept must be 4");
        return run_big(b, ctl, words, data, epoch, s);
    }
    if (c.variant == 6) return run_seg(b, c, ctl, words, data, epoch, s);
    if (c.variant == 7) return run_br(b, c, ctl, words, data, epoch, s);
    if (c.variant == 5) {
        switch (c.ept > 0 ? c.ept : 4) {
        case 4: return run_rts<4>(b, ctl, data, s);
        case 8: return run_rts<8>(b, ctl, data, s);
        default: return fail(SKEL_ERR_INVALID_ARG, "batched reduce-then-scan: ept must be 4 or 8");
        }
    }
    switch (c.ept > 0 ? c.ept : 4) {
    case 2: return run_v<2>(b, c, ctl, words, data, epoch, s);
    case 4: return run_v<4>(b, c, ctl, words, data, epoch, s);
    case 8: return run_v<8>(b, c, ctl, words, data, epoch, s);
    default: return fail(SKEL_ERR_INVALID_ARG, "batched: ept must be 2, 4 or 8");
    }
}

}  // namespace skel
