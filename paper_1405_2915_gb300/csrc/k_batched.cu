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
//             tiles of 96-160 KiB (staged partly in shared memory, partly
//             in registers) that restart at instance starts; a tile holding
//             a start publishes its tail at once, so look-back walks stop
//             there (one read);
//           7 flat_reread: the same flat segmented scan run by aggregator
//             warps (a ring of bulk copies) and re-reading scanner warps.
//           Variants 6 and 7 are in k_batched_seg.cu and k_batched_rr.cu.
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

int tile_of(const Choice &c)
{
    if (c.variant == 3) return kBigTile;
    if (c.variant == 6) return batched_seg_tile(c.tile);
    if (c.variant == 7) return 4096;   // the re-reading variant's tiles
    return kBlock * 4 * (c.ept > 0 ? c.ept : 4);
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
    // the flat variants: a flag and, per tile, its first instance (6) or a
    // 16-byte placement (7)
    if (c.variant == 6 || c.variant == 7)
        return 256 + (c.variant == 6 ? 8 : 16) * (size_t)ceil_div(b.total, (int64_t)tile_of(c));
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
    if (c.variant == 6) return batched_seg_launch(b, c, ctl, words, data, epoch, s);
    if (c.variant == 7) return batched_rr_launch(b, c, ctl, words, data, epoch, s);
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
