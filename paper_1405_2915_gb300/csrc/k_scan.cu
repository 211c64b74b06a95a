// Scan skeleton (Sec. III scan with (+)), inclusive or exclusive, over one
// sequence or over equal-length segments (rows of a 2D container), forward
// or reverse (the reverse scan is the adjoint of the scan).
//
// Variants:
//   0 reduce_then_scan  three kernels: per-tile sums -> per-segment scan of the
//                       tile sums -> tile scans plus their prefixes.  Reads the
//                       input twice (12 bytes per element for float32/int32).
//   1 lookback          single pass with decoupled look-back: tiles are taken
//                       in order from an atomic ticket (so a tile only ever
//                       waits on tiles already running), each publishes its
//                       aggregate, then its inclusive prefix, and finds its
//                       exclusive prefix by walking back over published
//                       predecessors.  8 bytes per element, the minimum.
//   2 one_block         one block walks the tiles in order with a carried
//                       prefix (small n: no inter-block traffic at all).
//   3 lookback_block    variant 1 with the whole block walking the look-back,
//                       one predecessor per thread (256 per round).
//   4 lookback_tma      persistent blocks, each with four tiles in flight in
//                       shared-memory stages filled by bulk copies
//                       (cp.async.bulk + mbarrier), so HBM reads continue
//                       while a block waits in its look-back; a tile's
//                       aggregate is published one iteration before it is
//                       scanned (forward scans, 16-byte aligned operands).
//   5 lookback_big      64 KiB tiles staged in shared memory by bulk copies,
//                       all warps walking the look-back; tile=1 publishes
//                       the aggregate before the in-place scans (16-byte
//                       aligned operands; reverse and row-wise scans need
//                       segments of a multiple of 4 elements).
//   7 lookback_hybrid   one block per tile staged partly in shared memory
//                       by bulk copies, partly in registers (tile=0: 96 + 64
//                       KiB, 3: 96 + 80 KiB, two blocks per SM; 1: 64 + 32
//                       KiB and 2: 64 + 48 KiB, three blocks per SM); warp
//                       totals first, the aggregate published at once, the
//                       look-back, then each warp scans and stores from its
//                       offset (same operand rules as variant 5).
//   8 lookback_reread   one persistent block per SM: aggregator warps
//                       stream tiles through a ring of bulk copies and
//                       publish their aggregates, scanner warps re-read
//                       each tile from L2 during its look-back (k_scan_rr.cu;
//                       same operand rules as variant 5).
//   6 lookback_ws       one persistent block per SM split into producer,
//                       scanner, look-back and store warps that pass tiles
//                       through a ring of staged tiles (tile=0: four 48 KiB
//                       stages, 1: six 32 KiB stages), so a tile's look-back
//                       overlaps the copies, scans and stores of its
//                       neighbours (same operand rules as variant 5).
// ept selects V, the 16-byte groups per thread (tile = 256 threads x 4V).
// float32: element arithmetic is float32; the prefix carried from tile to
// tile is float64 (one add per tile), rounded to float32 once per tile.
#include <type_traits>

#include "scan_tile.cuh"

namespace skel {
namespace {

using dev::LookbackDesc;
using dev::ScanTypes;
using dev::TileMap;

constexpr int kBlock = 256;

struct SegGeom {
    int64_t seglen;     // elements per segment
    int64_t tps;        // tiles per segment
    int64_t ntiles;     // total tiles
    bool rev;
    bool vec_ok;        // aligned pointers and segment length: full tiles may use 16-byte accesses
};

template <int TILE>
__device__ __forceinline__ TileMap tile_map(const SegGeom &g, int64_t tile, int64_t *first_tile)
{
    const int64_t s = tile / g.tps, ti = tile - s * g.tps;
    const int64_t e0 = ti * TILE;
    const int64_t seg0 = s * g.seglen;
    TileMap m;
    m.len = g.seglen - e0 < TILE ? g.seglen - e0 : TILE;
    m.rev = g.rev;
    m.base = g.rev ? seg0 + g.seglen - 1 - e0 : seg0 + e0;
    m.vec = g.vec_ok && m.len == TILE;
    *first_tile = s * g.tps;
    return m;
}

// BLK: the whole block walks the look-back (variant 3) instead of warp 0
// alone (variant 1).
template <class T, bool INCL, int V, bool BLK>
__global__ void __launch_bounds__(kBlock)
scan_lookback(const T *__restrict__ in, T *__restrict__ out, SegGeom g,
              LookbackDesc d, Control *ctl, uint32_t epoch,
              int64_t skip_tile, uint64_t limit_ns)
{
    using CT = typename ScanTypes<T>::CT;
    constexpr int TILE = kBlock * 4 * V;
    __shared__ T smem[kBlock / 32 + 1];
    __shared__ int64_t s_tile;
    __shared__ CT s_prefix;
    __shared__ dev::BlockLookbackSmem<CT, kBlock> lbs;
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(&ctl->ticket, 1u);
        if ((int64_t)t == g.ntiles - 1) ctl->ticket = 0u;   // the last ticket: every CTA has drawn
        s_tile = t;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    int64_t first;
    const TileMap m = tile_map<TILE>(g, tile, &first);
    T v[V][4];
    dev::tile_load<T, kBlock, V>(in, m, v);
    const T agg = dev::tile_scan_local<T, INCL, kBlock, V>(v, smem);
    CT p;
    if (BLK) {
        p = dev::block_lookback<CT, kBlock>(tile, first, (CT)agg, d, epoch, ctl, limit_ns, tile != skip_tile, lbs);
    } else {
        if (threadIdx.x < 32) {
            CT q = dev::lookback<CT>(tile, first, (CT)agg, d, epoch, ctl, limit_ns, tile != skip_tile);
            if (threadIdx.x == 0) s_prefix = q;
        }
        __syncthreads();
        p = s_prefix;
    }
    dev::tile_add_prefix<T, V>(v, dev::to_elem<T>(p));
    dev::tile_store<T, kBlock, V>(out, m, v);
}

// ------------------------------------------------ variant 4: TMA pipeline --
// A persistent block keeps kStages tiles in flight: thread 0 draws tickets in
// order and starts a bulk copy (cp.async.bulk, completing on the stage's
// mbarrier) of each drawn tile into a shared-memory stage.  Iteration i
// works on two tiles: it takes tile i+1 out of its stage into registers,
// refills that stage with a new ticket and publishes tile i+1's aggregate
// at once; then it scans tile i (already in registers), walks its
// look-back, adds the prefix and stores it.
//
// Publishing one tile ahead is what keeps the blocks independent.  A block
// that published a held tile's aggregate only when it came to scan it would
// make the next tile's look-back wait for the whole of its own previous
// tile, and that wait would chain through the blocks in ticket order,
// serialising them.  A block's current tile waits only on smaller tickets,
// each of which is already aggregated or is some block's current tile, so
// the smallest unfinished tile always progresses.
constexpr int kStages = 4;
constexpr int kTmaV = 4;
constexpr int kTmaTile = kBlock * 4 * kTmaV;             // 4096 elements = 16 KiB

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try(const uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return done;
}

// As mbar_try, but a thread whose phase is not complete is suspended until
// it completes or about hint_ns pass (instead of the short default limit),
// so waiting threads leave the shared-memory pipe and the issue slots to the
// warps that work.
__device__ __forceinline__ uint32_t mbar_try_sleep(const uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns) : "memory");
    return done;
}
constexpr uint32_t kSleepHintNs = 20000;   // 20 us per suspended try

// Thread 0: draws the next ticket for stage s and starts its copy.
template <class T>
__device__ __forceinline__ void tma_issue(const T *in, const SegGeom &g, Control *ctl, int s, unsigned char *bufs,
                                          uint64_t *bars, int64_t *tile_of)
{
    const int64_t t = (int64_t)atomicAdd(&ctl->ticket, 1u);
    tile_of[s] = t;
    if (t >= g.ntiles) return;
    int64_t first;
    const TileMap m = tile_map<kTmaTile>(g, t, &first);
    const uint32_t bytes = (uint32_t)((m.len * (int64_t)sizeof(T)) & ~(int64_t)15);   // whole 16-byte groups
    const uint32_t bar = smem_u32(bars + s);
    if (bytes == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
        return;
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(bufs + (size_t)s * kTmaTile * sizeof(T))), "l"(in + m.base), "r"(bytes), "r"(bar)
                 : "memory");
}

template <class T, bool INCL>
__global__ void __launch_bounds__(kBlock)
scan_tma(const T *__restrict__ in, T *__restrict__ out, SegGeom g, LookbackDesc d, Control *ctl, uint32_t epoch,
         int64_t skip_tile, uint64_t limit_ns)
{
    using CT = typename ScanTypes<T>::CT;
    using V4 = typename ScanTypes<T>::V4;
    using AddOp = typename std::conditional<std::is_same<T, float>::value, dev::AddF, dev::AddU>::type;
    constexpr int W = dev::Codec<CT>::W;
    extern __shared__ __align__(1024) unsigned char bufs[];   // kStages tiles
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ int64_t tile_of[kStages];
    __shared__ T smem[kBlock / 32 + 1];
    __shared__ T red[32];
    __shared__ dev::WideLookbackSmem<CT, kBlock / 32> lbs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(bars + s);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < kStages; ++s) tma_issue<T>(in, g, ctl, s, bufs, bars, tile_of);
    }
    __syncthreads();

    // Takes the tile of iteration i out of its stage: bounded wait for the
    // copy, a striped read into registers (conflict-free 16-byte reads),
    // the stage refilled with the next ticket, the aggregate published.
    // Returns false (block-uniform) when the wait ran out: the error is
    // recorded and the block waits (bounded) for its copies still landing.
    auto take = [&](uint32_t i, int64_t &tile, T (&v)[kTmaV][4], T &agg) -> bool {
        const int s = (int)(i % kStages);
        tile = tile_of[s];
        if (tile >= g.ntiles) return true;                  // block-uniform
        uint32_t done = 0;
        for (uint32_t k = 0; k < (1u << 22) && !done; ++k) done = mbar_try(bars + s, (i / kStages) & 1u);
        if (!__syncthreads_and(done)) {
            if (threadIdx.x == 0) {
                atomicOr(&ctl->error, kErrTimeout);
                for (uint32_t i2 = i + 1; i2 < i + kStages; ++i2) {
                    const int s2 = (int)(i2 % kStages);
                    if (tile_of[s2] >= g.ntiles) continue;
                    uint32_t ok = 0;
                    for (uint32_t k = 0; k < (1u << 22) && !ok; ++k) ok = mbar_try(bars + s2, (i2 / kStages) & 1u);
                }
            }
            return false;
        }
        int64_t first;
        const TileMap m = tile_map<kTmaTile>(g, tile, &first);
        const T *buf = reinterpret_cast<const T *>(bufs + (size_t)s * kTmaTile * sizeof(T));
        const int64_t whole = m.len & ~(int64_t)3;            // elements delivered by the copy
#pragma unroll
        for (int k = 0; k < kTmaV; ++k) {
            const int e = w * 128 * kTmaV + k * 128 + lane * 4;
            if (e + 3 < whole) {
                const V4 q = *reinterpret_cast<const V4 *>(buf + e);
                v[k][0] = q.x; v[k][1] = q.y; v[k][2] = q.z; v[k][3] = q.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    v[k][j] = e + j < whole ? buf[e + j] : (e + j < m.len ? in[m.base + e + j] : T(0));
            }
        }
        __syncthreads();                                      // the stage is consumed
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads before the async refill
            tma_issue<T>(in, g, ctl, s, bufs, bars, tile_of);
        }
        // aggregate: pairwise per thread (rounding depth 4), then the block trees
        T gs[kTmaV];
#pragma unroll
        for (int k = 0; k < kTmaV; ++k) gs[k] = (v[k][0] + v[k][1]) + (v[k][2] + v[k][3]);
        agg = dev::block_reduce<AddOp, T, kBlock>((gs[0] + gs[1]) + (gs[2] + gs[3]), red);
        if (threadIdx.x == 0 && tile != skip_tile) {
            if (tile == first) dev::Codec<CT>::put(d.incl + tile * W, (CT)agg, epoch);
            else dev::Codec<CT>::put(d.agg + tile * W, (CT)agg, epoch);
        }
        return true;
    };

    int64_t tile;
    T v[kTmaV][4];
    T agg;
    bool ok = take(0, tile, v, agg);
    for (uint32_t it = 0; ok && tile < g.ntiles; ++it) {     // block-uniform
        int64_t tile_n;
        T vn[kTmaV][4];
        T agg_n;
        ok = take(it + 1, tile_n, vn, agg_n);
        if (!ok) break;
        int64_t first;
        const TileMap m = tile_map<kTmaTile>(g, tile, &first);
        dev::tile_scan_local<T, INCL, kBlock, kTmaV>(v, smem);
        const CT p = dev::wide_lookback<CT, kBlock / 32>(tile, first, (CT)agg, d, epoch, ctl, limit_ns, false,
                                                         tile != skip_tile && tile != first, lbs);
        dev::tile_add_prefix<T, kTmaV>(v, dev::to_elem<T>(p));
        dev::tile_store<T, kBlock, kTmaV>(out, m, v);
        tile = tile_n;
        agg = agg_n;
#pragma unroll
        for (int k = 0; k < kTmaV; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) v[k][j] = vn[k][j];
    }
    // on the normal exit no copy is in flight: tickets are drawn in order, so
    // once a stage holds an invalid ticket every later stage does too
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t prev = atomicAdd(&ctl->exited, 1u);
        if (prev == gridDim.x - 1) {   // every block has drawn its last ticket
            ctl->ticket = 0u;
            ctl->exited = 0u;
        }
    }
}

// ------------------------------------------- variant 5: big staged tiles --
// One block per 64 KiB tile (four sub-tiles of 4096 elements), drawn in
// ticket order.  The tile arrives by bulk copies into shared memory; each
// sub-tile is scanned in place (registers -> shared memory, the same rounding
// depth as one 4096-element tile), the tile aggregate is published, the
// look-back is walked by all warps (one window of 32 each per round), and
// the prefix is added while the tile is stored.  Four times fewer tiles per
// byte than the 16 KiB tiles means a four times shorter look-back walk.

// EARLY publishes the tile aggregate before the in-place scans (one extra
// pass over the staged tile) so that successors stop waiting sooner;
// otherwise the aggregate follows the scans.  SUB sub-tiles of 16 KiB per
// tile: 64 KiB tiles fit three blocks per SM, 48 KiB tiles four, and the
// registers are capped so that all of them stay resident.
template <class T, bool INCL, bool REV, bool EARLY, int SUB>
__global__ void __launch_bounds__(kBlock, SUB == 4 ? 3 : 4)
scan_big(const T *__restrict__ in, T *__restrict__ out, SegGeom g, LookbackDesc d, Control *ctl, uint32_t epoch,
         int64_t skip_tile, uint64_t limit_ns)
{
    using CT = typename ScanTypes<T>::CT;
    using V4 = typename ScanTypes<T>::V4;
    extern __shared__ __align__(1024) unsigned char dyn[];   // (SUB * kTmaTile) elements
    T *buf = reinterpret_cast<T *>(dyn);
    __shared__ __align__(8) uint64_t bars[SUB];          // one per 16 KiB chunk
    __shared__ int64_t s_tile;
    __shared__ T smem[kBlock / 32 + 1];
    __shared__ dev::WideLookbackSmem<CT, kBlock / 32> lbs;
    __shared__ T red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(&ctl->ticket, 1u);
        if ((int64_t)t == g.ntiles - 1) ctl->ticket = 0u;   // the last ticket: every block has drawn
        s_tile = t;
#pragma unroll
        for (int c = 0; c < SUB; ++c) mbar_init(&bars[c]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        int64_t first0;
        const TileMap m0 = tile_map<SUB * kTmaTile>(g, t, &first0);
        // the tile's physical range: [base, base + len) forward, [base - len + 1, base] reverse
        const int64_t pstart = m0.rev ? m0.base - (m0.len - 1) : m0.base;
        const uint32_t bytes = (uint32_t)((m0.len * (int64_t)sizeof(T)) & ~(int64_t)15);
#pragma unroll
        for (int c = 0; c < SUB; ++c) {
            const uint32_t b = smem_u32(&bars[c]), o = (uint32_t)c * 16384u;
            if (o >= bytes) {   // nothing staged in this chunk: complete its phase at once
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
                continue;
            }
            const uint32_t sz = bytes - o < 16384u ? bytes - o : 16384u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(sz) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(dyn + o)), "l"(reinterpret_cast<const unsigned char *>(in + pstart) + o),
                            "r"(sz), "r"(b)
                         : "memory");
        }
    }
    __syncthreads();
    const int64_t tile = s_tile;
    int64_t first;
    const TileMap m = tile_map<SUB * kTmaTile>(g, tile, &first);
    // Bounded wait for chunks [c0, c1); block-uniform result.  On failure the
    // block records the timeout, waits (bounded) for every copy still landing
    // in its shared memory and leaves; the tile is never published, so its
    // successors' bounded waits give up too.
    auto wait_chunks = [&](int c0, int c1) -> bool {
        uint32_t ok = 1;
        for (int c = c0; c < c1; ++c) {
            uint32_t done = 0;
            for (uint32_t k = 0; k < (1u << 22) && !done; ++k)
                asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                             : "=r"(done) : "r"(smem_u32(&bars[c])) : "memory");
            ok &= done;
        }
        if (__syncthreads_and(ok)) return true;
        if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
        for (int c = 0; c < SUB; ++c) {
            uint32_t done = 0;
            for (uint32_t k = 0; k < (1u << 22) && !done; ++k)
                asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                             : "=r"(done) : "r"(smem_u32(&bars[c])) : "memory");
        }
        return false;
    };
    // Forward scans start on sub-tile j (its aggregate, or its in-place scan)
    // as soon as its chunk has landed; reverse scans wait for the whole tile.
    constexpr bool kProgressive = !REV;
    if (!kProgressive && !wait_chunks(0, SUB)) return;
    // Logical element e (scan order) sits at shared index e forward and
    // len-1-e reverse.  Reverse tiles have len % 4 == 0 (checked on the host),
    // so their groups of four are whole 16-byte vectors too.
    constexpr bool rev = REV;
    const int64_t len = m.len;
    const int64_t whole = len & ~(int64_t)3;   // staged elements
    auto src4 = [&](int64_t e, T (&a)[4]) {    // input values of logical e..e+3
        if (e + 3 < whole) {
            if (!rev) {
                const V4 q = *reinterpret_cast<const V4 *>(buf + e);
                a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
            } else {
                const V4 q = *reinterpret_cast<const V4 *>(buf + (len - 4 - e));
                a[0] = q.w; a[1] = q.z; a[2] = q.y; a[3] = q.x;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)   // the unstaged forward tail is read directly
                a[i] = e + i < whole ? buf[rev ? len - 1 - e - i : e + i] : (e + i < len ? in[m.base + e + i] : T(0));
        }
    };
    auto put4 = [&](int64_t e, const T (&a)[4]) {   // scanned values back into the same slots
        if (e + 3 < len) {
            V4 q;
            if (!rev) { q.x = a[0]; q.y = a[1]; q.z = a[2]; q.w = a[3]; *reinterpret_cast<V4 *>(buf + e) = q; }
            else { q.x = a[3]; q.y = a[2]; q.z = a[1]; q.w = a[0]; *reinterpret_cast<V4 *>(buf + (len - 4 - e)) = q; }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (e + i < len) buf[rev ? len - 1 - e - i : e + i] = a[i];
        }
    };
    auto get4 = [&](int64_t e, T (&a)[4]) {         // scanned values of logical e..e+3
        if (e + 3 < len) {
            if (!rev) {
                const V4 q = *reinterpret_cast<const V4 *>(buf + e);
                a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
            } else {
                const V4 q = *reinterpret_cast<const V4 *>(buf + (len - 4 - e));
                a[0] = q.w; a[1] = q.z; a[2] = q.y; a[3] = q.x;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = e + i < len ? buf[rev ? len - 1 - e - i : e + i] : T(0);
        }
    };
    // Early aggregate: pairwise sums of this thread's 16 groups, one sub-tile
    // at a time (float32 rounding depth 6), then the warp and block trees.
    // The first tile of a segment publishes its inclusive prefix (= the
    // aggregate) at once.
    const bool pub = tile != skip_tile;
    T tile_agg = T(0);
    if constexpr (EARLY) {
        using AddOp = typename std::conditional<std::is_same<T, float>::value, dev::AddF, dev::AddU>::type;
        T part[SUB];
#pragma unroll
        for (int j = 0; j < SUB; ++j) {
            if (kProgressive && !wait_chunks(j, j + 1)) return;   // block-uniform
            T gs[kTmaV];
#pragma unroll
            for (int k = 0; k < kTmaV; ++k) {
                T a[4];
                src4((int64_t)j * kTmaTile + w * 128 * kTmaV + k * 128 + lane * 4, a);
                gs[k] = (a[0] + a[1]) + (a[2] + a[3]);
            }
            part[j] = (gs[0] + gs[1]) + (gs[2] + gs[3]);
        }
#pragma unroll
        for (int st = 1; st < SUB; st *= 2)
#pragma unroll
            for (int i = 0; i + st < SUB; i += 2 * st) part[i] = part[i] + part[i + st];
        tile_agg = dev::block_reduce<AddOp, T, kBlock>(part[0], red);
        if (pub && threadIdx.x == 0) {
            constexpr int W = dev::Codec<CT>::W;
            if (tile == first) dev::Codec<CT>::put(d.incl + tile * W, (CT)tile_agg, epoch);
            else dev::Codec<CT>::put(d.agg + tile * W, (CT)tile_agg, epoch);
        }
    }
    // pass A: scan every sub-tile in place.  The carries between sub-tiles
    // are block-uniform and kept by thread 0 alone, in CT (a float64 add in
    // every thread would load the slow float64 pipe for nothing).
    __shared__ CT s_carry[SUB];
    __shared__ T s_pre[SUB];
    CT run = CT(0);                                          // meaningful in thread 0
#pragma unroll
    for (int j = 0; j < SUB; ++j) {
        if (threadIdx.x == 0) s_carry[j] = run;
        const int64_t off = (int64_t)j * kTmaTile;
        if (kProgressive && !EARLY && !wait_chunks(j, j + 1)) return;   // block-uniform
        if (off >= len) continue;                                       // block-uniform
        T v[kTmaV][4];
#pragma unroll
        for (int k = 0; k < kTmaV; ++k) src4(off + w * 128 * kTmaV + k * 128 + lane * 4, v[k]);
        const T agg = dev::tile_scan_local<T, INCL, kBlock, kTmaV>(v, smem);
#pragma unroll
        for (int k = 0; k < kTmaV; ++k) put4(off + w * 128 * kTmaV + k * 128 + lane * 4, v[k]);   // own slots
        if (threadIdx.x == 0) run = run + (CT)agg;
    }
    // EARLY: the aggregate is out already and the walk publishes the
    // inclusive prefix from that same value, so successors see one
    // consistent aggregate; otherwise the walk publishes both.
    const CT p = EARLY ? dev::wide_lookback<CT, kBlock / 32>(tile, first, (CT)tile_agg, d, epoch, ctl, limit_ns,
                                                             false, pub && tile != first, lbs)
                       : dev::wide_lookback<CT, kBlock / 32>(tile, first, run, d, epoch, ctl, limit_ns, pub, pub, lbs);
    // pass B: add the prefix and store, sub-tile by sub-tile
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < SUB; ++j) s_pre[j] = dev::to_elem<T>(p + s_carry[j]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SUB; ++j) {
        const int64_t off = (int64_t)j * kTmaTile;
        if (off >= len) continue;
        T v[kTmaV][4];
#pragma unroll
        for (int k = 0; k < kTmaV; ++k) get4(off + w * 128 * kTmaV + k * 128 + lane * 4, v[k]);
        dev::tile_add_prefix<T, kTmaV>(v, s_pre[j]);
        TileMap ms;
        ms.rev = rev;
        ms.base = rev ? m.base - off : m.base + off;
        ms.len = len - off < kTmaTile ? len - off : kTmaTile;
        ms.vec = ms.len == kTmaTile;
        dev::tile_store<T, kBlock, kTmaV>(out, ms, v);
    }
}

// ------------------------------------ variant 7: hybrid-staged tiles --
// One block per tile of (SUBS + SUBR) x 4096 elements, drawn in ticket
// order: the first SUBS sub-tiles arrive by bulk copies into shared memory,
// the last SUBR by 16-byte loads into registers (16 elements per thread
// each).  A tile waits in its look-back until every earlier tile's
// aggregate is out, in practice for the slowest load among the few hundred
// tiles in flight, so the scan's rate is set by how many bytes the SMs hold
// while their tiles wait; the registers add to what shared memory holds
// (three blocks of 64 KiB + 48 KiB hold 336 KiB per SM, against 192 KiB for
// four blocks of 48 KiB staged in shared memory alone).
//   pass 1: each warp sums its 512 elements of every sub-tile; one warp
//           scans those totals, which gives every warp its offset in the
//           tile and the tile aggregate, published at once;
//   look-back over the predecessors (all warps, a window of 32 each);
//   pass 2: each warp scans its elements with shuffles from its offset plus
//           the tile prefix and stores them (no shared-memory writes).
// Forward and reverse, 1D and per row (a reverse or row-wise scan needs
// segments of a multiple of 4 elements, like variant 5).  PART = false: the
// whole tiles, drawn in ticket order (tile = s * tps + ti, ti < tpsf); PART =
// true: a second launch, after the first on the same stream, for the last,
// partial tile of every segment (block s), whose predecessors are all out by
// then.  Keeping the ragged-tile logic out of the first kernel keeps its
// loops free of bounds checks and its registers below the three-blocks-per-
// SM limit.
template <class T, bool INCL, bool REV, int SUBS, int SUBR, int MINB, bool PART>
__global__ void __launch_bounds__(kBlock, MINB)
scan_hybrid(const T *__restrict__ in, T *__restrict__ out, SegGeom g, int64_t tpsf, LookbackDesc d, Control *ctl,
            uint32_t epoch, int64_t skip_tile, uint64_t limit_ns)
{
    using CT = typename ScanTypes<T>::CT;
    using V4 = typename ScanTypes<T>::V4;
    using AddOp = typename std::conditional<std::is_same<T, float>::value, dev::AddF, dev::AddU>::type;
    constexpr int NW = kBlock / 32, NS = SUBS + SUBR, TILE = NS * kTmaTile, SLEN = SUBS * kTmaTile;
    static_assert(NS * NW <= 96, "one warp scans at most 96 warp totals");
    extern __shared__ __align__(1024) unsigned char dyn[];   // SUBS * 16 KiB
    const T *buf = reinterpret_cast<const T *>(dyn);
    __shared__ __align__(8) uint64_t bars[SUBS];
    __shared__ int64_t s_tile;
    __shared__ T wtot[NS * NW], wex[NS * NW];
    __shared__ T s_agg;
    __shared__ dev::WideLookbackSmem<CT, NW> lbs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // tile -> (segment, index in it) and its placement
    auto place = [&](int64_t t, int64_t &seg, int64_t &ti, int64_t &base, int &len) {
        if (PART) { seg = t; ti = tpsf; }
        else { seg = t / tpsf; ti = t - seg * tpsf; }
        const int64_t e0 = ti * TILE, seg0 = seg * g.seglen;
        len = PART ? (int)(g.seglen - e0) : TILE;
        base = REV ? seg0 + g.seglen - 1 - e0 : seg0 + e0;
    };
    if (threadIdx.x == 0) {
        int64_t t;
        if (PART) t = blockIdx.x;
        else {
            t = atomicAdd(&ctl->ticket, 1u);
            if (t == (int64_t)gridDim.x - 1) ctl->ticket = 0u;   // the last ticket: every block has drawn
        }
        s_tile = t;
#pragma unroll
        for (int c = 0; c < SUBS; ++c) mbar_init(&bars[c]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        int64_t seg0, ti0, base0;
        int len0;
        place(t, seg0, ti0, base0, len0);
        const int slen0 = len0 < SLEN ? len0 : SLEN;
        // staged physical range: [base, base + slen) forward, [base - slen + 1, base] reverse
        const int64_t pstart = REV ? base0 - (slen0 - 1) : base0;
        const uint32_t bytes = (uint32_t)(slen0 * (int)sizeof(T)) & ~15u;
#pragma unroll
        for (int c = 0; c < SUBS; ++c) {
            const uint32_t b = smem_u32(&bars[c]), o = (uint32_t)c * 16384u;
            if (o >= bytes) {   // nothing staged in this chunk: complete its phase at once
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
                continue;
            }
            const uint32_t sz = bytes - o < 16384u ? bytes - o : 16384u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(sz) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(dyn + o)), "l"(reinterpret_cast<const unsigned char *>(in + pstart) + o),
                            "r"(sz), "r"(b)
                         : "memory");
        }
    }
    __syncthreads();
    int64_t segi, ti, mbase;
    int len;
    place(s_tile, segi, ti, mbase, len);
    const int64_t first = segi * g.tps, tile = first + ti;
    // offsets inside the tile fit in 32 bits; the operands are 16-byte
    // aligned and tiles start on multiples of 4 elements, so every group of
    // four that lies inside the tile is one aligned 16-byte access
    const int slen = len < SLEN ? len : SLEN;
    const int whole = slen & ~3;   // staged elements (reverse: slen % 4 == 0, all staged)
    const T *src = in + mbase;     // logical e at src[e] forward, src[-e] reverse
    T *dst = out + mbase;
    auto load4 = [&](const T *p0, int e) -> V4 {   // logical e..e+3 from global memory
        V4 q;
        if (!PART || e + 3 < len) {
            if (!REV) q = dev::ld_stream(reinterpret_cast<const V4 *>(p0 + e));
            else {
                const V4 r4 = dev::ld_stream(reinterpret_cast<const V4 *>(p0 - e - 3));
                q.x = r4.w; q.y = r4.z; q.z = r4.y; q.w = r4.x;
            }
        } else {   // the last, partial group of a forward 1D scan
            q.x = e < len ? p0[e] : T(0);
            q.y = e + 1 < len ? p0[e + 1] : T(0);
            q.z = e + 2 < len ? p0[e + 2] : T(0);
            q.w = T(0);
        }
        return q;
    };
    // the register sub-tiles: logical elements SLEN + r * 4096 + w * 512 + k * 128 + lane * 4 + i
    V4 rv[SUBR][4];
#pragma unroll
    for (int r = 0; r < SUBR; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) rv[r][k] = load4(src, SLEN + r * kTmaTile + w * 512 + k * 128 + lane * 4);
    // input values of logical e..e+3 of the shared-memory part
    auto src4 = [&](int e) -> V4 {
        if (!PART || e + 3 < whole) {
            if (!REV) return *reinterpret_cast<const V4 *>(buf + e);
            const V4 r4 = *reinterpret_cast<const V4 *>(buf + (slen - 4 - e));
            V4 q;
            q.x = r4.w; q.y = r4.z; q.z = r4.y; q.w = r4.x;
            return q;
        }
        if (e >= slen) return V4{T(0), T(0), T(0), T(0)};
        return load4(src, e);   // the unstaged forward tail (fewer than 4 elements) is read directly
    };
    // Bounded wait for chunk c; block-uniform.  On failure the block records
    // the timeout, waits (bounded) for every copy still landing in its
    // shared memory and leaves; its tile is never published, so its
    // successors' bounded waits give up too.
    auto wait_chunk = [&](int c) -> bool {
        uint32_t done = 0;
        for (uint32_t k = 0; k < (1u << 22) && !done; ++k) done = mbar_try(&bars[c], 0);
        if (__syncthreads_and(done)) return true;
        if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
        for (int cc = 0; cc < SUBS; ++cc) {
            uint32_t dd = 0;
            for (uint32_t k = 0; k < (1u << 22) && !dd; ++k) dd = mbar_try(&bars[cc], 0);
        }
        return false;
    };
    // pass 1: warp totals of every sub-tile.  Forward, logical sub-tile j is
    // staged chunk j, so it starts as soon as that chunk has landed; reverse,
    // the logical order runs backwards through the staged range, so every
    // chunk is awaited first.
    if (REV) {
#pragma unroll
        for (int j = 0; j < SUBS; ++j)
            if (!wait_chunk(j)) return;
    }
#pragma unroll
    for (int j = 0; j < SUBS; ++j) {
        if (!REV && !wait_chunk(j)) return;
        T gs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const V4 q = src4(j * kTmaTile + w * 512 + k * 128 + lane * 4);
            gs[k] = (q.x + q.y) + (q.z + q.w);
        }
        const T s = dev::warp_reduce<AddOp>((gs[0] + gs[1]) + (gs[2] + gs[3]));
        if (lane == 0) wtot[j * NW + w] = s;
    }
#pragma unroll
    for (int r = 0; r < SUBR; ++r) {
        T gs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) gs[k] = (rv[r][k].x + rv[r][k].y) + (rv[r][k].z + rv[r][k].w);
        const T s = dev::warp_reduce<AddOp>((gs[0] + gs[1]) + (gs[2] + gs[3]));
        if (lane == 0) wtot[(SUBS + r) * NW + w] = s;
    }
    __syncthreads();
    if (w == 0) {   // exclusive scan of the warp totals in tile order, PL per lane
        constexpr int PL = (NS * NW + 31) / 32;
        T a[PL];
        T sum = T(0);
#pragma unroll
        for (int i = 0; i < PL; ++i) {
            a[i] = PL * lane + i < NS * NW ? wtot[PL * lane + i] : T(0);
            sum = sum + a[i];
        }
        const T inc = dev::warp_incl_scan_add(sum);
        T ex = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) ex = T(0);
#pragma unroll
        for (int i = 0; i < PL; ++i) {
            if (PL * lane + i < NS * NW) wex[PL * lane + i] = ex;
            ex = ex + a[i];
        }
        if (lane == 31) s_agg = inc;
    }
    __syncthreads();
    {
        const T agg = s_agg;
        const bool pub = tile != skip_tile;
        if (pub && threadIdx.x == 0) {
            constexpr int W = dev::Codec<CT>::W;
            if (tile == first) dev::Codec<CT>::put(d.incl + tile * W, (CT)agg, epoch);
            else dev::Codec<CT>::put(d.agg + tile * W, (CT)agg, epoch);
        }
        const CT p = dev::wide_lookback<CT, NW>(tile, first, (CT)agg, d, epoch, ctl, limit_ns, false,
                                                pub && tile != first, lbs);
        // this warp's base of every sub-tile: the tile prefix plus its offset
        if (lane < NS) wtot[lane * NW + w] = dev::to_elem<T>(p + (CT)wex[lane * NW + w]);
        __syncwarp();
    }
    // pass 2: scan each warp's elements from its base and store them
    auto scan_store = [&](int j, const V4 (&v)[4]) {
        const T base = wtot[j * NW + w];
        T carry = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = j * kTmaTile + w * 512 + k * 128 + lane * 4;
            const T s0 = v[k].x, s1 = s0 + v[k].y, s2 = s1 + v[k].z, s3 = s2 + v[k].w;
            const T wi = dev::warp_incl_scan_add(s3);
            T lex = __shfl_up_sync(0xffffffffu, wi, 1);
            if (lane == 0) lex = T(0);
            const T wt = __shfl_sync(0xffffffffu, wi, 31);
            const T b = base + (carry + lex);
            V4 o;
            if (INCL) { o.x = b + s0; o.y = b + s1; o.z = b + s2; o.w = b + s3; }
            else { o.x = b; o.y = b + s0; o.z = b + s1; o.w = b + s2; }
            if (!PART || e + 3 < len) {
                if (!REV) dev::st_stream(reinterpret_cast<V4 *>(dst + e), o);
                else {
                    V4 r4;
                    r4.x = o.w; r4.y = o.z; r4.z = o.y; r4.w = o.x;
                    dev::st_stream(reinterpret_cast<V4 *>(dst - e - 3), r4);
                }
            } else {   // the last, partial group of a forward 1D scan
                if (e < len) dst[e] = o.x;
                if (e + 1 < len) dst[e + 1] = o.y;
                if (e + 2 < len) dst[e + 2] = o.z;
            }
            carry = carry + wt;
        }
    };
#pragma unroll
    for (int j = 0; j < SUBS; ++j) {
        if (PART && j * kTmaTile >= len) break;   // block-uniform
        V4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = src4(j * kTmaTile + w * 512 + k * 128 + lane * 4);
        scan_store(j, v);
    }
#pragma unroll
    for (int r = 0; r < SUBR; ++r) {
        if (PART && SLEN + r * kTmaTile >= len) break;   // block-uniform
        scan_store(SUBS + r, rv[r]);
    }
}

// ------------------------------------ variant 6: warp-specialised stages --
// One persistent block per SM whose warps split into four roles; a tile
// moves through them in a ring of shared-memory stages, each hand-over an
// mbarrier phase:
//   producer  (warp 0, one thread): draws tickets in order and starts the bulk
//             copies of each drawn tile into the next free stage (full[s]);
//   reducers  (4 warps): sum the tile's eight chunks, publish the tile
//             aggregate at once (reduced[s]);
//   look-back (8 warps): walk the tile's predecessors, 512 per round, publish
//             its inclusive prefix and give each chunk its prefix
//             (prefixed[s]);
//   scanners  (8 warps, one chunk each): scan the chunk with warp scans in
//             registers, add the prefix and store it, then free the stage
//             (empty[s]).
// A block that runs the phases one after another (variant 5) holds each tile
// through its look-back round trip and its stores while no copy is in
// flight.  Here the look-back of tile i overlaps the reduction of tile i+1,
// the scans and stores of tile i-1 and the copies of the tiles after them.
// The scan itself needs no block barrier: a chunk's prefix (the tile prefix
// plus the sums of the chunks before it) is known before its warp starts.
//
// The look-back rounds are twice as wide as variant 5's because the blocks
// move in step: the predecessors drawn in the same round of tickets (one per
// block) are still walking, and their inclusive prefixes appear about when
// this walk starts; 512 predecessors reach back past them to tiles published
// a whole period earlier, so a walk usually ends after one round trip.
//
// Progress: tickets are drawn in order and every role takes its block's
// tiles in that order, so the smallest unfinished tile has all of its
// predecessors finished and each of its roles free to take it.  Every wait
// is bounded (globaltimer); a wait that runs out records kErrTimeout and
// sets the block's abort word, which ends the other roles' waits; before
// the block leaves, the producer waits (bounded) for each copy it issued.
constexpr int kWsRedW = 4, kWsLookW = 8, kWsScanW = 8;
constexpr int kWsThreads = 32 * (1 + kWsRedW + kWsLookW + kWsScanW);   // 672
constexpr int kWsChunks = kWsScanW;                                    // chunks per tile
constexpr int kWsLookE = 2;                                            // windows per look-back lane
constexpr int kWsBarRed = 1, kWsBarLook = 2, kWsBarScan = 3;           // named barriers (0: __syncthreads)

__device__ __forceinline__ void mbar_init_count(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}
// Barrier over one role's threads that also ANDs a predicate across them.
__device__ __forceinline__ bool group_and(int id, int nthreads, bool p)
{
    uint32_t r;
    asm volatile("{ .reg .pred pi, po; setp.ne.u32 pi, %1, 0; bar.red.and.pred po, %2, %3, pi; selp.u32 %0, 1, 0, po; }"
                 : "=r"(r) : "r"((uint32_t)p), "r"(id), "r"(nthreads) : "memory");
    return r != 0;
}

// Bounded wait for the phase of parity par; false when it ran out or the
// block's abort word was set.
__device__ __forceinline__ bool ws_wait(const uint64_t *bar, uint32_t par, const volatile int *abort_word,
                                        uint64_t limit_ns)
{
    const uint64_t t0 = dev::globaltimer();
    for (uint32_t k = 0; k < (1u << 26); ++k) {
        if (mbar_try_sleep(bar, par, kSleepHintNs)) return true;
        if (*abort_word || dev::globaltimer() - t0 > limit_ns) return false;
    }
    return false;
}

// The wide look-back walk run by one role of NW warps, each lane polling NE
// predecessors per round: window k (k = w + NW*e, 32 predecessors) holds
// pred - 32k - lane, so the windows are numbered by distance.  A warp polls
// until its windows are ready up to its nearest inclusive prefix; warp 0
// then adds windows 0..kmax (kmax: the nearest window holding a published
// prefix).  The aggregate (and a segment's first inclusive prefix) was
// published by the reducers.
template <class CT, int NW, int NE>
__device__ __forceinline__ CT group_lookback(int64_t tile, int64_t first, CT agg, LookbackDesc d, uint32_t epoch,
                                             Control *ctl, uint64_t limit_ns, bool pub_incl,
                                             dev::WideLookbackSmem<CT, NW * NE> &sm, int w, int lane, int id)
{
    constexpr int W = dev::Codec<CT>::W;
    if (tile == first) return CT(0);
    CT excl = CT(0);
    int64_t pred = tile - 1;
    uint64_t t0 = 0;
    bool gave_up = false;
    while (true) {
        uint32_t status[NE];
        unsigned incl_mask[NE];
        CT val[NE];
        while (true) {
            bool ok = true, seen_incl = false;
            // every poll of the round is in flight before any is looked at
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int64_t p = pred - 32 * (w + NW * e) - lane;
                if (p >= first) status[e] = dev::peek<CT>(d, p, epoch, val[e]);
                else { status[e] = dev::kStIncl; val[e] = CT(0); }   // before the segment start: prefix 0
            }
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const unsigned ready_mask = __ballot_sync(0xffffffffu, status[e] != 0);
                incl_mask[e] = __ballot_sync(0xffffffffu, status[e] == dev::kStIncl);
                const unsigned need = incl_mask[e] ? (((incl_mask[e] & (0u - incl_mask[e])) << 1) - 1u) : 0xffffffffu;
                if (!seen_incl) ok = ok && (ready_mask & need) == need;   // windows past this warp's first prefix do not count
                seen_incl = seen_incl || incl_mask[e] != 0u;
            }
            if (ok || gave_up) break;
            if (t0 == 0) t0 = dev::globaltimer();
            bool expired = (dev::globaltimer() - t0 > limit_ns) || dev::ld_volatile(&ctl->abort) == epoch;
            expired = __any_sync(0xffffffffu, expired);
            if (expired) {
                if (lane == 0) {
                    atomicOr(&ctl->error, kErrTimeout);
                    atomicExch(&ctl->abort, epoch);
                }
                gave_up = true;
            }
        }
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const unsigned lim = incl_mask[e] ? (((incl_mask[e] & (0u - incl_mask[e])) << 1) - 1u) : 0xffffffffu;
            CT v = val[e];
            if (!((lim >> lane) & 1u) || status[e] == 0) v = CT(0);
            sm.vals[(w + NW * e) * 32 + lane] = v;
            if (lane == 0) sm.incl[w + NW * e] = incl_mask[e] != 0u;
        }
        group_sync(id, NW * 32);
        if (w == 0) {
            int kmax = NW * NE - 1;
            bool found_any = false;
#pragma unroll
            for (int k = NW * NE - 1; k >= 0; --k)
                if (sm.incl[k]) { kmax = k; found_any = true; }
            CT wv[NW * NE];   // all loads in flight at once, then a pairwise sum
#pragma unroll
            for (int k = 0; k < NW * NE; ++k) wv[k] = k <= kmax ? sm.vals[k * 32 + lane] : CT(0);
#pragma unroll
            for (int st = 1; st < NW * NE; st *= 2)
#pragma unroll
                for (int k = 0; k + st < NW * NE; k += 2 * st) wv[k] = wv[k] + wv[k + st];
            CT acc = wv[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = acc + dev::shfl_xor_ct(acc, o);
            if (lane == 0) {
                sm.total = excl + acc;
                sm.found = found_any;
            }
        }
        group_sync(id, NW * 32);
        excl = sm.total;
        const bool found = sm.found;
        group_sync(id, NW * 32);   // sm is rewritten by the next round
        if (found) break;
        pred -= 32 * NW * NE;
    }
    if (pub_incl && w == 0 && lane == 0) dev::Codec<CT>::put(d.incl + tile * W, excl + agg, epoch);
    return excl;
}

template <class T, bool INCL, bool REV, int SUB, int STAGES>
__global__ void __launch_bounds__(kWsThreads, 1)
scan_ws(const T *__restrict__ in, T *__restrict__ out, SegGeom g, LookbackDesc d, Control *ctl, uint32_t epoch,
        int64_t skip_tile, uint64_t limit_ns)
{
    using CT = typename ScanTypes<T>::CT;
    using V4 = typename ScanTypes<T>::V4;
    using AddOp = typename std::conditional<std::is_same<T, float>::value, dev::AddF, dev::AddU>::type;
    constexpr int TILE = SUB * kTmaTile;
    constexpr int CH = TILE / kWsChunks;   // elements per chunk (a multiple of 512)
    constexpr int KS = CH / 128;           // 16-byte groups per lane in a chunk
    constexpr int W = dev::Codec<CT>::W;
    static_assert(CH % 512 == 0, "chunks are scanned four 128-element steps at a time");
    extern __shared__ __align__(1024) unsigned char dyn[];   // STAGES tiles
    __shared__ __align__(8) uint64_t full[STAGES], reduced[STAGES], prefixed[STAGES], empty[STAGES];
    __shared__ int64_t tile_of[STAGES];
    __shared__ CT agg_of[STAGES];
    __shared__ CT cpre_of[STAGES][kWsChunks];   // exclusive prefix of the chunk sums
    __shared__ T pre_of[STAGES][kWsChunks];     // each chunk's prefix, in element type
    __shared__ T csum[kWsChunks];
    __shared__ dev::WideLookbackSmem<CT, kWsLookW * kWsLookE> lbs;
    __shared__ int abort_word;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init_count(&full[s], 1);
            mbar_init_count(&reduced[s], 1);
            mbar_init_count(&prefixed[s], 1);
            mbar_init_count(&empty[s], 1);
        }
        abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();   // the last block-wide barrier: the roles part here
    volatile int *abort_v = &abort_word;
    auto stage = [&](int s) { return reinterpret_cast<T *>(dyn + (size_t)s * TILE * sizeof(T)); };
    auto give_up = [&]() {
        *abort_v = 1;
        atomicOr(&ctl->error, kErrTimeout);
    };
    // Input values of logical elements e..e+3 of a staged tile of len
    // elements: slot e forward, len-1-e reverse (reverse tiles have
    // len % 4 == 0); the unstaged forward tail (len % 4 elements) is read
    // from global memory.
    auto src4 = [&](const T *buf, const TileMap &m, int64_t e, T (&a)[4]) {
        const int64_t len = m.len, whole = len & ~(int64_t)3;
        if (e + 3 < whole) {
            const V4 q = *reinterpret_cast<const V4 *>(buf + (REV ? len - 4 - e : e));
            if (!REV) { a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w; }
            else      { a[0] = q.w; a[1] = q.z; a[2] = q.y; a[3] = q.x; }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                a[u] = e + u < whole ? buf[REV ? len - 1 - e - u : e + u] : (e + u < len ? in[m.base + e + u] : T(0));
        }
    };

    if (warp == 0) {
        // ------------------------------------------------------ producer --
        if (lane != 0) return;
        uint32_t last_par[STAGES];
        bool used[STAGES];
#pragma unroll
        for (int s = 0; s < STAGES; ++s) used[s] = false;
        for (uint32_t i = 0;; ++i) {
            const int s = (int)(i % STAGES);
            if (i >= STAGES && !ws_wait(&empty[s], ((i / STAGES) - 1u) & 1u, abort_v, limit_ns)) {
                give_up();
                break;
            }
            const int64_t t = (int64_t)atomicAdd(&ctl->ticket, 1u);
            tile_of[s] = t;
            used[s] = true;
            last_par[s] = (i / STAGES) & 1u;
            if (t >= g.ntiles) {   // the end marker: a phase with no bytes
                mbar_arrive(&full[s]);
                break;
            }
            int64_t first;
            const TileMap m = tile_map<TILE>(g, t, &first);
            const int64_t pstart = m.rev ? m.base - (m.len - 1) : m.base;
            const uint32_t bytes = (uint32_t)((m.len * (int64_t)sizeof(T)) & ~(int64_t)15);
            const uint32_t bar = smem_u32(&full[s]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the scanners' reads before the refill
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
            for (uint32_t o = 0; o < bytes; o += 16384u) {
                const uint32_t sz = bytes - o < 16384u ? bytes - o : 16384u;
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(smem_u32(reinterpret_cast<unsigned char *>(stage(s)) + o)),
                                "l"(reinterpret_cast<const unsigned char *>(in + pstart) + o), "r"(sz), "r"(bar)
                             : "memory");
            }
        }
        // every block has drawn its last ticket once the count reaches the grid
        if (atomicAdd(&ctl->exited, 1u) == gridDim.x - 1) {
            ctl->ticket = 0u;
            ctl->exited = 0u;
        }
        // no copy may land after the block has left: wait (bounded) for the
        // last phase issued on each stage (at once unless a role gave up)
#pragma unroll
        for (int s = 0; s < STAGES; ++s) {
            if (!used[s]) continue;
            uint32_t ok = 0;
            for (uint32_t k = 0; k < (1u << 22) && !ok; ++k) ok = mbar_try(&full[s], last_par[s]);
        }
        return;
    }

    if (warp <= kWsRedW) {
        // ------------------------------------------------------ reducers --
        // warp r sums chunks r and r + kWsRedW: pairwise within each lane,
        // then a warp tree; the leader adds the chunk sums in order.
        const int r = warp - 1, gt = threadIdx.x - 32;
        constexpr int kN = kWsRedW * 32;
        for (uint32_t i = 0;; ++i) {
            const int s = (int)(i % STAGES);
            if (!group_and(kWsBarRed, kN, ws_wait(&full[s], (i / STAGES) & 1u, abort_v, limit_ns))) {
                if (gt == 0) give_up();
                return;
            }
            const int64_t tile = tile_of[s];
            if (tile >= g.ntiles) {
                if (gt == 0) mbar_arrive(&reduced[s]);
                return;
            }
            int64_t first;
            const TileMap m = tile_map<TILE>(g, tile, &first);
            const T *buf = stage(s);
#pragma unroll 1
            for (int cc = 0; cc < kWsChunks / kWsRedW; ++cc) {
                const int c = r + kWsRedW * cc;
                // four running sums of pairwise groups, then a pairwise finish
                T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 1
                for (int k0 = 0; k0 < KS; k0 += 4) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        T a[4];
                        src4(buf, m, (int64_t)c * CH + (k0 + k) * 128 + lane * 4, a);
                        acc[k] = acc[k] + ((a[0] + a[1]) + (a[2] + a[3]));
                    }
                }
                const T cs = dev::warp_reduce<AddOp>((acc[0] + acc[1]) + (acc[2] + acc[3]));
                if (lane == 0) csum[c] = cs;
            }
            group_sync(kWsBarRed, kN);
            if (gt == 0) {
                CT run = CT(0);
#pragma unroll
                for (int c = 0; c < kWsChunks; ++c) {
                    cpre_of[s][c] = run;
                    run = run + (CT)csum[c];
                }
                agg_of[s] = run;
                if (tile != skip_tile) {
                    if (tile == first) dev::Codec<CT>::put(d.incl + tile * W, run, epoch);
                    else dev::Codec<CT>::put(d.agg + tile * W, run, epoch);
                }
                mbar_arrive(&reduced[s]);
            }
            group_sync(kWsBarRed, kN);   // csum is rewritten by the next tile
        }
    }

    if (warp <= kWsRedW + kWsLookW) {
        // ----------------------------------------------------- look-back --
        const int w = warp - 1 - kWsRedW, gt = threadIdx.x - 32 * (1 + kWsRedW);
        constexpr int kN = kWsLookW * 32;
        for (uint32_t i = 0;; ++i) {
            const int s = (int)(i % STAGES);
            if (!group_and(kWsBarLook, kN, ws_wait(&reduced[s], (i / STAGES) & 1u, abort_v, limit_ns))) {
                if (gt == 0) give_up();
                return;
            }
            const int64_t tile = tile_of[s];
            if (tile >= g.ntiles) {
                if (gt == 0) mbar_arrive(&prefixed[s]);
                return;
            }
            int64_t first;
            (void)tile_map<TILE>(g, tile, &first);
            const CT agg = agg_of[s];
            const CT p = group_lookback<CT, kWsLookW, kWsLookE>(tile, first, agg, d, epoch, ctl, limit_ns,
                                                                tile != skip_tile, lbs, w, lane, kWsBarLook);
            if (gt == 0) {
#pragma unroll
                for (int c = 0; c < kWsChunks; ++c) pre_of[s][c] = dev::to_elem<T>(p + cpre_of[s][c]);
                mbar_arrive(&prefixed[s]);
            }
        }
    }

    {
        // ------------------------------------------------------ scanners --
        // warp c scans chunk c in steps of 128 elements (4 per lane): an
        // in-thread scan of 4, a warp scan of the lane totals, a running
        // chunk-local carry; the chunk prefix is added last, once per element.
        const int c = warp - 1 - kWsRedW - kWsLookW, gt = threadIdx.x - 32 * (1 + kWsRedW + kWsLookW);
        constexpr int kN = kWsScanW * 32;
        for (uint32_t i = 0;; ++i) {
            const int s = (int)(i % STAGES);
            const uint32_t par = (i / STAGES) & 1u;
            // the full wait (complete already) makes the staged bytes visible here directly
            if (!group_and(kWsBarScan, kN, ws_wait(&prefixed[s], par, abort_v, limit_ns) &&
                                           ws_wait(&full[s], par, abort_v, limit_ns))) {
                if (gt == 0) give_up();
                return;
            }
            const int64_t tile = tile_of[s];
            if (tile >= g.ntiles) return;
            int64_t first;
            const TileMap m = tile_map<TILE>(g, tile, &first);
            const int64_t len = m.len;
            const int64_t pstart = m.rev ? m.base - (len - 1) : m.base;
            const T *buf = stage(s);
            const T pre = pre_of[s][c];
            T carry = T(0);
#pragma unroll 1
            for (int k0 = 0; k0 < KS; k0 += 4) {
                T v[4][4];
                T lex[4], wtot[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    src4(buf, m, (int64_t)c * CH + (k0 + k) * 128 + lane * 4, v[k]);
                    v[k][1] = v[k][0] + v[k][1];
                    v[k][2] = v[k][1] + v[k][2];
                    v[k][3] = v[k][2] + v[k][3];
                    const T wi = dev::warp_incl_scan_add(v[k][3]);
                    T x = __shfl_up_sync(0xffffffffu, wi, 1);
                    lex[k] = lane == 0 ? T(0) : x;
                    wtot[k] = __shfl_sync(0xffffffffu, wi, 31);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const T b = carry + lex[k];
                    carry = carry + wtot[k];
                    T o[4];
                    if (INCL) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) o[u] = pre + (b + v[k][u]);
                    } else {
                        o[0] = pre + b;
#pragma unroll
                        for (int u = 1; u < 4; ++u) o[u] = pre + (b + v[k][u - 1]);
                    }
                    const int64_t e = (int64_t)c * CH + (k0 + k) * 128 + lane * 4;   // logical
                    if (e + 3 < len) {
                        V4 q;
                        if (!REV) { q.x = o[0]; q.y = o[1]; q.z = o[2]; q.w = o[3]; }
                        else      { q.x = o[3]; q.y = o[2]; q.z = o[1]; q.w = o[0]; }
                        dev::st_stream(reinterpret_cast<V4 *>(out + pstart + (REV ? len - 4 - e : e)), q);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (e + u < len) out[pstart + (REV ? len - 1 - e - u : e + u)] = o[u];
                    }
                }
            }
            group_sync(kWsBarScan, kN);   // every scanner has read the stage
            if (gt == 0) mbar_arrive(&empty[s]);
        }
    }
}

template <class T, bool INCL, bool REV, int SUB, int STAGES>
int launch_scan_ws(const ScanLaunch &sc, cudaStream_t s)
{
    const T *in = static_cast<const T *>(sc.in);
    T *out = static_cast<T *>(sc.out);
    constexpr int TILE = SUB * kTmaTile;
    SegGeom g;
    g.seglen = sc.seg > 0 ? sc.seg : sc.n;
    g.tps = ceil_div(g.seglen, TILE);
    g.ntiles = g.tps * (sc.n / g.seglen);
    g.rev = REV;
    g.vec_ok = true;
    if (g.ntiles > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "scan: too many tiles");
    auto kern = scan_ws<T, INCL, REV, SUB, STAGES>;
    const int dyn = STAGES * TILE * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return fail_cuda(e, "scan ws: shared memory opt-in");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWsThreads, dyn);
    if (e != cudaSuccess || occ < 1) return fail(SKEL_ERR_UNSUPPORTED, "scan ws: kernel does not fit an SM");
    int64_t grid = (int64_t)device_info().sms * occ;
    if (grid > g.ntiles) grid = g.ntiles;
    Scratch scr{};
    int rc = get_scratch(s, 0, 2 * (size_t)g.ntiles, &scr);
    if (rc) return rc;
    LookbackDesc d{scr.words, scr.words + g.ntiles};
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)grid, kWsThreads, (size_t)dyn, s, in, out, g, d, scr.ctl, scr.epoch,
                  k.scan_skip_publish_tile, k.wait_limit_ns);
    e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "scan ws launch");
}

// tile: 0 selects 48 KiB tiles in four stages, 1 selects 32 KiB tiles in six.
template <class T, bool INCL>
int run_scan_ws(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.ept > 0 && c.ept != kTmaV) return fail(SKEL_ERR_INVALID_ARG, "scan ws: ept must be 4");
    if (c.tile < 0 || c.tile > 1) return fail(SKEL_ERR_INVALID_ARG, "scan ws: tile must be 0 or 1");
    const int64_t seglen = sc.seg > 0 ? sc.seg : sc.n;
    if (!aligned16(sc.in) || !aligned16(sc.out) || ((sc.seg > 0 || sc.reverse) && seglen % 4))
        return fail(SKEL_ERR_UNSUPPORTED, "scan ws: 16-byte aligned operands and segments needed");
    if (sc.reverse)
        return c.tile ? launch_scan_ws<T, INCL, true, 2, 6>(sc, s) : launch_scan_ws<T, INCL, true, 3, 4>(sc, s);
    return c.tile ? launch_scan_ws<T, INCL, false, 2, 6>(sc, s) : launch_scan_ws<T, INCL, false, 3, 4>(sc, s);
}

// Variant 0, kernel 1: per-tile aggregate (the tile is scanned to obtain it
// in the same order the apply kernel uses).
template <class T, int V>
__global__ void __launch_bounds__(kBlock)
scan_tile_sums(const T *__restrict__ in, SegGeom g, typename ScanTypes<T>::CT *__restrict__ sums)
{
    constexpr int TILE = kBlock * 4 * V;
    __shared__ T smem[kBlock / 32 + 1];
    int64_t first;
    const TileMap m = tile_map<TILE>(g, blockIdx.x, &first);
    T v[V][4];
    dev::tile_load<T, kBlock, V>(in, m, v);
    const T agg = dev::tile_scan_local<T, true, kBlock, V>(v, smem);
    if (threadIdx.x == 0) sums[blockIdx.x] = (typename ScanTypes<T>::CT)agg;
}

// Variant 0, kernel 2: exclusive scan of the tile sums of one segment per
// block, in place, in the carry type.
template <class CT>
__global__ void __launch_bounds__(1024)
scan_tile_prefixes(CT *__restrict__ sums, int64_t tps)
{
    constexpr int IPT = 8;
    __shared__ CT smem[33];
    CT *s = sums + (int64_t)blockIdx.x * tps;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    CT carry = CT(0);
    for (int64_t c0 = 0; c0 < tps; c0 += 1024 * IPT) {
        CT v[IPT];
        CT t = CT(0);
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int64_t j = c0 + (int64_t)threadIdx.x * IPT + i;
            v[i] = j < tps ? s[j] : CT(0);
            t = t + v[i];
        }
        CT wi = dev::warp_incl_scan_add(t);
        if (lane == 31) smem[w] = wi;
        __syncthreads();
        if (w == 0) {
            CT a = smem[lane];
            CT ai = dev::warp_incl_scan_add(a);
            smem[lane] = ai - a;   // exact for integers; float64 rounding far below float32 output
            if (lane == 31) smem[32] = ai;
        }
        __syncthreads();
        CT run = carry + smem[w] + (wi - t);
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int64_t j = c0 + (int64_t)threadIdx.x * IPT + i;
            if (j < tps) s[j] = run;
            run = run + v[i];
        }
        carry = carry + smem[32];
        __syncthreads();
    }
}

// Variant 0, kernel 3: tile scan plus the tile's exclusive prefix.
template <class T, bool INCL, int V>
__global__ void __launch_bounds__(kBlock)
scan_tile_apply(const T *__restrict__ in, T *__restrict__ out, SegGeom g,
                const typename ScanTypes<T>::CT *__restrict__ prefixes)
{
    constexpr int TILE = kBlock * 4 * V;
    __shared__ T smem[kBlock / 32 + 1];
    int64_t first;
    const TileMap m = tile_map<TILE>(g, blockIdx.x, &first);
    T v[V][4];
    dev::tile_load<T, kBlock, V>(in, m, v);
    dev::tile_scan_local<T, INCL, kBlock, V>(v, smem);
    dev::tile_add_prefix<T, V>(v, dev::to_elem<T>(prefixes[blockIdx.x]));
    dev::tile_store<T, kBlock, V>(out, m, v);
}

// Variant 2: one block, tiles in order, prefix carried (reset per segment).
template <class T, bool INCL, int V>
__global__ void __launch_bounds__(kBlock)
scan_one_block(const T *__restrict__ in, T *__restrict__ out, SegGeom g)
{
    using CT = typename ScanTypes<T>::CT;
    constexpr int TILE = kBlock * 4 * V;
    __shared__ T smem[kBlock / 32 + 1];
    CT carry = CT(0);
    for (int64_t tile = 0; tile < g.ntiles; ++tile) {
        int64_t first;
        const TileMap m = tile_map<TILE>(g, tile, &first);
        if (tile == first) carry = CT(0);
        T v[V][4];
        dev::tile_load<T, kBlock, V>(in, m, v);
        const T agg = dev::tile_scan_local<T, INCL, kBlock, V>(v, smem);
        dev::tile_add_prefix<T, V>(v, dev::to_elem<T>(carry));
        dev::tile_store<T, kBlock, V>(out, m, v);
        carry = carry + (CT)agg;
    }
}

template <class T, bool INCL, int V>
int run_scan(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    using CT = typename ScanTypes<T>::CT;
    constexpr int TILE = kBlock * 4 * V;
    const T *in = static_cast<const T *>(sc.in);
    T *out = static_cast<T *>(sc.out);
    SegGeom g;
    g.seglen = sc.seg > 0 ? sc.seg : sc.n;
    if (g.seglen == 0) return SKEL_OK;
    g.tps = ceil_div(g.seglen, TILE);
    g.ntiles = g.tps * (sc.n / g.seglen);
    g.rev = sc.reverse;
    // 16-byte accesses need aligned pointers and, for every full tile, a
    // start (forward) or end (reverse) on a 4-element boundary.
    const bool ptr_ok = aligned16(in) && aligned16(out);
    const bool seg_ok = sc.seg > 0 ? (g.seglen % 4 == 0) : (!sc.reverse || g.seglen % 4 == 0);
    g.vec_ok = ptr_ok && seg_ok;
    if (g.ntiles > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "scan: too many tiles");
    if (c.variant == 2) {
        launch_kernel(scan_one_block<T, INCL, V>, 1, kBlock, 0, s, in, out, g);
    } else if (c.variant == 0) {
        Scratch scr{};
        int rc = get_scratch(s, (size_t)g.ntiles * sizeof(CT), 0, &scr);
        if (rc) return rc;
        CT *sums = reinterpret_cast<CT *>(scr.data);
        launch_kernel(scan_tile_sums<T, V>, (unsigned)g.ntiles, kBlock, 0, s, in, g, sums);
        launch_kernel(scan_tile_prefixes<CT>, (unsigned)(g.ntiles / g.tps), 1024, 0, s, sums, g.tps);
        launch_kernel(scan_tile_apply<T, INCL, V>, (unsigned)g.ntiles, kBlock, 0, s, in, out, g, sums);
    } else {
        Scratch scr{};
        int rc = get_scratch(s, 0, 2 * (size_t)g.ntiles, &scr);   // one aggregate + one prefix word per tile
        if (rc) return rc;
        LookbackDesc d{scr.words, scr.words + g.ntiles};
        const DebugKnobs k = debug_knobs();
        if (c.variant == 3)
            launch_kernel(scan_lookback<T, INCL, V, true>, (unsigned)g.ntiles, kBlock, 0, s,
                          in, out, g, d, scr.ctl, scr.epoch, k.scan_skip_publish_tile, k.wait_limit_ns);
        else
            launch_kernel(scan_lookback<T, INCL, V, false>, (unsigned)g.ntiles, kBlock, 0, s,
                          in, out, g, d, scr.ctl, scr.epoch, k.scan_skip_publish_tile, k.wait_limit_ns);
    }
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "scan launch");
}

template <class T, bool INCL>
int run_scan_tma(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    const T *in = static_cast<const T *>(sc.in);
    T *out = static_cast<T *>(sc.out);
    if (sc.reverse) return fail(SKEL_ERR_UNSUPPORTED, "scan tma: forward scans only");
    if (c.ept > 0 && c.ept != kTmaV) return fail(SKEL_ERR_INVALID_ARG, "scan tma: ept must be 4");
    SegGeom g;
    g.seglen = sc.seg > 0 ? sc.seg : sc.n;
    g.tps = ceil_div(g.seglen, kTmaTile);
    g.ntiles = g.tps * (sc.n / g.seglen);
    g.rev = false;
    // bulk copies start on 16-byte boundaries: aligned pointers, segments of a multiple of 4 elements
    if (!aligned16(in) || !aligned16(out) || (sc.seg > 0 && g.seglen % 4))
        return fail(SKEL_ERR_UNSUPPORTED, "scan tma: 16-byte aligned operands and segments needed");
    g.vec_ok = true;
    if (g.ntiles > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "scan: too many tiles");
    auto kern = scan_tma<T, INCL>;
    const int dyn = kStages * kTmaTile * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return fail_cuda(e, "scan tma: shared memory opt-in");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, dyn);
    if (e != cudaSuccess || occ < 1) return fail(SKEL_ERR_UNSUPPORTED, "scan tma: kernel does not fit an SM");
    int64_t grid = (int64_t)device_info().sms * occ;
    if (grid > g.ntiles) grid = g.ntiles;
    Scratch scr{};
    int rc = get_scratch(s, 0, 2 * (size_t)g.ntiles, &scr);
    if (rc) return rc;
    LookbackDesc d{scr.words, scr.words + g.ntiles};
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)grid, kBlock, (size_t)dyn, s, in, out, g, d, scr.ctl, scr.epoch,
                  k.scan_skip_publish_tile, k.wait_limit_ns);
    e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "scan tma launch");
}

template <class T, bool INCL, bool REV, int SUB>
int launch_scan_big(const ScanLaunch &sc, bool early, cudaStream_t s)
{
    const T *in = static_cast<const T *>(sc.in);
    T *out = static_cast<T *>(sc.out);
    constexpr int TILE = SUB * kTmaTile;
    SegGeom g;
    g.seglen = sc.seg > 0 ? sc.seg : sc.n;
    g.tps = ceil_div(g.seglen, TILE);
    g.ntiles = g.tps * (sc.n / g.seglen);
    g.rev = REV;
    g.vec_ok = true;
    if (g.ntiles > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "scan: too many tiles");
    auto kern = early ? scan_big<T, INCL, REV, true, SUB> : scan_big<T, INCL, REV, false, SUB>;
    const int dyn = TILE * (int)sizeof(T);
    cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea != cudaSuccess) return fail_cuda(ea, "scan big: shared memory opt-in");
    Scratch scr{};
    int rc = get_scratch(s, 0, 2 * (size_t)g.ntiles, &scr);
    if (rc) return rc;
    LookbackDesc d{scr.words, scr.words + g.ntiles};
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)g.ntiles, kBlock, (size_t)dyn, s, in, out, g, d, scr.ctl, scr.epoch,
                  k.scan_skip_publish_tile, k.wait_limit_ns);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "scan big launch");
}

// tile: bit 0 publishes the aggregate early; bit 1 selects 48 KiB tiles
// (three sub-tiles) instead of 64 KiB ones.
template <class T, bool INCL>
int run_scan_big(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.ept > 0 && c.ept != kTmaV) return fail(SKEL_ERR_INVALID_ARG, "scan big: ept must be 4");
    if (c.tile < 0 || c.tile > 3) return fail(SKEL_ERR_INVALID_ARG, "scan big: tile must be 0..3");
    // bulk copies start on 16-byte boundaries: aligned operands, and segments
    // of a multiple of 4 elements (reverse 1D scans: n % 4 == 0)
    const int64_t seglen = sc.seg > 0 ? sc.seg : sc.n;
    if (!aligned16(sc.in) || !aligned16(sc.out) || ((sc.seg > 0 || sc.reverse) && seglen % 4))
        return fail(SKEL_ERR_UNSUPPORTED, "scan big: 16-byte aligned operands and segments needed");
    const bool early = c.tile & 1, sub3 = c.tile & 2;
    if (sc.reverse)
        return sub3 ? launch_scan_big<T, INCL, true, 3>(sc, early, s) : launch_scan_big<T, INCL, true, 4>(sc, early, s);
    return sub3 ? launch_scan_big<T, INCL, false, 3>(sc, early, s) : launch_scan_big<T, INCL, false, 4>(sc, early, s);
}

template <class T, bool INCL, bool REV, int SUBS, int SUBR, int MINB>
int launch_scan_hybrid(const ScanLaunch &sc, cudaStream_t s)
{
    const T *in = static_cast<const T *>(sc.in);
    T *out = static_cast<T *>(sc.out);
    constexpr int TILE = (SUBS + SUBR) * kTmaTile;
    SegGeom g;
    g.seglen = sc.seg > 0 ? sc.seg : sc.n;
    g.tps = ceil_div(g.seglen, TILE);
    g.ntiles = g.tps * (sc.n / g.seglen);
    g.rev = REV;
    g.vec_ok = true;
    const int64_t nseg = sc.n / g.seglen, tpsf = g.seglen / TILE, nfull = nseg * tpsf;
    if (g.ntiles > 0x7fffffffLL || nseg > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "scan: too many tiles");
    auto kfull = scan_hybrid<T, INCL, REV, SUBS, SUBR, MINB, false>;
    auto kpart = scan_hybrid<T, INCL, REV, SUBS, SUBR, MINB, true>;
    const int dyn = SUBS * kTmaTile * (int)sizeof(T);
    cudaError_t ea = cudaFuncSetAttribute(kfull, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea == cudaSuccess) ea = cudaFuncSetAttribute(kpart, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (ea != cudaSuccess) return fail_cuda(ea, "scan hybrid: shared memory opt-in");
    Scratch scr{};
    int rc = get_scratch(s, 0, 2 * (size_t)g.ntiles, &scr);
    if (rc) return rc;
    LookbackDesc d{scr.words, scr.words + g.ntiles};
    const DebugKnobs k = debug_knobs();
    if (nfull > 0)
        launch_kernel(kfull, (unsigned)nfull, kBlock, (size_t)dyn, s, in, out, g, tpsf, d, scr.ctl, scr.epoch,
                      k.scan_skip_publish_tile, k.wait_limit_ns);
    if (g.seglen % TILE)   // every segment's last, partial tile, after the whole ones
        launch_kernel(kpart, (unsigned)nseg, kBlock, (size_t)dyn, s, in, out, g, tpsf, d, scr.ctl, scr.epoch,
                      k.scan_skip_publish_tile, k.wait_limit_ns);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "scan hybrid launch");
}

// tile: 0 = 96 KiB staged + 64 KiB in registers (two blocks per SM),
// 1 = 64 KiB + 32 KiB (three blocks per SM), 2 = 64 KiB + 48 KiB (three
// blocks per SM), 3 = 96 KiB + 80 KiB (two blocks per SM).
template <class T, bool INCL, bool REV>
int run_scan_hybrid_dir(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.tile == 0) return launch_scan_hybrid<T, INCL, REV, 6, 4, 2>(sc, s);
    if (c.tile == 1) return launch_scan_hybrid<T, INCL, REV, 4, 2, 3>(sc, s);
    if (c.tile == 2) return launch_scan_hybrid<T, INCL, REV, 4, 3, 3>(sc, s);
    return launch_scan_hybrid<T, INCL, REV, 6, 5, 2>(sc, s);
}

template <class T, bool INCL>
int run_scan_hybrid(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.ept > 0 && c.ept != kTmaV) return fail(SKEL_ERR_INVALID_ARG, "scan hybrid: ept must be 4");
    if (c.tile < 0 || c.tile > 3) return fail(SKEL_ERR_INVALID_ARG, "scan hybrid: tile must be 0..3");
    // bulk copies start on 16-byte boundaries: aligned operands, and segments
    // of a multiple of 4 elements (reverse 1D scans: n % 4 == 0)
    const int64_t seglen = sc.seg > 0 ? sc.seg : sc.n;
    if (!aligned16(sc.in) || !aligned16(sc.out) || ((sc.seg > 0 || sc.reverse) && seglen % 4))
        return fail(SKEL_ERR_UNSUPPORTED, "scan hybrid: 16-byte aligned operands and segments needed");
    return sc.reverse ? run_scan_hybrid_dir<T, INCL, true>(sc, c, s) : run_scan_hybrid_dir<T, INCL, false>(sc, c, s);
}

template <class T, bool INCL>
int run_scan_v(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.variant == 4) return run_scan_tma<T, INCL>(sc, c, s);
    if (c.variant == 5) return run_scan_big<T, INCL>(sc, c, s);
    if (c.variant == 7) return run_scan_hybrid<T, INCL>(sc, c, s);
    if (c.variant == 6) return run_scan_ws<T, INCL>(sc, c, s);
    const int v = c.ept > 0 ? c.ept : 4;
    switch (v) {
    case 2: return run_scan<T, INCL, 2>(sc, c, s);
    case 4: return run_scan<T, INCL, 4>(sc, c, s);
    case 8: return run_scan<T, INCL, 8>(sc, c, s);
    default: return fail(SKEL_ERR_INVALID_ARG, "scan: ept (16-byte groups per thread) must be 2, 4 or 8");
    }
}

}  // namespace

int scan_variant_count() { return 9; }
const char *scan_variant_name(int v)
{
    static const char *names[] = {"reduce_then_scan", "lookback", "one_block", "lookback_block", "lookback_tma",
                                  "lookback_big", "lookback_ws", "lookback_hybrid", "lookback_reread"};
    return v >= 0 && v < 9 ? names[v] : "?";
}
Choice scan_default() { return Choice{0, 256, 4, 0}; }

int launch_scan(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (sc.n == 0) return SKEL_OK;
    if (c.variant < 0 || c.variant > 8) return fail(SKEL_ERR_INVALID_ARG, "scan: unknown variant");
    if (c.block > 0 && c.block != kBlock) return fail(SKEL_ERR_INVALID_ARG, "scan: block must be 256");
    if (sc.seg > 0 && sc.n % sc.seg) return fail(SKEL_ERR_SHAPE, "scan: n is not a multiple of the segment");
    if (c.variant == 8) return scan_rr_launch(sc, c, s);
    if (sc.dtype == SKEL_F32)
        return sc.inclusive ? run_scan_v<float, true>(sc, c, s) : run_scan_v<float, false>(sc, c, s);
    if (sc.dtype == SKEL_I32)
        return sc.inclusive ? run_scan_v<uint32_t, true>(sc, c, s) : run_scan_v<uint32_t, false>(sc, c, s);
    return fail(SKEL_ERR_DTYPE, "scan: float32 or int32 only");
}

}  // namespace skel
