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
//                       one predecessor per thread (256 per round): with many
//                       tiles in flight the nearest published prefix lies far
//                       back, and warp 0 alone needs many rounds while the
//                       other warps wait at the barrier.
// ept selects V, the 16-byte groups per thread (tile = 256 threads x 4V).
// float32: element arithmetic is float32; the prefix carried from tile to
// tile is float64 (one add per tile), rounded to float32 once per tile.
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
int run_scan_v(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    const int v = c.ept > 0 ? c.ept : 4;
    switch (v) {
    case 2: return run_scan<T, INCL, 2>(sc, c, s);
    case 4: return run_scan<T, INCL, 4>(sc, c, s);
    case 8: return run_scan<T, INCL, 8>(sc, c, s);
    default: return fail(SKEL_ERR_INVALID_ARG, "scan: ept (16-byte groups per thread) must be 2, 4 or 8");
    }
}

}  // namespace

int scan_variant_count() { return 4; }
const char *scan_variant_name(int v)
{
    static const char *names[] = {"reduce_then_scan", "lookback", "one_block", "lookback_block"};
    return v >= 0 && v < 4 ? names[v] : "?";
}
Choice scan_default() { return Choice{0, 256, 4, 0}; }

int launch_scan(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (sc.n == 0) return SKEL_OK;
    if (c.variant < 0 || c.variant > 3) return fail(SKEL_ERR_INVALID_ARG, "scan: unknown variant");
    if (c.block > 0 && c.block != kBlock) return fail(SKEL_ERR_INVALID_ARG, "scan: block must be 256");
    if (sc.seg > 0 && sc.n % sc.seg) return fail(SKEL_ERR_SHAPE, "scan: n is not a multiple of the segment");
    if (sc.dtype == SKEL_F32)
        return sc.inclusive ? run_scan_v<float, true>(sc, c, s) : run_scan_v<float, false>(sc, c, s);
    if (sc.dtype == SKEL_I32)
        return sc.inclusive ? run_scan_v<uint32_t, true>(sc, c, s) : run_scan_v<uint32_t, false>(sc, c, s);
    return fail(SKEL_ERR_DTYPE, "scan: float32 or int32 only");
}

}  // namespace skel
