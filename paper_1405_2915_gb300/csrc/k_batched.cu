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
// Variants: 0 persistent (grid = SMs x resident blocks per SM), look-back
//             walked by warp 0;
//           1 one_per_tile (grid = the tile bound; surplus blocks exit);
//           2 persistent with the whole block walking the look-back.
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

// BLK: the whole block walks the look-back (variant 2) or warp 0 alone
// (variants 0, 1).  words: 2 * max_t aggregate words, then 2 * max_t prefix words.
template <bool SCAN, bool RED, bool INCL, int V, bool BLK>
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
    const int64_t total = *reinterpret_cast<volatile int64_t *>(L.total_tiles);
    const dev::LookbackDesc d{words, words + 2 * max_t};
    while (true) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(&ctl->queue, 1u);
        __syncthreads();
        const int64_t t = s_tile;
        if (t >= total) break;
        const int64_t b = L.tile_inst[t];
        const int64_t lo = off[b], hi = off[b + 1];
        const int64_t first = L.tile_start[b];
        const int64_t last = L.tile_start[b + 1] - 1;
        const int64_t fbase = (lo & ~(int64_t)3) + (t - first) * TILE;
        float v[V][4];
        load_masked<V>(values, fbase, lo, hi, v);
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
        const Pair agg((double)sagg, (double)q);
        Pair p(0.0);
        if (first != last) {   // block-uniform
            if (BLK) {
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
    auto kern = c.variant == 2 ? batched_main<SCAN, RED, INCL, V, true> : batched_main<SCAN, RED, INCL, V, false>;
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

int tile_of(const Choice &c) { return kBlock * 4 * (c.ept > 0 ? c.ept : 4); }

}  // namespace

int batched_variant_count() { return 3; }
const char *batched_variant_name(int v)
{
    static const char *names[] = {"persistent", "one_per_tile", "persistent_block_lookback"};
    return v >= 0 && v < 3 ? names[v] : "?";
}
Choice batched_default() { return Choice{0, 256, 4, 0}; }

size_t batched_data_bytes(const BatchedLaunch &b, const Choice &c) { return layout_bytes(b, tile_of(c)); }
// aggregate and prefix of every tile, two words (scan carry, sum of squares) each
size_t batched_word_count(const BatchedLaunch &b, const Choice &c) { return 4 * (size_t)max_tiles(b, tile_of(c)); }

int launch_batched(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
                   uint32_t epoch, cudaStream_t s)
{
    if (c.variant < 0 || c.variant > 2) return fail(SKEL_ERR_INVALID_ARG, "batched: unknown variant");
    if (c.block > 0 && c.block != kBlock) return fail(SKEL_ERR_INVALID_ARG, "batched: block must be 256");
    if (!aligned16(b.values) || (b.scan_out && !aligned16(b.scan_out)))
        return fail(SKEL_ERR_UNSUPPORTED, "batched: values and scan_out must be 16-byte aligned");
    if (b.B == 0) return SKEL_OK;
    switch (c.ept > 0 ? c.ept : 4) {
    case 2: return run_v<2>(b, c, ctl, words, data, epoch, s);
    case 4: return run_v<4>(b, c, ctl, words, data, epoch, s);
    case 8: return run_v<8>(b, c, ctl, words, data, epoch, s);
    default: return fail(SKEL_ERR_INVALID_ARG, "batched: ept must be 2, 4 or 8");
    }
}

}  // namespace skel
