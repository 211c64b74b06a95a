// Batched variant 6 (the dispatch and the other variants are in
// k_batched.cu): the instances as one flat segmented scan in tiles staged
// partly in shared memory and partly in registers.
#include "batched_flat.cuh"

namespace skel {
namespace {

// ---------------------------------------- variant 6: flat segmented ----
// The instances lie end to end in `values`, so the batched call is one scan
// of the whole array that restarts at every instance start (a segmented
// scan), plus a segmented sum of squares read at every instance's last
// element.  Tiles of the flat array (every tile but the last is whole and
// 16-byte aligned, unlike per-instance frames, so short instances share a
// tile instead of each taking one), staged partly in shared memory and
// partly in registers as in scan variant 7, drawn in ticket order:
//   heads:  the instance starts inside the tile (from the instance holding
//           the tile's first element, which the offsets check tabulates, on
//           through the sorted offsets), as a bitmap in shared memory, with
//           the first kSegOffCap of them listed for the result index;
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
// Warp ranges with no instance start or end take a plain scan.  The combine
// of (sum, sum of squares, has-head) triples is in batched_flat.cuh.

// Offsets of a tile's instances kept in shared memory.
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
        if (!SCAN && head_free(j)) return;   // nothing to store and no instance ends here
        if (SCAN && head_free(j)) {   // a plain scan of the sums; no instance ends here, so no squares are needed
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

// variant 6 tile shapes (the config's tile index): sub-tiles staged in
// shared memory, sub-tiles held in registers, blocks per SM
constexpr int kSegShape[2][3] = {{6, 2, 2}, {4, 2, 3}};
constexpr int seg_tile(int shape) { return (kSegShape[shape][0] + kSegShape[shape][1]) * kSubTile; }


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
    if (c.tile < 0 || c.tile > 1) return fail(SKEL_ERR_INVALID_ARG, "batched segmented: tile shape must be 0 or 1");
    const int tile = seg_tile(c.tile);
    if (ceil_div(b.total, tile) > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "batched: too many tiles");
    int *ok = reinterpret_cast<int *>(data);
    int64_t *tile_inst = reinterpret_cast<int64_t *>(data + 256);
    launch_kernel(batched_seg_prep, 1, 1024, 0, s, b.offsets, b.B, b.total, tile, b.results, ok, tile_inst, ctl);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail_cuda(cudaGetLastError(), "batched segmented prep launch");
    if (b.total == 0) return SKEL_OK;
    return c.tile ? run_seg_shape<1>(b, ctl, words, ok, tile_inst, epoch, s)
                  : run_seg_shape<0>(b, ctl, words, ok, tile_inst, epoch, s);
}

}  // namespace

int batched_seg_tile(int tile) { return seg_tile(tile == 1 ? 1 : 0); }

int batched_seg_launch(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
                       uint32_t epoch, cudaStream_t s)
{
    return run_seg(b, c, ctl, words, data, epoch, s);
}

}  // namespace skel
