// Scan variant 8 (the other variants and the dispatch are in k_scan.cu):
// aggregator warps and re-reading scanner warps in one persistent block per
// SM.
#include <type_traits>

#include "scan_tile.cuh"

namespace skel {
namespace {

using dev::LookbackDesc;
using dev::ScanTypes;

constexpr int kTmaV = 4;   // 16-byte groups per thread of the tile layout (the only ept accepted)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
}

// Try the phase of parity `parity`; a thread whose phase is not complete is
// suspended until it completes or about hint_ns pass.
__device__ __forceinline__ uint32_t mbar_try_sleep(const uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns) : "memory");
    return done;
}
constexpr uint32_t kSleepHintNs = 20000;   // 20 us per suspended try

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

// ---------------------------- variant 8: aggregator warps, re-reading scanners --
// One persistent block per SM whose warps take two roles:
//   aggregators (kRrAggW warps): draw tile tickets in order, stream each
//     tile through a ring of shared-memory slots (one bulk copy per tile),
//     sum it as soon as it lands, publish its aggregate, hand (tile,
//     aggregate) to the scanners through a queue in shared memory and start
//     the next ticket's copy into the slot at once;
//   scanners (NC warps, one tile each): take the next tile from the queue,
//     start a second bulk copy of it into the warp's own buffer (the tile
//     was read microseconds before, so it comes from L2), walk the
//     look-back while that copy lands, publish the inclusive prefix, then
//     scan the buffer with warp scans and store the result.
// Variants 5 and 7 keep a tile in shared memory or registers through its
// look-back wait, about a third of a tile's life on this GPU, and that
// staging has no copy in flight meanwhile.  Here a ring slot holds a tile
// only while its copy lands, so the ring always carries copies in flight;
// the look-back wait is spent by scanner warps whose buffers are fed from
// L2.  DRAM traffic stays one read and one write per element as long as
// the second read hits L2 (the tiles between the two reads take a few tens
// of MB of the 129 MB L2).
// Progress: tickets are drawn in order and each block's queue is taken in
// order, so the smallest tile without an inclusive prefix is one whose
// aggregate is published (aggregators never wait on look-back) and whose
// scanner only waits for its predecessors, all of which have prefixes.
// An aggregator waits only for its own copies and for room in its block's
// queue, which its scanners free without waiting on anything.  Every wait
// is bounded;
// one that runs out records kErrTimeout and the call's abort tag, which ends
// every other waiter of the call; blocks wait (bounded) for their copies
// before leaving, and the last block to leave resets the ticket counter.
constexpr int kRrTE = 4096;   // elements per tile
constexpr int kRrAggW = 2;    // aggregator warps
constexpr int kRrQueue = 16;  // queue entries per block
constexpr int kRrBar = 1;     // named barrier of the aggregators (0: __syncthreads)

// The scanner's running prefix across a tile's 512-element blocks.  int32:
// one uint32.  float32: an unevaluated sum hi + lo of two floats, advanced by
// an exact two-sum (Knuth's TwoSum) so that it carries about 48 bits, like
// the float64 prefix it starts from, with float32 operations only (float64
// units are few on this GPU and the carry is a dependent chain).
template <class T> struct RrCarry;
template <> struct RrCarry<uint32_t> {
    uint32_t c;
    __device__ __forceinline__ explicit RrCarry(uint32_t e) : c(e) {}
    __device__ __forceinline__ uint32_t base() const { return c; }
    __device__ __forceinline__ void add(uint32_t v) { c += v; }
};
template <> struct RrCarry<float> {
    float hi, lo;
    __device__ __forceinline__ explicit RrCarry(double e) : hi((float)e), lo((float)(e - (double)(float)e)) {}
    __device__ __forceinline__ float base() const { return hi + lo; }
    __device__ __forceinline__ void add(float v)
    {
        const float s = hi + v, bv = s - hi;
        lo += (hi - (s - bv)) + (v - bv);   // the rounding error of hi + v, exactly
        hi = s;
    }
};

template <class T, bool INCL, bool REV, bool ROWS, int R, int NC>
__global__ void __launch_bounds__((kRrAggW + NC) * 32, 1)
scan_rr(const T *__restrict__ in, T *__restrict__ out, int64_t seglen, int64_t tps, int64_t ntiles, LookbackDesc d,
        Control *ctl, uint32_t epoch, int64_t skip_tile, uint64_t limit_ns)
{
    using CT = typename ScanTypes<T>::CT;
    using V4 = typename ScanTypes<T>::V4;
    using AddOp = typename std::conditional<std::is_same<T, float>::value, dev::AddF, dev::AddU>::type;
    constexpr int TE = kRrTE, NA = kRrAggW, QC = kRrQueue;
    constexpr uint32_t TB = TE * sizeof(T);
    constexpr int W = dev::Codec<CT>::W;
    extern __shared__ __align__(1024) unsigned char dyn[];   // R ring slots, then one buffer per scanner warp
    __shared__ __align__(8) uint64_t ring_full[R], buf_full[NC];
    __shared__ int64_t slot_tile[R];
    __shared__ int64_t q_tile[QC];
    __shared__ T q_agg[QC];
    __shared__ T a_part[NA];
    __shared__ int q_tail, q_claim, q_read, a_done, s_stop;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // tile t is tile t % tps of segment t / tps (ROWS: rows of seglen
    // elements; else one segment and no division on the tile's path)
    auto seg_of = [&](int64_t t) -> int64_t { return ROWS ? (int64_t)((uint32_t)t / (uint32_t)tps) : 0; };
    auto first_of = [&](int64_t t) -> int64_t { return seg_of(t) * tps; };
    auto tile_len = [&](int64_t t) -> int {
        const int64_t e0 = (t - seg_of(t) * tps) * TE;
        return seglen - e0 < TE ? (int)(seglen - e0) : TE;
    };
    // physical index of logical element e of tile t
    auto phys = [&](int64_t t, int64_t e) -> int64_t {
        const int64_t sg = seg_of(t), e0 = (t - sg * tps) * TE;
        return REV ? (sg + 1) * seglen - 1 - e0 - e : sg * seglen + e0 + e;
    };
    // first physical element of whole tile t
    auto tile_start = [&](int64_t t) -> int64_t {
        const int64_t sg = seg_of(t), e0 = (t - sg * tps) * TE;
        return REV ? (sg + 1) * seglen - e0 - TE : sg * seglen + e0;
    };
    auto gave_up = [&]() { return dev::ld_volatile(&ctl->abort) == epoch; };
    auto give_up = [&]() {
        atomicOr(&ctl->error, kErrTimeout);
        atomicExch(&ctl->abort, epoch);
    };
    // bounded wait for the phase of parity par: false when the limit ran out
    // or another waiter of the call gave up
    auto wait_phase = [&](const uint64_t *bar, uint32_t par) -> bool {
        const uint64_t t0 = dev::globaltimer();
        for (uint32_t k = 0; k < (1u << 26); ++k) {
            if (mbar_try_sleep(bar, par, kSleepHintNs)) return true;
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
        for (int r = 0; r < R; ++r) mbar_init(&ring_full[r]);
        for (int r = 0; r < NC; ++r) mbar_init(&buf_full[r]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (w < NA) {
        // ---------------------------------------------------------- aggregators
        // thread 0: the copy of ticket t into the slot, the partial last tile
        // by a plain arrival (it is summed from global memory), or the end mark
        auto start = [&](int slot, uint32_t t) {
            if (s_stop || (int64_t)t >= ntiles) {
                s_stop = 1;
                slot_tile[slot] = ntiles;
                return;
            }
            slot_tile[slot] = t;
            const uint32_t b = smem_u32(&ring_full[slot]);
            if (tile_len(t) < TE) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
                return;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(TB) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(dyn + slot * TB)), "l"(in + tile_start(t)), "r"(TB), "r"(b) : "memory");
        };
        if (threadIdx.x == 0) {
            uint32_t first[R];
#pragma unroll
            for (int s = 0; s < R; ++s) first[s] = atomicAdd(&ctl->ticket, 1u);   // all in flight at once
#pragma unroll
            for (int s = 0; s < R; ++s) start(s, first[s]);
        }
        group_sync(kRrBar, NA * 32);
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
            if (!group_and(kRrBar, NA * 32, done)) {   // a copy never landed
                if (threadIdx.x == 0) give_up();
                // drain every slot still waiting on a copy (parity of its pending phase)
                for (int j = 0; j < R; ++j) {
                    if (slot_tile[j] >= ntiles) continue;
                    const uint32_t pj = (uint32_t)(i / R + (j < slot ? 1 : 0)) & 1u;
                    const uint64_t t0 = dev::globaltimer();
                    for (uint32_t k = 0; k < (1u << 26); ++k)
                        if (mbar_try_sleep(&ring_full[j], pj, kSleepHintNs) || dev::globaltimer() - t0 > limit_ns) break;
                }
                break;
            }
            // the tile sum: four accumulators per thread, each over groups of four (a shallow sum)
            T acc[4] = {T(0), T(0), T(0), T(0)};
            const int len = tile_len(t);
            if (len == TE) {
                const V4 *src = reinterpret_cast<const V4 *>(dyn + slot * TB);
                constexpr int PER = TE / 4 / (NA * 32);   // groups of four per thread
                static_assert(PER % 4 == 0, "whole rounds of the four accumulators");
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const V4 q = src[k * NA * 32 + threadIdx.x];
                    acc[k & 3] = acc[k & 3] + ((q.x + q.y) + (q.z + q.w));
                }
            } else {
                for (int k0 = 0; k0 * NA * 32 * 4 < len; k0 += 4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int e = ((k0 + j) * NA * 32 + threadIdx.x) * 4;
                        const T x0 = e < len ? in[phys(t, e)] : T(0), x1 = e + 1 < len ? in[phys(t, e + 1)] : T(0);
                        const T x2 = e + 2 < len ? in[phys(t, e + 2)] : T(0), x3 = e + 3 < len ? in[phys(t, e + 3)] : T(0);
                        acc[j] = acc[j] + ((x0 + x1) + (x2 + x3));
                    }
                }
            }
            const T s = dev::warp_reduce<AddOp>((acc[0] + acc[1]) + (acc[2] + acc[3]));
            if (lane == 0) a_part[w] = s;
            group_sync(kRrBar, NA * 32);   // every read of the slot is done; the partial sums are visible
            if (threadIdx.x == 0) {
                T agg = a_part[0];
#pragma unroll
                for (int j = 1; j < NA; ++j) agg = agg + a_part[j];
                if (t != skip_tile) {   // a segment's first tile: its sum is its inclusive prefix
                    if (t == first_of(t)) dev::Codec<CT>::put(d.incl + t * W, (CT)agg, epoch);
                    else dev::Codec<CT>::put(d.agg + t * W, (CT)agg, epoch);
                }
                const uint64_t t0 = dev::globaltimer();
                for (uint32_t k = 0; k < (1u << 26); ++k) {   // room in the queue (bounded)
                    if (q_tail - *(volatile int *)&q_read < QC) break;
                    if (gave_up() || dev::globaltimer() - t0 > limit_ns) break;
                    __nanosleep(64);
                }
                if (q_tail - *(volatile int *)&q_read < QC) {
                    q_tile[q_tail % QC] = t;
                    q_agg[q_tail % QC] = agg;
                    __threadfence_block();
                    *(volatile int *)&q_tail = q_tail + 1;
                } else {
                    give_up();   // the tile is dropped; the call reports the timeout
                }
                start(slot, next);
            }
            // slot_tile[] is read again only after later barriers of this group
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
    uint32_t cpar = 0;
    while (true) {
        int k = 0, have = 0;
        if (lane == 0) {
            k = atomicAdd(&q_claim, 1);
            const uint64_t t0 = dev::globaltimer();
            for (uint32_t it = 0; it < (1u << 26); ++it) {
                const int dn = *(volatile int *)&a_done;
                __threadfence_block();
                if (k < *(volatile int *)&q_tail) { have = 1; break; }
                if (dn) break;
                if (dev::globaltimer() - t0 > 4 * limit_ns) { give_up(); break; }   // the aggregators stopped answering
                __nanosleep(64);
            }
        }
        if (!__shfl_sync(0xffffffffu, have, 0)) break;
        int64_t t = 0;
        T agg = T(0);
        if (lane == 0) {
            __threadfence_block();
            t = q_tile[k % QC];
            agg = q_agg[k % QC];
            __threadfence_block();
            atomicAdd(&q_read, 1);
            // the tile again, into this warp's buffer (whole tiles; the partial one is read directly)
            const uint32_t b = smem_u32(&buf_full[cw]);
            if (tile_len(t) == TE) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(TB) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(smem_u32(buf)), "l"(in + tile_start(t)), "r"(TB), "r"(b) : "memory");
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
            }
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        agg = __shfl_sync(0xffffffffu, agg, 0);
        const int64_t first = first_of(t);
        const CT excl = dev::lookback<CT>(t, first, (CT)agg, d, epoch, ctl, limit_ns, false);
        if (lane == 0 && t != first && t != skip_tile) dev::Codec<CT>::put(d.incl + t * W, excl + (CT)agg, epoch);
        const bool landed = __all_sync(0xffffffffu, wait_phase(&buf_full[cw], cpar));
        cpar ^= 1u;
        if (!landed) {   // the copy never landed: record, wait once more (bounded), stop taking tiles
            if (lane == 0) give_up();
            const uint64_t t0 = dev::globaltimer();
            for (uint32_t it = 0; it < (1u << 26); ++it)
                if (mbar_try_sleep(&buf_full[cw], cpar ^ 1u, kSleepHintNs) || dev::globaltimer() - t0 > limit_ns) break;
            break;
        }
        // the scan: blocks of 512 elements from the running prefix, four
        // 128-element warp scans in the element type inside each block
        RrCarry<T> carry(excl);
        const int len = tile_len(t);
        if (len == TE) {
            const V4 *src = reinterpret_cast<const V4 *>(buf);
            V4 *dst = reinterpret_cast<V4 *>(out + tile_start(t));
#pragma unroll 1
            for (int blk = 0; blk < TE / 512; ++blk) {
                const T base = carry.base();
                T loc = T(0);
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) {
                    const int g = blk * 4 + gg;
                    const int vi = REV ? (TE - 4 - 128 * g - 4 * lane) / 4 : g * 32 + lane;
                    const V4 r4 = src[vi];
                    V4 q;
                    if (REV) { q.x = r4.w; q.y = r4.z; q.z = r4.y; q.w = r4.x; }
                    else q = r4;
                    const T s0 = q.x, s1 = s0 + q.y, s2 = s1 + q.z, s3 = s2 + q.w;
                    const T wi = dev::warp_incl_scan_add(s3);
                    T lex = __shfl_up_sync(0xffffffffu, wi, 1);
                    if (lane == 0) lex = T(0);
                    const T b = base + (loc + lex);
                    V4 o;
                    if (INCL) { o.x = b + s0; o.y = b + s1; o.z = b + s2; o.w = b + s3; }
                    else { o.x = b; o.y = b + s0; o.z = b + s1; o.w = b + s2; }
                    if (REV) { V4 r; r.x = o.w; r.y = o.z; r.z = o.y; r.w = o.x; o = r; }
                    dev::st_stream(dst + vi, o);
                    loc = loc + __shfl_sync(0xffffffffu, wi, 31);
                }
                carry.add(loc);
            }
        } else {   // a segment's partial last tile, element by element
#pragma unroll 1
            for (int blk = 0; blk * 512 < len; ++blk) {
                const T base = carry.base();
                T loc = T(0);
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) {
                    const int e = (blk * 4 + gg) * 128 + 4 * lane;
                    T x[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) x[i] = e + i < len ? in[phys(t, e + i)] : T(0);
                    const T s0 = x[0], s1 = s0 + x[1], s2 = s1 + x[2], s3 = s2 + x[3];
                    const T wi = dev::warp_incl_scan_add(s3);
                    T lex = __shfl_up_sync(0xffffffffu, wi, 1);
                    if (lane == 0) lex = T(0);
                    const T b = base + (loc + lex);
                    const T o[4] = {INCL ? b + s0 : b, INCL ? b + s1 : b + s0, INCL ? b + s2 : b + s1,
                                    INCL ? b + s3 : b + s2};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (e + i < len) out[phys(t, e + i)] = o[i];
                    loc = loc + __shfl_sync(0xffffffffu, wi, 31);
                }
                carry.add(loc);
            }
        }
        __syncwarp();   // every read of the buffer is done before its next copy
    }
}

template <class T, bool INCL, bool REV, int R, int NC>
int launch_scan_rr(const ScanLaunch &sc, cudaStream_t s)
{
    const T *in = static_cast<const T *>(sc.in);
    T *out = static_cast<T *>(sc.out);
    const int64_t seglen = sc.seg > 0 ? sc.seg : sc.n, tps = ceil_div(seglen, (int64_t)kRrTE);
    const int64_t ntiles = tps * (sc.n / seglen);
    if (ntiles > 0x7fffffffLL) return fail(SKEL_ERR_SHAPE, "scan: too many tiles");
    auto kern = seglen < sc.n ? scan_rr<T, INCL, REV, true, R, NC> : scan_rr<T, INCL, REV, false, R, NC>;
    const int dyn = (R + NC) * kRrTE * (int)sizeof(T);
    const int threads = (kRrAggW + NC) * 32;
    const int occ = kernel_occupancy(kern, threads, dyn);
    if (occ < 1) return fail(SKEL_ERR_UNSUPPORTED, "scan rr: kernel does not fit an SM");
    const int64_t grid = (int64_t)device_info().sms * occ;
    Scratch scr{};
    int rc = get_scratch(s, 0, 2 * (size_t)ntiles, &scr);
    if (rc) return rc;
    LookbackDesc d{scr.words, scr.words + ntiles};
    const DebugKnobs k = debug_knobs();
    launch_kernel(kern, (unsigned)grid, threads, (size_t)dyn, s, in, out, seglen, tps, ntiles, d, scr.ctl, scr.epoch,
                  k.scan_skip_publish_tile, k.wait_limit_ns);
    const cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "scan rr launch");
}

// tile: the ring's tiles and the scanner warps (16 KiB each, one block per
// SM): 0 = 6 + 6, 1 = 4 + 8, 2 = 6 + 8, 3 = 5 + 8.
template <class T, bool INCL, bool REV>
int run_scan_rr_dir(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.tile == 0) return launch_scan_rr<T, INCL, REV, 6, 6>(sc, s);
    if (c.tile == 1) return launch_scan_rr<T, INCL, REV, 4, 8>(sc, s);
    if (c.tile == 2) return launch_scan_rr<T, INCL, REV, 6, 8>(sc, s);
    return launch_scan_rr<T, INCL, REV, 5, 8>(sc, s);
}

template <class T, bool INCL>
int run_scan_rr(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (c.ept > 0 && c.ept != kTmaV) return fail(SKEL_ERR_INVALID_ARG, "scan rr: ept must be 4");
    if (c.tile < 0 || c.tile > 3) return fail(SKEL_ERR_INVALID_ARG, "scan rr: tile must be 0..3");
    // bulk copies start on 16-byte boundaries: aligned operands, and segments
    // of a multiple of 4 elements (reverse 1D scans: n % 4 == 0)
    const int64_t seglen = sc.seg > 0 ? sc.seg : sc.n;
    if (!aligned16(sc.in) || !aligned16(sc.out) || ((sc.seg > 0 || sc.reverse) && seglen % 4))
        return fail(SKEL_ERR_UNSUPPORTED, "scan rr: 16-byte aligned operands and segments needed");
    return sc.reverse ? run_scan_rr_dir<T, INCL, true>(sc, c, s) : run_scan_rr_dir<T, INCL, false>(sc, c, s);
}

}  // namespace

int scan_rr_launch(const ScanLaunch &sc, const Choice &c, cudaStream_t s)
{
    if (sc.dtype == SKEL_F32)
        return sc.inclusive ? run_scan_rr<float, true>(sc, c, s) : run_scan_rr<float, false>(sc, c, s);
    if (sc.dtype == SKEL_I32)
        return sc.inclusive ? run_scan_rr<uint32_t, true>(sc, c, s) : run_scan_rr<uint32_t, false>(sc, c, s);
    return fail(SKEL_ERR_DTYPE, "scan: float32 or int32 only");
}

}  // namespace skel
