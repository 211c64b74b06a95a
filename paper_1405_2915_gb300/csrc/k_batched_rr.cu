// Batched variant 7 (the dispatch and the other variants are in
// k_batched.cu): the flat segmented scan run by aggregator warps and
// re-reading scanner warps.
#include "batched_flat.cuh"

namespace skel {
namespace {

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

}  // namespace

int batched_rr_launch(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
                      uint32_t epoch, cudaStream_t s)
{
    return run_br(b, c, ctl, words, data, epoch, s);
}

}  // namespace skel
