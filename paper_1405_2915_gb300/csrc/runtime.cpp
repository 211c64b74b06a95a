// Host runtime of libskel.so: error reporting, device properties, the
// allocator hook, per-stream scratch memory, and the execution-plan table
// that maps a call context to an implementation variant (Sec. II off-line
// tuned dispatch; Sec. III execution plans).
#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace skel {

// ------------------------------------------------------------------ errors --
static thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int fail_cuda(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SKEL_ERR_CUDA;
}

const char *last_error_cstr() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

// ---------------------------------------------------------------- launches --
static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ device --
const DeviceInfo &device_info()
{
    static std::mutex mu;
    static std::map<int, DeviceInfo> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    DeviceInfo d{};
    d.device = dev;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    d.sms = v > 0 ? v : 1;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    d.max_smem_optin = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
    d.l2_bytes = (size_t)v;
    return cache.emplace(dev, d).first->second;
}

// --------------------------------------------------------------- allocator --
static std::mutex g_alloc_mu;
static Allocator g_alloc{nullptr, nullptr, nullptr};

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

void set_allocator(const Allocator &a)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = a;
}

// The built-in allocator draws from a memory pool of the library's own on
// each device, with no release threshold: what a call frees stays with the
// pool for the next call.  (The device's default pool hands freed memory
// back at every synchronisation, so a call with large temporaries, such as
// the per-call composed chain, would have them mapped again each time.)
// skel_release_cached() returns the pools' unused memory.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaMemPool_t own_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t stream)
{
    if (bytes == 0) bytes = 256;
    if (a.alloc) return a.alloc(bytes, (void *)stream, a.ctx);
    void *p = nullptr;
    cudaMemPool_t pool = own_pool();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, stream) : cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(const Allocator &a, void *p, cudaStream_t stream)
{
    if (!p) return;
    if (a.alloc) {
        if (a.free_fn) a.free_fn(p, (void *)stream, a.ctx);
        return;
    }
    cudaFreeAsync(p, stream);
}

// ----------------------------------------------------------------- scratch --
namespace {
struct ScratchBlock {
    void *base = nullptr;
    size_t word_cap = 0;    // 64-bit look-back words
    size_t data_cap = 0;    // bytes
    uint32_t epoch = 0;
    Allocator alloc{};
};
std::mutex g_scr_mu;
std::map<std::pair<int, cudaStream_t>, ScratchBlock> g_scratch;

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

int get_scratch(cudaStream_t stream, size_t data_bytes, size_t word_count, Scratch *out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_scr_mu);
    ScratchBlock &b = g_scratch[{dev, stream}];
    const bool grow = !b.base || data_bytes > b.data_cap || word_count > b.word_cap;
    if (grow) {
        size_t wc = std::max(word_count, b.word_cap);
        size_t dc = std::max(data_bytes, b.data_cap);
        // grow geometrically so that a size sweep does not reallocate each call
        if (b.base) {
            wc = std::max(wc, b.word_cap + b.word_cap / 2);
            dc = std::max(dc, b.data_cap + b.data_cap / 2);
        }
        wc = std::max<size_t>(round256(wc * 8) / 8, 32);
        dc = std::max<size_t>(round256(dc), 256);
        if (b.base) dev_free(b.alloc, b.base, stream);
        b.alloc = current_allocator();
        const size_t total = sizeof(Control) + wc * 8 + dc;
        b.base = dev_alloc(b.alloc, total, stream);
        if (!b.base) {
            b = ScratchBlock{};
            return fail(SKEL_ERR_OOM, "scratch allocation failed");
        }
        b.word_cap = wc;
        b.data_cap = dc;
        b.epoch = 0;
        cudaError_t e = cudaMemsetAsync(b.base, 0, total, stream);
        if (e != cudaSuccess) return fail_cuda(e, "scratch clear");
    }
    unsigned char *base = static_cast<unsigned char *>(b.base);
    out->ctl = reinterpret_cast<Control *>(base);
    out->words = reinterpret_cast<uint64_t *>(base + sizeof(Control));
    out->data = base + sizeof(Control) + b.word_cap * 8;
    out->data_bytes = b.data_cap;
    if (word_count > 0) {
        b.epoch += 1;
        if (b.epoch > kMaxEpoch) {   // tag space used up: clear every word and the abort tag, restart
            b.epoch = 1;
            cudaError_t e = cudaMemsetAsync(out->words, 0, b.word_cap * 8, stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(&out->ctl->abort, 0, sizeof(uint32_t), stream);
            if (e != cudaSuccess) return fail_cuda(e, "look-back word clear");
        }
    }
    out->epoch = b.epoch == 0 ? 1 : b.epoch;
    return SKEL_OK;
}

// A small device buffer per (device, stream) that receives scalar results
// (reduce / mapreduce without a result container).  Allocated once, never
// moved, so a launch can hold its address.
static std::map<std::pair<int, cudaStream_t>, std::pair<void *, Allocator>> g_slots;

int result_slot(cudaStream_t stream, void **out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_scr_mu);
    auto &e = g_slots[{dev, stream}];
    if (!e.first) {
        e.second = current_allocator();
        e.first = dev_alloc(e.second, 256, stream);
        if (!e.first) return fail(SKEL_ERR_OOM, "result slot allocation failed");
    }
    *out = e.first;
    return SKEL_OK;
}

// Device-side status words of the scratch of `stream` (current device), or
// nullptr if the stream never used scratch.
Control *scratch_control(cudaStream_t stream)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_scr_mu);
    auto it = g_scratch.find({dev, stream});
    if (it == g_scratch.end() || !it->second.base) return nullptr;
    return reinterpret_cast<Control *>(it->second.base);
}

int release_scratch()
{
    std::lock_guard<std::mutex> lk(g_scr_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_scratch) {
        if (!kv.second.base) continue;
        cudaSetDevice(kv.first.first);
        cudaStreamSynchronize(kv.first.second);
        dev_free(kv.second.alloc, kv.second.base, kv.first.second);
    }
    for (auto &kv : g_slots) {
        if (!kv.second.first) continue;
        cudaSetDevice(kv.first.first);
        cudaStreamSynchronize(kv.first.second);
        dev_free(kv.second.second, kv.second.first, kv.first.second);
    }
    cudaSetDevice(cur);
    g_scratch.clear();
    g_slots.clear();
    std::lock_guard<std::mutex> lp(g_pool_mu);
    for (cudaMemPool_t pool : g_pool)
        if (pool) cudaMemPoolTrimTo(pool, 0);   // memory no allocation holds goes back
    return SKEL_OK;
}

// ------------------------------------------------------------------- debug --
static std::mutex g_dbg_mu;
static DebugKnobs g_dbg{-1, 2000000000ull};

DebugKnobs debug_knobs()
{
    std::lock_guard<std::mutex> lk(g_dbg_mu);
    return g_dbg;
}

int set_debug(int key, int64_t value)
{
    std::lock_guard<std::mutex> lk(g_dbg_mu);
    if (key == 1) { g_dbg.scan_skip_publish_tile = value; return SKEL_OK; }
    if (key == 2) {
        if (value <= 0) return fail(SKEL_ERR_INVALID_ARG, "wait limit must be positive");
        g_dbg.wait_limit_ns = (uint64_t)value * 1000ull;
        return SKEL_OK;
    }
    return fail(SKEL_ERR_INVALID_ARG, "unknown debug key");
}

// ---------------------------------------------------------------- dispatch --
namespace {
constexpr int kBuckets = 16;

struct GroupKey {
    int sk, fn, dt, radius, res;
    bool operator<(const GroupKey &o) const
    {
        return std::tie(sk, fn, dt, radius, res) < std::tie(o.sk, o.fn, o.dt, o.radius, o.res);
    }
};
struct Group {
    std::array<Choice, kBuckets> e;
    std::array<bool, kBuckets> present{};
};

std::mutex g_tab_mu;
std::map<GroupKey, Group> g_table;
std::array<Choice, SKEL_SK_COUNT> g_force = [] {
    std::array<Choice, SKEL_SK_COUNT> a;
    for (auto &c : a) c = Choice{-1, 0, 0, 0};
    return a;
}();
thread_local std::array<Choice, SKEL_SK_COUNT> t_last = [] {
    std::array<Choice, SKEL_SK_COUNT> a;
    for (auto &c : a) c = Choice{-1, -1, -1, -1};
    return a;
}();

Choice builtin_default(int sk)
{
    switch (sk) {
    case SKEL_SK_MAP: return map_default();
    case SKEL_SK_REDUCE:
    case SKEL_SK_MAPREDUCE: return reduce_default();
    case SKEL_SK_SCAN: return scan_default();
    case SKEL_SK_MAPOVERLAP1D: return stencil_default(1);
    case SKEL_SK_MAPOVERLAP2D: return stencil_default(2);
    case SKEL_SK_MAPARRAY: return maparray_default();
    case SKEL_SK_BATCHED: return batched_default();
    case SKEL_SK_CHAIN2D: return chain_default();
    case SKEL_SK_COMPOSE: return compose_default();
    default: return Choice{0, 0, 0, 0};
    }
}
}  // namespace

Choice skeleton_default(int sk) { return builtin_default(sk); }

int bucket_of(int64_t n)
{
    if (n <= 1) return 0;
    int l = 63 - __builtin_clzll((unsigned long long)n);   // floor(log2 n)
    int b = l / 2;
    return b < kBuckets ? b : kBuckets - 1;
}

Choice select_variant(const Context &ctx, bool *forced)
{
    std::lock_guard<std::mutex> lk(g_tab_mu);
    *forced = false;
    if (ctx.skeleton >= 0 && ctx.skeleton < SKEL_SK_COUNT && g_force[ctx.skeleton].variant >= 0) {
        *forced = true;
        return g_force[ctx.skeleton];
    }
    auto it = g_table.find(GroupKey{ctx.skeleton, ctx.fn, ctx.dtype, ctx.radius, ctx.residency});
    if (it == g_table.end() && ctx.residency != 0)   // untuned residency: use the device-resident plan
        it = g_table.find(GroupKey{ctx.skeleton, ctx.fn, ctx.dtype, ctx.radius, 0});
    if (it != g_table.end()) {
        const Group &g = it->second;
        const int b = bucket_of(ctx.n);
        // an entry with variant -1 records that the built-in default won there
        auto pick = [&](int k) { return g.e[k].variant < 0 ? builtin_default(ctx.skeleton) : g.e[k]; };
        if (g.present[b]) return pick(b);
        for (int k = b - 1; k >= 0; --k) if (g.present[k]) return pick(k);   // extrapolate upward
        for (int k = b + 1; k < kBuckets; ++k) if (g.present[k]) return pick(k);
    }
    return builtin_default(ctx.skeleton);
}

void record_last(int sk, const Choice &c)
{
    if (sk >= 0 && sk < SKEL_SK_COUNT) t_last[sk] = c;
}

int last_choice(int sk, Choice *c)
{
    if (sk < 0 || sk >= SKEL_SK_COUNT) return fail(SKEL_ERR_INVALID_ARG, "unknown skeleton");
    *c = t_last[sk];
    return SKEL_OK;
}

int force_variant(int sk, const Choice &c)
{
    if (sk < 0 || sk >= SKEL_SK_COUNT) return fail(SKEL_ERR_INVALID_ARG, "unknown skeleton");
    std::lock_guard<std::mutex> lk(g_tab_mu);
    g_force[sk] = c.variant < 0 ? Choice{-1, 0, 0, 0} : c;
    return SKEL_OK;
}

int dispatch_set(int sk, int fn, int dt, int bucket, int radius, int res, const Choice &c)
{
    if (sk < 0 || sk >= SKEL_SK_COUNT) return fail(SKEL_ERR_INVALID_ARG, "unknown skeleton");
    if (bucket < 0 || bucket >= kBuckets) return fail(SKEL_ERR_INVALID_ARG, "bucket out of range");
    if (c.variant < -1) return fail(SKEL_ERR_INVALID_ARG, "variant must be >= 0, or -1 for the built-in default");
    std::lock_guard<std::mutex> lk(g_tab_mu);
    Group &g = g_table[GroupKey{sk, fn, dt, radius, res}];
    g.e[bucket] = c;
    g.present[bucket] = true;
    return SKEL_OK;
}

int dispatch_size()
{
    std::lock_guard<std::mutex> lk(g_tab_mu);
    int n = 0;
    for (auto &kv : g_table)
        for (bool p : kv.second.present) n += p;
    return n;
}

int dispatch_load(const char *path)
{
    if (!path) {
        std::lock_guard<std::mutex> lk(g_tab_mu);
        g_table.clear();
        return SKEL_OK;
    }
    std::ifstream f(path);
    if (!f) return fail(SKEL_ERR_TABLE, std::string("cannot open dispatch table ") + path);
    std::map<GroupKey, Group> fresh;
    std::string line;
    int lineno = 0;
    while (std::getline(f, line)) {
        ++lineno;
        size_t h = line.find('#');
        if (h != std::string::npos) line.resize(h);
        std::istringstream ss(line);
        int v[10];
        int k = 0;
        while (k < 10 && (ss >> v[k])) ++k;
        if (k == 0) continue;
        std::string extra;
        if (k != 10 || (ss >> extra))
            return fail(SKEL_ERR_TABLE, std::string(path) + ":" + std::to_string(lineno) +
                                            ": expected 10 integers");
        if (v[0] < 0 || v[0] >= SKEL_SK_COUNT || v[3] < 0 || v[3] >= kBuckets || v[6] < -1)
            return fail(SKEL_ERR_TABLE, std::string(path) + ":" + std::to_string(lineno) +
                                            ": field out of range");
        Group &g = fresh[GroupKey{v[0], v[1], v[2], v[4], v[5]}];
        g.e[v[3]] = Choice{v[6], v[7], v[8], v[9]};
        g.present[v[3]] = true;
    }
    std::lock_guard<std::mutex> lk(g_tab_mu);
    for (auto &kv : fresh) {
        Group &g = g_table[kv.first];
        for (int b = 0; b < kBuckets; ++b)
            if (kv.second.present[b]) { g.e[b] = kv.second.e[b]; g.present[b] = true; }
    }
    return SKEL_OK;
}

}  // namespace skel
