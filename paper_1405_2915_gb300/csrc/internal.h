// Internal declarations of libskel.so shared by the host runtime (api.cpp)
// and the kernel translation units (k_*.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "skel.h"

namespace skel {

// ----------------------------------------------------------------- errors --
// Sets the thread-local message returned by skel_last_error and returns code.
int fail(int code, const std::string &msg);
int fail_cuda(cudaError_t e, const char *what);

#define SKEL_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return ::skel::fail_cuda(e_, #expr); \
    } while (0)

// Process-wide count of kernel launches made by the library.
void note_launch();
int64_t launch_count();

// ---------------------------------------------------------------- device --
struct DeviceInfo {
    int device;
    int sms;                  // multiprocessor count (152 on GB300)
    int max_smem_optin;       // bytes of shared memory a block may opt into
    size_t l2_bytes;
};
const DeviceInfo &device_info();  // of the current device

// Opts kern in to dyn bytes of dynamic shared memory and returns its resident
// blocks per SM at that size (0 or less: it does not fit), set up once per
// kernel, block size and device, so that no host query sits between the
// launches of a call.
template <class K>
int kernel_occupancy(K kern, int threads, int dyn)
{
    struct Entry {
        const void *k;
        int dev, threads, dyn, occ;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry &e : cache)
        if (e.k == reinterpret_cast<const void *>(kern) && e.dev == dev && e.threads == threads && e.dyn == dyn)
            return e.occ;
    int occ = 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, dyn);
    if (e != cudaSuccess) {
        cudaGetLastError();
        occ = -1;
    }
    cache.push_back(Entry{reinterpret_cast<const void *>(kern), dev, threads, dyn, occ});
    return occ;
}

// ------------------------------------------------------- scratch memory --
// Layout of a scratch block: a 256-byte control block, a region of look-back
// descriptor words, then the data region.  Kernels leave the control counters
// at zero when they finish.  The word region holds nothing but self-validating
// look-back words tagged with a call's epoch (1..255), so a stale word can
// only carry an older epoch; the region is cleared when the epoch wraps.
struct Control {
    uint32_t ticket;     // tile ticket counter (single-pass scan, batched)
    uint32_t done;       // blocks finished (single-pass reduce)
    uint32_t error;      // device-side status bits (kErrTimeout)
    uint32_t abort;      // epoch of a call whose bounded wait gave up; its other waiters stop
    uint32_t queue;      // work queue of persistent kernels
    uint32_t exited;     // persistent blocks that left the work loop
    uint32_t epoch;      // last look-back tag of a kernel that keeps its tag on the device (0: none yet)
    uint32_t pad[57];
};
static_assert(sizeof(Control) == 256, "control block is 256 bytes");
constexpr uint32_t kErrTimeout = 1u;   // a bounded wait gave up
constexpr uint32_t kErrInput = 2u;     // device-resident input failed validation (batched offsets)

struct Scratch {
    Control *ctl;        // device address of the control block
    uint64_t *words;     // look-back descriptor words (word_count requested)
    unsigned char *data; // device address of the data region (256-byte aligned)
    size_t data_bytes;
    uint32_t epoch;      // tag of this call's look-back words, 1..255
};
constexpr uint32_t kMaxEpoch = 255;

// Returns scratch for `stream` with at least `data_bytes` of data region and
// `word_count` descriptor words.  Scratch is cached per (device, stream) and
// reused by later calls on the same stream (stream order serialises them).
// A call asking for words gets a fresh epoch (the words are cleared when the
// epoch counter wraps or the region grows).
int get_scratch(cudaStream_t stream, size_t data_bytes, size_t word_count, Scratch *out);

// Control block of the scratch of `stream`, or nullptr if none was made.
Control *scratch_control(cudaStream_t stream);
int release_scratch();
// Device status bits recorded by the allocation-free scan on the current
// device (its control block lives in a static array, not in a stream's
// scratch); *err = 0 if that entry point never ran on this device.  Clears
// them.  Synchronous.
int noalloc_take_status(uint32_t *err);
// Fixed 256-byte device buffer of `stream` for scalar results.
int result_slot(cudaStream_t stream, void **out);

// Allocation through the active allocator; free_dev must be given the same
// allocator record that allocated.
struct Allocator {
    void *(*alloc)(size_t, void *, void *);
    void (*free_fn)(void *, void *, void *);
    void *ctx;
};
Allocator current_allocator();
void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t stream);
void dev_free(const Allocator &a, void *p, cudaStream_t stream);

// ------------------------------------------------------------- debugging --
struct DebugKnobs {
    int64_t scan_skip_publish_tile;  // -1: off
    uint64_t wait_limit_ns;          // bounded-wait limit
};
DebugKnobs debug_knobs();
int set_debug(int key, int64_t value);

// --------------------------------------------------------------- dispatch --
struct Choice {
    int variant;
    int block;
    int ept;
    int tile;
};

// Context of a call (the key of the execution-plan table).
struct Context {
    int skeleton;
    int fn;
    int dtype;
    int64_t n;
    int radius;
    int residency;  // 0: operands device-valid; 1: at least one needs a host->device copy
};

int bucket_of(int64_t n);
// Table lookup with nearest-bucket extrapolation; falls back to the
// skeleton's built-in default.  Honors skel_force_variant.  *forced is set
// when the choice came from a force.
Choice select_variant(const Context &ctx, bool *forced);
void record_last(int skeleton, const Choice &c);
int last_choice(int skeleton, Choice *c);
int force_variant(int skeleton, const Choice &c);
int dispatch_set(int sk, int fn, int dt, int bucket, int radius, int res, const Choice &c);
int dispatch_size();
int dispatch_load(const char *path);
Choice skeleton_default(int skeleton);
void set_allocator(const Allocator &a);
const char *last_error_cstr();
void clear_error();

// ------------------------------------------------------ kernel launchers --
// Each launcher validates its own selectability constraint: it returns
// SKEL_ERR_UNSUPPORTED (with a message) when the chosen variant cannot run
// this call, so that the caller can fall back to the default variant.

struct MapLaunch {
    int fn;
    float a;
    const float *in0;
    const float *in1;
    float *out;
    int64_t n;
    bool alias = false;  // out is in0 or in1 (in place): no restrict, coherent loads
};
int launch_map(const MapLaunch &m, const Choice &c, cudaStream_t s);
int map_variant_count();
const char *map_variant_name(int v);
Choice map_default();

struct ReduceLaunch {
    int op;         // SKEL_FN_ADD / SKEL_FN_MAX
    int map_fn;     // -1 (plain reduce), SKEL_FN_MUL, SKEL_FN_SQ
    int dtype;      // SKEL_F32 / SKEL_I32
    const void *in0;
    const void *in1;
    void *out;      // device address of the 1-element result
    int64_t n;
};
int launch_reduce(const ReduceLaunch &r, const Choice &c, cudaStream_t s);
int reduce_variant_count();
const char *reduce_variant_name(int v);
Choice reduce_default();

struct ScanLaunch {
    int dtype;      // SKEL_F32 / SKEL_I32
    bool inclusive;
    bool reverse;   // scan from the end (the adjoint of scan)
    const void *in;
    void *out;
    int64_t n;      // total elements
    int64_t seg;    // segment length for row-wise scans (0: one segment)
};
int launch_scan(const ScanLaunch &sc, const Choice &c, cudaStream_t s);
int scan_rr_launch(const ScanLaunch &sc, const Choice &c, cudaStream_t s);   // variant 8 (k_scan_rr.cu)
int scan_variant_count();
const char *scan_variant_name(int v);
Choice scan_default();

struct StencilLaunch {
    int ndim;            // 1 or 2
    int radius;
    int boundary;
    const float *w;      // host copy of weights: 2r+1 (1D) or 9 (2D, row-major 3x3)
    int taps5;           // 2D: 1 if the 5-point cross (corner weights ignored)
    const float *in;
    float *out;
    int64_t rows, cols;  // 1D: rows = 1, cols = n
    bool transpose;      // adjoint (mirrored weights, clamp folding)
};
int launch_stencil(const StencilLaunch &st, const Choice &c, cudaStream_t s);
// `steps` applications of a 2D forward stencil fused tile-wise, c.tile steps
// per pass (ping-pong between st.out and tmp, the last pass writes st.out).
int launch_stencil_chain_fused(const StencilLaunch &st, int steps, float *tmp, const Choice &c, cudaStream_t s);
int chain_variant_count();
const char *chain_variant_name(int v);
Choice chain_default();
int stencil_variant_count(int ndim);
const char *stencil_variant_name(int ndim, int v);
Choice stencil_default(int ndim);

// The composed chain Map -> MapOverlap (2D, radius 1) -> MapReduce(sq, +),
// fused into one pass over x (variant 1 of SKEL_SK_COMPOSE).
struct ComposeLaunch {
    int map_fn;          // SKEL_FN_TANH / SQ / SCALE / COPY
    float a;             // the map's parameter (SCALE)
    int boundary;
    const float *w;      // 9 weights, host copy (row-major 3x3)
    int taps5;
    const float *in;
    int64_t rows, cols;
};
// Checks the fused variant's constraints; *nparts: the partial sums it writes.
int compose_fused_check(const ComposeLaunch &cl, const Choice &c, int64_t *nparts);
int launch_compose_fused(const ComposeLaunch &cl, const Choice &c, float *partials, cudaStream_t s);
int compose_variant_count();
const char *compose_variant_name(int v);
Choice compose_default();

// MapArray over a grid (fn COULOMB): atoms (m x 4 float32: x, y, z, q),
// out rows x cols, grid position of out[i, j] = (j*h, i*h, z0).
struct CoulombLaunch {
    const float *atoms;
    int64_t m;
    float *out;
    int64_t rows, cols;
    float h, z0;
};
int launch_coulomb(const CoulombLaunch &cl, const Choice &c, cudaStream_t s);

struct MapArrayLaunch {
    int fn;              // SKEL_FN_GATHER / SKEL_FN_ROWDOT
    const float *A;
    int64_t m;
    const void *B;       // int32 indices (gather) or float rows n x m (rowdot)
    float *out;
    int64_t n;
};
int launch_maparray(const MapArrayLaunch &ma, const Choice &c, cudaStream_t s);
int maparray_variant_count();
const char *maparray_variant_name(int v);
Choice maparray_default();

struct BatchedLaunch {
    bool want_reduce;
    bool want_scan;
    bool inclusive;
    const float *values;
    const int64_t *offsets;   // B+1 entries (device)
    int64_t B;
    int64_t total;            // offsets[B] (host-known length of values)
    float *results;           // B (may be NULL)
    float *scan_out;          // total (may be NULL)
};
// Scratch the batched launch needs for this call: data bytes and look-back
// descriptor words (upper bounds from the total length and the instance
// count; the plan allocates them itself, the direct call uses the stream's
// scratch).
size_t batched_data_bytes(const BatchedLaunch &b, const Choice &c);
// The flat segmented batched variants: 6 (k_batched_seg.cu; elements per
// tile of a tile shape, and the call's launches) and 7 (k_batched_rr.cu).
int batched_seg_tile(int tile);
int batched_seg_launch(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
                       uint32_t epoch, cudaStream_t s);
int batched_rr_launch(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words, unsigned char *data,
                      uint32_t epoch, cudaStream_t s);
size_t batched_word_count(const BatchedLaunch &b, const Choice &c);
int launch_batched(const BatchedLaunch &b, const Choice &c, Control *ctl, uint64_t *words,
                   unsigned char *data, uint32_t epoch, cudaStream_t s);
int batched_variant_count();
const char *batched_variant_name(int v);
Choice batched_default();

// Backward helpers (elementwise adjoints and broadcasts).
struct MapBwdLaunch {
    int fn;
    float a;
    int tanh_from_output;
    const float *in0;
    const float *in1;
    const float *g;      // per-element upstream gradient (NULL: use *g_scalar)
    const float *g2;     // a second per-element upstream gradient added to g, or NULL
    const float *g_scalar_dev;  // device scalar (mapreduce/reduce adjoint), or NULL
    float g_scalar_host;
    float *gin0;
    float *gin1;
    int64_t n;
};
int launch_map_bwd(const MapBwdLaunch &m, cudaStream_t s);

// Measurement probes (k_probe.cu): empty launches back to back, and random
// 4-byte reads from an L2-resident table of m (a power of two) floats; the
// number of reads the latter makes for a request is probe_l2_random_reads.
int probe_launch_empty(int count, cudaStream_t s);
int probe_launch_l2_random(const float *table, int64_t m, int64_t reads, float *sink, cudaStream_t s);
int64_t probe_l2_random_reads(int64_t reads);

}  // namespace skel
