// C ABI of libskel.so: smart containers (Sec. IV) and the skeleton entry
// points (Sec. III), each routed through the execution-plan table to one of
// its CUDA variants.  See include/skel.h for the contract of every function.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace skel;

// ----------------------------------------------------------- containers --
namespace {

size_t dtype_size(int dt)
{
    switch (dt) {
    case SKEL_F32: return 4;
    case SKEL_I32: return 4;
    case SKEL_I64: return 8;
    default: return 0;
    }
}

// Storage shared by a container and its views, with the coherence state.
struct Storage {
    int refs = 1;
    size_t bytes = 0;
    void *host = nullptr;
    bool host_owned = false;
    void *dev = nullptr;
    bool dev_owned = false;
    Allocator dev_alloc_rec{};
    int device = -1;
    int valid = 0;                    // bits of skel_unit holding a valid copy
    cudaStream_t last_stream = nullptr;
    bool used_on_device = false;      // some device work on the storage was enqueued
    int direct_reads = 0;             // device reads of the host copy in place since it was last written
    int64_t h2d_count = 0, d2h_count = 0, h2d_bytes = 0, d2h_bytes = 0;
};

}  // namespace

struct skel_container_s {
    Storage *st;
    int dtype;
    int ndim;
    int64_t shape[2];
    int64_t n;
    size_t offset;   // bytes from the storage start
    int views;       // live views of this container
    skel_container_s *parent;
};

namespace {

int coherence_step(int valid, int unit, int mode, int *nv, int *transfer)
{
    const int other = unit == SKEL_UNIT_HOST ? SKEL_UNIT_DEVICE : SKEL_UNIT_HOST;
    int t = 0;
    if (mode & SKEL_READ) {
        if (!(valid & unit) && (valid & other)) {
            t = unit == SKEL_UNIT_DEVICE ? 1 : 2;
            valid |= unit;
        }
    }
    if (mode & SKEL_WRITE) valid = unit;
    *nv = valid;
    *transfer = t;
    return SKEL_OK;
}

bool valid_handle(skel_handle h) { return h && h->st && h->st->refs > 0; }

int check_shape(int ndim, const int64_t *shape, int64_t *n)
{
    if (ndim != 1 && ndim != 2) return fail(SKEL_ERR_SHAPE, "ndim must be 1 or 2");
    if (!shape) return fail(SKEL_ERR_INVALID_ARG, "shape is NULL");
    int64_t t = 1;
    for (int d = 0; d < ndim; ++d) {
        if (shape[d] < 0) return fail(SKEL_ERR_SHAPE, "negative extent");
        if (shape[d] && t > INT64_MAX / shape[d]) return fail(SKEL_ERR_SHAPE, "size overflow");
        t *= shape[d];
    }
    *n = t;
    return SKEL_OK;
}

// Makes `s` wait for the storage's earlier device work if it was enqueued
// on another stream (dependence tracking, Sec. IV).
int order_after_last_use(Storage *st, cudaStream_t s)
{
    if (!st->used_on_device || st->last_stream == s) return SKEL_OK;
    cudaEvent_t ev;
    SKEL_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, st->last_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return fail_cuda(e, "cross-stream ordering");
    return SKEL_OK;
}

// Device access of a container: lazy host->device copy (Sec. IV).
int acquire_device(skel_handle h, int mode, cudaStream_t s, void **ptr)
{
    Storage *st = h->st;
    int dev = 0;
    cudaGetDevice(&dev);
    if (st->dev && st->device >= 0 && st->device != dev)
        return fail(SKEL_ERR_INVALID_ARG, "container device memory belongs to another device");
    if (!st->dev) {
        st->dev_alloc_rec = current_allocator();
        st->dev = dev_alloc(st->dev_alloc_rec, st->bytes, s);
        if (!st->dev) return fail(SKEL_ERR_OOM, "device allocation of container failed");
        st->dev_owned = true;
        st->device = dev;
    }
    if (st->device < 0) st->device = dev;
    int rc = order_after_last_use(st, s);
    if (rc) return rc;
    int nv, tr;
    coherence_step(st->valid, SKEL_UNIT_DEVICE, mode, &nv, &tr);
    if (tr == 1) {
        SKEL_CUDA_TRY(cudaMemcpyAsync(st->dev, st->host, st->bytes, cudaMemcpyHostToDevice, s));
        st->h2d_count += 1;
        st->h2d_bytes += (int64_t)st->bytes;
    }
    st->valid = nv;
    st->last_stream = s;
    st->used_on_device = true;
    *ptr = static_cast<char *>(st->dev) + h->offset;
    return SKEL_OK;
}

// Host access: waits for device work, lazy device->host copy (Sec. IV).
int acquire_host(skel_handle h, int mode, cudaStream_t s, void **ptr)
{
    Storage *st = h->st;
    if (!st->host) {
        SKEL_CUDA_TRY(cudaMallocHost(&st->host, st->bytes ? st->bytes : 1));
        st->host_owned = true;
    }
    if (st->used_on_device) SKEL_CUDA_TRY(cudaStreamSynchronize(st->last_stream));
    int nv, tr;
    coherence_step(st->valid, SKEL_UNIT_HOST, mode, &nv, &tr);
    if (mode & SKEL_WRITE) st->direct_reads = 0;
    if (tr == 2) {
        SKEL_CUDA_TRY(cudaMemcpyAsync(st->host, st->dev, st->bytes, cudaMemcpyDeviceToHost, s));
        SKEL_CUDA_TRY(cudaStreamSynchronize(s));
        st->d2h_count += 1;
        st->d2h_bytes += (int64_t)st->bytes;
    }
    st->valid = nv;
    *ptr = static_cast<char *>(st->host) + h->offset;
    return SKEL_OK;
}

bool device_valid(skel_handle h) { return (h->st->valid & SKEL_UNIT_DEVICE) != 0; }

struct ErrorScope {
    ErrorScope() { clear_error(); }
};

template <class F>
int guarded(F f)
{
    clear_error();
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return fail(SKEL_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SKEL_ERR_INVALID_ARG, "unexpected exception");
    }
}

}  // namespace

// ------------------------------------------------------------- C entry --
extern "C" {

const char *skel_version(void) { return "libskel 1.0 (sm_103a)"; }

const char *skel_last_error(void) { return last_error_cstr(); }

int skel_set_allocator(void *(*alloc)(size_t, void *, void *), void (*free_fn)(void *, void *, void *),
                       void *ctx)
{
    return guarded([&] {
        if (alloc && !free_fn) return fail(SKEL_ERR_INVALID_ARG, "free function required");
        set_allocator(Allocator{alloc, alloc ? free_fn : nullptr, alloc ? ctx : nullptr});
        return (int)SKEL_OK;
    });
}

int skel_release_cached(void) { return guarded([&] { return release_scratch(); }); }

int64_t skel_launch_count(void) { return launch_count(); }

int skel_coherence_step(int valid_units, int unit, int mode, int *new_valid, int *transfer)
{
    return guarded([&] {
        if (!new_valid || !transfer) return fail(SKEL_ERR_INVALID_ARG, "NULL out-parameter");
        if (valid_units & ~3) return fail(SKEL_ERR_INVALID_ARG, "valid set has unknown bits");
        if (unit != SKEL_UNIT_HOST && unit != SKEL_UNIT_DEVICE) return fail(SKEL_ERR_INVALID_ARG, "unknown unit");
        if (mode < 1 || mode > 3) return fail(SKEL_ERR_INVALID_ARG, "unknown access mode");
        return coherence_step(valid_units, unit, mode, new_valid, transfer);
    });
}

int skel_container_create(skel_dtype dtype, int ndim, const int64_t *shape, skel_handle *out)
{
    return guarded([&] {
        if (!out) return fail(SKEL_ERR_INVALID_ARG, "out is NULL");
        if (!dtype_size(dtype)) return fail(SKEL_ERR_DTYPE, "unknown dtype");
        int64_t n;
        int rc = check_shape(ndim, shape, &n);
        if (rc) return rc;
        Storage *st = new Storage();
        st->bytes = (size_t)n * dtype_size(dtype);
        auto *h = new skel_container_s{st, dtype, ndim, {shape[0], ndim == 2 ? shape[1] : 1}, n, 0, 0, nullptr};
        *out = h;
        return (int)SKEL_OK;
    });
}

int skel_container_wrap(skel_dtype dtype, int ndim, const int64_t *shape, void *host_ptr, void *dev_ptr,
                        int valid_units, skel_handle *out)
{
    return guarded([&] {
        if (!out) return fail(SKEL_ERR_INVALID_ARG, "out is NULL");
        if (!dtype_size(dtype)) return fail(SKEL_ERR_DTYPE, "unknown dtype");
        if (valid_units & ~3) return fail(SKEL_ERR_INVALID_ARG, "valid_units has unknown bits");
        int64_t n;
        int rc = check_shape(ndim, shape, &n);
        if (rc) return rc;
        if (n > 0 && (valid_units & SKEL_UNIT_HOST) && !host_ptr)
            return fail(SKEL_ERR_INVALID_ARG, "host marked valid without a host pointer");
        if (n > 0 && (valid_units & SKEL_UNIT_DEVICE) && !dev_ptr)
            return fail(SKEL_ERR_INVALID_ARG, "device marked valid without a device pointer");
        Storage *st = new Storage();
        st->bytes = (size_t)n * dtype_size(dtype);
        st->host = host_ptr;
        st->dev = dev_ptr;
        st->valid = valid_units;
        if (dev_ptr) {
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, dev_ptr) == cudaSuccess && a.type == cudaMemoryTypeDevice)
                st->device = a.device;
            else
                cudaGetLastError();
        }
        auto *h = new skel_container_s{st, dtype, ndim, {shape[0], ndim == 2 ? shape[1] : 1}, n, 0, 0, nullptr};
        *out = h;
        return (int)SKEL_OK;
    });
}

int skel_container_view(skel_handle parent, int64_t offset, int ndim, const int64_t *shape, skel_handle *out)
{
    return guarded([&] {
        if (!valid_handle(parent) || !out) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        int64_t n;
        int rc = check_shape(ndim, shape, &n);
        if (rc) return rc;
        if (offset < 0 || offset > parent->n || n > parent->n - offset) return fail(SKEL_ERR_SHAPE, "view out of range");
        parent->st->refs += 1;
        parent->views += 1;
        auto *h = new skel_container_s{parent->st, parent->dtype, ndim, {shape[0], ndim == 2 ? shape[1] : 1}, n,
                                       parent->offset + (size_t)offset * dtype_size(parent->dtype), 0, parent};
        *out = h;
        return (int)SKEL_OK;
    });
}

int skel_container_host_ptr(skel_handle h, int mode, void *stream, void **ptr)
{
    return guarded([&] {
        if (!valid_handle(h) || !ptr) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (mode < 1 || mode > 3) return fail(SKEL_ERR_INVALID_ARG, "unknown access mode");
        return acquire_host(h, mode, (cudaStream_t)stream, ptr);
    });
}

int skel_container_device_ptr(skel_handle h, int mode, void *stream, void **ptr)
{
    return guarded([&] {
        if (!valid_handle(h) || !ptr) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (mode < 1 || mode > 3) return fail(SKEL_ERR_INVALID_ARG, "unknown access mode");
        return acquire_device(h, mode, (cudaStream_t)stream, ptr);
    });
}

int skel_container_mark(skel_handle h, int units)
{
    return guarded([&] {
        if (!valid_handle(h)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (units & ~3) return fail(SKEL_ERR_INVALID_ARG, "unknown unit bits");
        if ((units & SKEL_UNIT_HOST) && !h->st->host) return fail(SKEL_ERR_INVALID_ARG, "no host copy exists");
        if ((units & SKEL_UNIT_DEVICE) && !h->st->dev) return fail(SKEL_ERR_INVALID_ARG, "no device copy exists");
        h->st->valid = units;
        h->st->direct_reads = 0;
        return (int)SKEL_OK;
    });
}

int skel_container_prefetch(skel_handle h, int unit, void *stream)
{
    return guarded([&] {
        if (!valid_handle(h)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (unit != SKEL_UNIT_HOST && unit != SKEL_UNIT_DEVICE) return fail(SKEL_ERR_INVALID_ARG, "unknown unit");
        Storage *st = h->st;
        if ((st->valid & unit) || st->valid == 0) return (int)SKEL_OK;
        cudaStream_t s = (cudaStream_t)stream;
        if (unit == SKEL_UNIT_DEVICE) {
            void *p = nullptr;
            return acquire_device(h, SKEL_READ, s, &p);   // enqueues the copy, does not wait
        }
        if (!st->host) {
            SKEL_CUDA_TRY(cudaMallocHost(&st->host, st->bytes ? st->bytes : 1));
            st->host_owned = true;
        }
        int rc = order_after_last_use(st, s);
        if (rc) return rc;
        SKEL_CUDA_TRY(cudaMemcpyAsync(st->host, st->dev, st->bytes, cudaMemcpyDeviceToHost, s));
        st->d2h_count += 1;
        st->d2h_bytes += (int64_t)st->bytes;
        st->valid |= SKEL_UNIT_HOST;          // a read copy: both units valid
        st->last_stream = s;                  // a host access waits for this stream
        st->used_on_device = true;
        return (int)SKEL_OK;
    });
}

int skel_container_info(skel_handle h, int *dtype, int *ndim, int64_t *shape, int *valid_units)
{
    return guarded([&] {
        if (!valid_handle(h)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (dtype) *dtype = h->dtype;
        if (ndim) *ndim = h->ndim;
        if (shape) { shape[0] = h->shape[0]; shape[1] = h->shape[1]; }
        if (valid_units) *valid_units = h->st->valid;
        return (int)SKEL_OK;
    });
}

int skel_container_stats(skel_handle h, int64_t *h2d_count, int64_t *d2h_count, int64_t *h2d_bytes,
                         int64_t *d2h_bytes)
{
    return guarded([&] {
        if (!valid_handle(h)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (h2d_count) *h2d_count = h->st->h2d_count;
        if (d2h_count) *d2h_count = h->st->d2h_count;
        if (h2d_bytes) *h2d_bytes = h->st->h2d_bytes;
        if (d2h_bytes) *d2h_bytes = h->st->d2h_bytes;
        return (int)SKEL_OK;
    });
}

int skel_container_destroy(skel_handle h)
{
    return guarded([&] {
        if (!valid_handle(h)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (h->views > 0) return fail(SKEL_ERR_INVALID_ARG, "container still has live views");
        Storage *st = h->st;
        if (h->parent) h->parent->views -= 1;
        st->refs -= 1;
        if (st->refs == 0) {
            if (st->dev_owned && st->dev) dev_free(st->dev_alloc_rec, st->dev, st->last_stream);
            if (st->host_owned && st->host) {
                if (st->used_on_device) cudaStreamSynchronize(st->last_stream);
                cudaFreeHost(st->host);
            }
            delete st;
        }
        h->st = nullptr;
        delete h;
        return (int)SKEL_OK;
    });
}

}  // extern "C"

// ------------------------------------------------------- skeleton calls --
namespace {

// Acquires a list of operands for a call: inputs READ, outputs WRITE (or
// READWRITE when an output is also an input).  Returns the residency class
// of the call (1 if any input needed a host->device copy).
struct Operand {
    skel_handle h;
    int mode;
    void *ptr = nullptr;
};

int acquire_all(std::vector<Operand> &ops, cudaStream_t s, int *residency)
{
    int res = 0;
    for (auto &o : ops)
        if ((o.mode & SKEL_READ) && !device_valid(o.h) && (o.h->st->valid & SKEL_UNIT_HOST)) res = 1;
    for (size_t i = 0; i < ops.size(); ++i) {
        int mode = ops[i].mode;
        for (size_t j = 0; j < ops.size(); ++j)
            if (j != i && ops[j].h->st == ops[i].h->st) mode |= ops[j].mode;   // same storage: union of modes
        int rc = acquire_device(ops[i].h, mode, s, &ops[i].ptr);
        if (rc) return rc;
    }
    if (residency) *residency = res;
    return SKEL_OK;
}

bool same_storage(skel_handle a, skel_handle b) { return a && b && a->st == b->st; }

bool overlaps(skel_handle a, skel_handle b)
{
    if (!same_storage(a, b)) return false;
    const size_t es = dtype_size(a->dtype);
    size_t a0 = a->offset, a1 = a->offset + a->n * es;
    size_t b0 = b->offset, b1 = b->offset + b->n * dtype_size(b->dtype);
    return a0 < b1 && b0 < a1;
}

// Whether the device copies of a and b share bytes: views of one storage by
// their offsets, distinct storages (two containers wrapping the same device
// memory) by their device addresses.  *exact: both start at one address.
bool device_overlap(skel_handle a, skel_handle b, bool *exact)
{
    *exact = false;
    if (a->n == 0 || b->n == 0) return false;
    if (same_storage(a, b)) {
        const bool o = overlaps(a, b);
        *exact = o && a->offset == b->offset;
        return o;
    }
    if (!a->st->dev || !b->st->dev) return false;
    const char *a0 = static_cast<const char *>(a->st->dev) + a->offset, *a1 = a0 + a->n * dtype_size(a->dtype);
    const char *b0 = static_cast<const char *>(b->st->dev) + b->offset, *b1 = b0 + b->n * dtype_size(b->dtype);
    const bool o = a0 < b1 && b0 < a1;
    *exact = o && a0 == b0;
    return o;
}

template <class Launch>
int run_with_fallback(int sk, const Context &ctx, Launch launch, Choice (*def)())
{
    // Selectability (conditional composition): a variant whose constraint
    // fails for this call reports SKEL_ERR_UNSUPPORTED; the call then falls
    // back to the built-in default, and finally to variant 0, which every
    // skeleton implements without constraints.
    bool forced = false;
    Choice c = select_variant(ctx, &forced);
    int rc = launch(c);
    if (rc == SKEL_ERR_UNSUPPORTED && !forced) {
        const Choice fallbacks[2] = {def(), Choice{0, 0, 0, 0}};
        for (const Choice &d : fallbacks) {
            if (rc != SKEL_ERR_UNSUPPORTED) break;
            if (d.variant == c.variant && d.block == c.block && d.ept == c.ept && d.tile == c.tile) continue;
            clear_error();
            c = d;
            rc = launch(c);
        }
    }
    if (rc == SKEL_OK) record_last(sk, c);
    return rc;
}

int map_nin(int fn)
{
    switch (fn) {
    case SKEL_FN_ADD: case SKEL_FN_SUB: case SKEL_FN_MUL: case SKEL_FN_MAX: case SKEL_FN_AXPY: return 2;
    case SKEL_FN_TANH: case SKEL_FN_SQ: case SKEL_FN_SCALE: case SKEL_FN_COPY: return 1;
    default: return 0;
    }
}

bool map_needs_param(int fn) { return fn == SKEL_FN_AXPY || fn == SKEL_FN_SCALE; }

int copy_result_to_host(void *dst, const void *src_dev, size_t bytes, cudaStream_t s)
{
    SKEL_CUDA_TRY(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDeviceToHost, s));
    SKEL_CUDA_TRY(cudaStreamSynchronize(s));
    return SKEL_OK;
}

Choice reduce_def() { return reduce_default(); }
Choice map_def() { return map_default(); }
Choice scan_def() { return scan_default(); }
Choice st1_def() { return stencil_default(1); }
Choice st2_def() { return stencil_default(2); }
Choice ma_def() { return maparray_default(); }
Choice bat_def() { return batched_default(); }

// ------------------------------------------------------------ host edge --
// A call whose inputs are valid only in host memory (residency 1) first
// chooses how those bytes cross the host link (Sec. IV: the lazy copy is the
// container protocol; where it happens is an implementation choice, tuned
// per residency like any other variant):
//   0 copy     the whole lazy copy, then the call (the protocol as it stands);
//   1 chunked  the copy split into chunks on a copy stream; each chunk's part
//              of the call starts as soon as its chunk has landed, so link
//              and kernels overlap; the device copy ends valid, as with 0
//              (containers covering their whole storage only);
//   2 direct   the kernels read the pinned host copy in place over the link;
//              no device copy is made and the container stays valid only on
//              the host (pinned host memory only).
// Offered for Map, Reduce and MapReduce (the streaming skeletons); tile
// selects the chunk: 8 MiB << (2 * tile).
enum { kEdgeCopy = 0, kEdgeChunked = 1, kEdgeDirect = 2 };

bool host_only(skel_handle h) { return (h->st->valid & SKEL_UNIT_HOST) && !(h->st->valid & SKEL_UNIT_DEVICE); }

bool whole_storage(skel_handle h) { return h->offset == 0 && (size_t)h->n * dtype_size(h->dtype) == h->st->bytes; }

// The device's address of a host-only operand's pinned host copy; nullptr
// when the host copy is pageable.
const void *pinned_view(skel_handle h)
{
    cudaPointerAttributes a{};
    if (!h->st->host || cudaPointerGetAttributes(&a, h->st->host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<const char *>(a.devicePointer) + h->offset;
}

std::mutex g_copy_mu;
cudaStream_t g_copy_stream[64] = {};

int copy_stream(cudaStream_t *out)
{
    int dev = 0;
    SKEL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SKEL_ERR_UNSUPPORTED, "host edge: device index out of range");
    std::lock_guard<std::mutex> lk(g_copy_mu);
    if (!g_copy_stream[dev]) SKEL_CUDA_TRY(cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking));
    *out = g_copy_stream[dev];
    return SKEL_OK;
}

// One input of an edge call: its device-side address, and whether its bytes
// still have to cross the link (host-only, first occurrence of its storage).
struct EdgeIn {
    skel_handle h;
    bool host = false;
    bool first = true;
    const void *ptr = nullptr;
};

// The residency class of a call's READ operands, without acquiring them.
int residency_of(const std::vector<skel_handle> &ins)
{
    for (skel_handle h : ins)
        if (host_only(h)) return 1;
    return 0;
}

// Checks that edge variant v applies (before any state changes), then
// acquires the inputs: device-valid ones as usual, host-only ones with a
// device allocation and no copy (chunked) or at their pinned host address
// (direct).  The output must not share storage with a host-only input.
int edge_prepare(std::vector<EdgeIn> &ins, skel_handle out, int v, cudaStream_t s)
{
    for (size_t i = 0; i < ins.size(); ++i) {
        EdgeIn &e = ins[i];
        e.host = host_only(e.h);
        for (size_t j = 0; j < i; ++j)
            if (ins[j].h->st == e.h->st) e.first = false;
        if (!e.host) continue;
        if (out && same_storage(out, e.h)) return fail(SKEL_ERR_UNSUPPORTED, "host edge: output aliases a host-only input");
        if (v == kEdgeChunked && !whole_storage(e.h))
            return fail(SKEL_ERR_UNSUPPORTED, "chunked host edge: views are copied whole");
        if (v == kEdgeDirect && e.h->n > 0 && !pinned_view(e.h))
            return fail(SKEL_ERR_UNSUPPORTED, "direct host edge: the host copy is not pinned");
    }
    for (EdgeIn &e : ins) {
        Storage *st = e.h->st;
        if (!e.host) {
            void *p = nullptr;
            int rc = acquire_device(e.h, SKEL_READ, s, &p);
            if (rc) return rc;
            e.ptr = p;
            continue;
        }
        int rc = order_after_last_use(st, s);
        if (rc) return rc;
        if (v == kEdgeDirect) {
            e.ptr = e.h->n > 0 ? pinned_view(e.h) : nullptr;   // nothing to read when empty
            if (e.first) st->direct_reads += 1;
        } else {
            int dev = 0;
            cudaGetDevice(&dev);
            if (st->dev && st->device >= 0 && st->device != dev)
                return fail(SKEL_ERR_INVALID_ARG, "container device memory belongs to another device");
            if (!st->dev) {
                st->dev_alloc_rec = current_allocator();
                st->dev = dev_alloc(st->dev_alloc_rec, st->bytes, s);
                if (!st->dev) return fail(SKEL_ERR_OOM, "device allocation of container failed");
                st->dev_owned = true;
                st->device = dev;
            }
            e.ptr = static_cast<char *>(st->dev) + e.h->offset;
        }
        st->last_stream = s;
        st->used_on_device = true;
    }
    return SKEL_OK;
}

// The chunked pipeline: chunk k of every host-only input goes over the link
// on the copy stream, then `launch(off, len, k)` runs that chunk's part of
// the call on s.  The copy stream first waits for the work already queued
// on s (earlier users of the device copies).  Afterwards the host-only
// inputs are valid on both units, as after the whole lazy copy.
template <class Launch>
int edge_chunked(std::vector<EdgeIn> &ins, int64_t n, size_t es, int tile, cudaStream_t s, Launch launch)
{
    if (tile < 0 || tile > 3) return fail(SKEL_ERR_INVALID_ARG, "host edge: tile (chunk size) must be 0..3");
    const int64_t chunk = (int64_t)((size_t(8) << 20 << (2 * tile)) / es);
    cudaStream_t cs;
    int rc = copy_stream(&cs);
    if (rc) return rc;
    cudaEvent_t ev;
    SKEL_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    auto hop = [&](cudaStream_t from, cudaStream_t to) -> cudaError_t {   // `to` waits for `from`
        cudaError_t e = cudaEventRecord(ev, from);
        return e == cudaSuccess ? cudaStreamWaitEvent(to, ev, 0) : e;
    };
    cudaError_t e = hop(s, cs);
    for (int64_t off = 0, k = 0; e == cudaSuccess && off < n; off += chunk, ++k) {
        const int64_t len = n - off < chunk ? n - off : chunk;
        for (const EdgeIn &in : ins) {
            if (!in.host || !in.first || e != cudaSuccess) continue;
            e = cudaMemcpyAsync(const_cast<char *>(static_cast<const char *>(in.ptr)) + off * es,
                                static_cast<const char *>(in.h->st->host) + in.h->offset + off * es, (size_t)len * es,
                                cudaMemcpyHostToDevice, cs);
        }
        if (e == cudaSuccess) e = hop(cs, s);
        if (e == cudaSuccess && (rc = launch(off, len, k))) break;
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return fail_cuda(e, "chunked host edge");
    if (rc) return rc;
    for (const EdgeIn &in : ins) {
        if (!in.host || !in.first) continue;
        Storage *st = in.h->st;
        st->valid |= SKEL_UNIT_DEVICE;
        st->h2d_count += 1;
        st->h2d_bytes += (int64_t)st->bytes;
    }
    return SKEL_OK;
}

// The table's choice for a call on host-only inputs.  Second touch: an
// input already read in place since its host copy was last written is being
// reused, so a direct choice becomes the whole copy (later calls then find
// it on the device) unless the variant is forced.
Choice edge_choice(int sk, int dt, int64_t n, const skel_handle *ins, int nin, bool *forced)
{
    Choice c = select_variant(Context{SKEL_SK_EDGE, sk, dt, n, 0, 1}, forced);
    if (c.variant == kEdgeDirect && !*forced)
        for (int k = 0; k < nin; ++k)
            if (host_only(ins[k]) && ins[k]->st->direct_reads > 0) return Choice{kEdgeCopy, 0, 0, 0};
    return c;
}

// Map through edge variant 1 or 2; SKEL_ERR_UNSUPPORTED (nothing done) when
// the variant does not apply to this call.
int map_edge(int fn, float a, const skel_handle *ins, int nin, skel_handle out, const Choice &ec, cudaStream_t s)
{
    std::vector<EdgeIn> ei;
    for (int k = 0; k < nin; ++k) ei.push_back(EdgeIn{ins[k]});
    int rc = edge_prepare(ei, out, ec.variant, s);
    if (rc) return rc;
    void *po = nullptr;
    if ((rc = acquire_device(out, SKEL_WRITE, s, &po))) return rc;
    const float *i0 = (const float *)ei[0].ptr, *i1 = nin == 2 ? (const float *)ei[1].ptr : nullptr;
    float *o = (float *)po;
    auto run = [&](int64_t off, int64_t len, int res) {
        MapLaunch m{fn, a, i0 + off, i1 ? i1 + off : nullptr, o + off, len};
        m.alias = i0 == o || (i1 && i1 == o);
        Context ctx{SKEL_SK_MAP, fn, SKEL_F32, len, 0, res};
        return run_with_fallback(SKEL_SK_MAP, ctx, [&](const Choice &c) { return launch_map(m, c, s); }, map_def);
    };
    if (ec.variant == kEdgeDirect) return run(0, out->n, 1);
    return edge_chunked(ei, out->n, 4, ec.tile, s, [&](int64_t off, int64_t len, int64_t) { return run(off, len, 0); });
}

// Reduce / MapReduce through edge variant 1 or 2.  Chunked: each chunk's
// reduction writes its own partial; one more reduction (op, or + for
// MapReduce) adds the partials up into `out`.
int reduce_edge(int sk, int map_fn, int op, const skel_handle *ins, int nin, skel_handle result_dev, void **outp,
                const Choice &ec, cudaStream_t s)
{
    std::vector<EdgeIn> ei;
    for (int k = 0; k < nin; ++k) ei.push_back(EdgeIn{ins[k]});
    int rc = edge_prepare(ei, result_dev, ec.variant, s);
    if (rc) return rc;
    void *out = nullptr;
    if (result_dev) rc = acquire_device(result_dev, SKEL_WRITE, s, &out);
    else rc = result_slot(s, &out);
    if (rc) return rc;
    *outp = out;
    const int dt = ins[0]->dtype;
    const int64_t n = ins[0]->n;
    const size_t es = dtype_size(dt);
    const int fkey = sk == SKEL_SK_MAPREDUCE ? map_fn : op;
    auto run = [&](int64_t off, int64_t len, void *dst, int res) {
        ReduceLaunch r{op, map_fn, dt, static_cast<const char *>(ei[0].ptr) + off * es,
                       nin == 2 ? static_cast<const char *>(ei[1].ptr) + off * es : nullptr, dst, len};
        Context ctx{sk, fkey, dt, len, 0, res};
        return run_with_fallback(sk, ctx, [&](const Choice &c) { return launch_reduce(r, c, s); }, reduce_def);
    };
    if (ec.variant == kEdgeDirect) return run(0, n, out, 1);
    if (ec.tile < 0 || ec.tile > 3) return fail(SKEL_ERR_INVALID_ARG, "host edge: tile (chunk size) must be 0..3");
    const int64_t chunk = (int64_t)((size_t(8) << 20 << (2 * ec.tile)) / es);
    const int64_t nchunks = n == 0 ? 1 : (n + chunk - 1) / chunk;
    const Allocator rec = current_allocator();
    char *partials = static_cast<char *>(dev_alloc(rec, (size_t)nchunks * es, s));
    if (!partials) return fail(SKEL_ERR_OOM, "host edge: partial results");
    rc = edge_chunked(ei, n, es, ec.tile, s,
                      [&](int64_t off, int64_t len, int64_t k) { return run(off, len, partials + k * es, 0); });
    if (!rc && n == 0) rc = run(0, 0, partials, 0);   // the identity
    if (!rc) {
        ReduceLaunch r{sk == SKEL_SK_MAPREDUCE ? (int)SKEL_FN_ADD : op, -1, dt, partials, nullptr, out, nchunks};
        Context ctx{SKEL_SK_REDUCE, r.op, dt, nchunks, 0, 0};
        rc = run_with_fallback(SKEL_SK_REDUCE, ctx, [&](const Choice &c) { return launch_reduce(r, c, s); }, reduce_def);
    }
    dev_free(rec, partials, s);
    return rc;
}


int reduce_common(int sk, int map_fn, int op, const skel_handle *ins, int nin, void *result_host,
                  skel_handle result_dev, cudaStream_t s)
{
    for (int k = 0; k < nin; ++k)
        if (!valid_handle(ins[k])) return fail(SKEL_ERR_INVALID_ARG, "bad input handle");
    const int dt = ins[0]->dtype;
    if (nin == 2 && (ins[1]->dtype != dt || ins[1]->n != ins[0]->n))
        return fail(SKEL_ERR_SHAPE, "inputs differ in dtype or length");
    if (!result_host && !result_dev) return fail(SKEL_ERR_INVALID_ARG, "no result destination");
    if (result_dev && (!valid_handle(result_dev) || result_dev->n != 1 || result_dev->dtype != dt))
        return fail(SKEL_ERR_SHAPE, "result container must hold 1 element of the input dtype");
    if (residency_of(std::vector<skel_handle>(ins, ins + nin))) {
        bool forced = false;
        const Choice ec = edge_choice(sk, dt, ins[0]->n, ins, nin, &forced);
        if (ec.variant == kEdgeChunked || ec.variant == kEdgeDirect) {
            void *out = nullptr;
            int rc = reduce_edge(sk, map_fn, op, ins, nin, result_dev, &out, ec, s);
            if (rc == SKEL_OK) {
                record_last(SKEL_SK_EDGE, ec);
                return result_host ? copy_result_to_host(result_host, out, 4, s) : (int)SKEL_OK;
            }
            if (rc != SKEL_ERR_UNSUPPORTED || forced) return rc;
            clear_error();   // not applicable: the whole lazy copy
        } else if (ec.variant != kEdgeCopy) {
            return fail(SKEL_ERR_INVALID_ARG, "host edge: unknown variant");
        }
        record_last(SKEL_SK_EDGE, Choice{kEdgeCopy, 0, 0, 0});
    }
    std::vector<Operand> ops;
    for (int k = 0; k < nin; ++k) ops.push_back({ins[k], SKEL_READ});
    if (result_dev) ops.push_back({result_dev, SKEL_WRITE});
    int res = 0;
    int rc = acquire_all(ops, s, &res);
    if (rc) return rc;
    void *out = nullptr;
    if (result_dev) out = ops.back().ptr;
    else if ((rc = result_slot(s, &out))) return rc;
    ReduceLaunch r{op, map_fn, dt, ops[0].ptr, nin == 2 ? ops[1].ptr : nullptr, out, ins[0]->n};
    Context ctx{sk, sk == SKEL_SK_MAPREDUCE ? map_fn : op, dt, ins[0]->n, 0, res};
    rc = run_with_fallback(sk, ctx, [&](const Choice &c) { return launch_reduce(r, c, s); }, reduce_def);
    if (rc) return rc;
    if (result_host) return copy_result_to_host(result_host, out, 4, s);
    return SKEL_OK;
}

const float *default_weights(int fn, int radius, std::vector<float> &buf)
{
    if (fn == SKEL_FN_STENCIL5) {
        buf = {0.f, 0.125f, 0.f, 0.125f, 0.5f, 0.125f, 0.f, 0.125f, 0.f};
    } else if (fn == SKEL_FN_STENCIL9) {
        buf = {0.0625f, 0.125f, 0.0625f, 0.125f, 0.25f, 0.125f, 0.0625f, 0.125f, 0.0625f};
    } else {
        // binomial C(2r, k) / 4^r, computed in double and rounded once
        buf.assign(2 * radius + 1, 0.f);
        double c = 1.0;
        const double denom = std::ldexp(1.0, 2 * radius);
        for (int k = 0; k <= 2 * radius; ++k) {
            buf[k] = (float)(c / denom);
            c = c * (double)(2 * radius - k) / (double)(k + 1);
        }
    }
    return buf.data();
}

int stencil_common(skel_fn fn, int radius, const float *weights, int nweights, skel_boundary boundary,
                   skel_handle in, skel_handle out, cudaStream_t s, bool transpose)
{
    if (!valid_handle(in) || !valid_handle(out)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
    if (in->dtype != SKEL_F32 || out->dtype != SKEL_F32) return fail(SKEL_ERR_DTYPE, "mapoverlap: float32 only");
    if (in->n != out->n || in->ndim != out->ndim || in->shape[0] != out->shape[0])
        return fail(SKEL_ERR_SHAPE, "mapoverlap: input and output shapes differ");
    if (overlaps(in, out)) return fail(SKEL_ERR_INVALID_ARG, "mapoverlap: output must not alias the input");
    if (boundary < SKEL_CLAMP || boundary > SKEL_PERIODIC) return fail(SKEL_ERR_INVALID_ARG, "unknown boundary");
    std::vector<float> wbuf;
    StencilLaunch st{};
    st.boundary = boundary;
    st.transpose = transpose;
    if (in->ndim == 1) {
        if (fn != SKEL_FN_STENCIL1D) return fail(SKEL_ERR_UNSUPPORTED, "1D mapoverlap needs STENCIL1D");
        if (radius < 0 || radius > 16) return fail(SKEL_ERR_UNSUPPORTED, "1D radius must be 0..16");
        if (weights && nweights != 2 * radius + 1) return fail(SKEL_ERR_SHAPE, "1D weights: need 2r+1 values");
        st.ndim = 1;
        st.rows = 1;
        st.cols = in->n;
        st.w = weights ? weights : default_weights(fn, radius, wbuf);
    } else {
        if (fn != SKEL_FN_STENCIL5 && fn != SKEL_FN_STENCIL9) return fail(SKEL_ERR_UNSUPPORTED, "2D mapoverlap needs STENCIL5 or STENCIL9");
        if (radius != 1) return fail(SKEL_ERR_UNSUPPORTED, "2D stencils have radius 1");
        if (weights && nweights != 9) return fail(SKEL_ERR_SHAPE, "2D weights: need 9 values (3x3 row-major)");
        st.ndim = 2;
        st.rows = in->shape[0];
        st.cols = in->shape[1];
        st.taps5 = fn == SKEL_FN_STENCIL5;
        st.w = weights ? weights : default_weights(fn, 1, wbuf);
    }
    st.radius = radius;
    std::vector<Operand> ops{{in, SKEL_READ}, {out, SKEL_WRITE}};
    int res = 0;
    int rc = acquire_all(ops, s, &res);
    if (rc) return rc;
    st.in = static_cast<const float *>(ops[0].ptr);
    st.out = static_cast<float *>(ops[1].ptr);
    if (in->n == 0) return SKEL_OK;
    const int sk = in->ndim == 1 ? SKEL_SK_MAPOVERLAP1D : SKEL_SK_MAPOVERLAP2D;
    Context ctx{sk, fn, SKEL_F32, in->n, radius, res};
    return run_with_fallback(sk, ctx, [&](const Choice &c) { return launch_stencil(st, c, s); },
                             in->ndim == 1 ? st1_def : st2_def);
}

}  // namespace

extern "C" {

int skel_map(skel_fn fn, const double *params, int nparams, const skel_handle *ins, int nin, skel_handle out,
             void *stream)
{
    return guarded([&] {
        const int need = map_nin(fn);
        if (!need) return fail(SKEL_ERR_UNSUPPORTED, "map: function not offered");
        if (nin != need || !ins) return fail(SKEL_ERR_INVALID_ARG, "map: wrong number of inputs for this function");
        if (map_needs_param(fn) && (!params || nparams < 1)) return fail(SKEL_ERR_INVALID_ARG, "map: function needs params[0]");
        if (!valid_handle(out)) return fail(SKEL_ERR_INVALID_ARG, "bad output handle");
        for (int k = 0; k < nin; ++k) {
            if (!valid_handle(ins[k])) return fail(SKEL_ERR_INVALID_ARG, "bad input handle");
            if (ins[k]->dtype != SKEL_F32) return fail(SKEL_ERR_DTYPE, "map: float32 only");
            if (ins[k]->n != out->n) return fail(SKEL_ERR_SHAPE, "map: operands differ in length");
            bool exact = false;
            if (device_overlap(ins[k], out, &exact) && !exact)
                return fail(SKEL_ERR_INVALID_ARG, "map: output partially overlaps an input");
        }
        if (out->dtype != SKEL_F32) return fail(SKEL_ERR_DTYPE, "map: float32 only");
        cudaStream_t s = (cudaStream_t)stream;
        const float a = map_needs_param(fn) ? (float)params[0] : 0.f;
        if (residency_of(std::vector<skel_handle>(ins, ins + nin))) {
            bool forced = false;
            const Choice ec = edge_choice(SKEL_SK_MAP, SKEL_F32, out->n, ins, nin, &forced);
            if (ec.variant == kEdgeChunked || ec.variant == kEdgeDirect) {
                int rc = map_edge(fn, a, ins, nin, out, ec, s);
                if (rc == SKEL_OK) {
                    record_last(SKEL_SK_EDGE, ec);
                    return rc;
                }
                if (rc != SKEL_ERR_UNSUPPORTED || forced) return rc;
                clear_error();   // not applicable: the whole lazy copy
            } else if (ec.variant != kEdgeCopy) {
                return fail(SKEL_ERR_INVALID_ARG, "host edge: unknown variant");
            }
            record_last(SKEL_SK_EDGE, Choice{kEdgeCopy, 0, 0, 0});
        }
        std::vector<Operand> ops;
        for (int k = 0; k < nin; ++k) ops.push_back({ins[k], SKEL_READ});
        ops.push_back({out, SKEL_WRITE});
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        MapLaunch m{fn, a, (const float *)ops[0].ptr,
                    nin == 2 ? (const float *)ops[1].ptr : nullptr, (float *)ops.back().ptr, out->n};
        m.alias = m.in0 == m.out || (m.in1 && m.in1 == m.out);
        Context ctx{SKEL_SK_MAP, fn, SKEL_F32, out->n, 0, res};
        return run_with_fallback(SKEL_SK_MAP, ctx, [&](const Choice &c) { return launch_map(m, c, s); }, map_def);
    });
}

int skel_reduce(skel_fn op, skel_handle in, void *result_host, skel_handle result_dev, void *stream)
{
    return guarded([&] {
        if (op != SKEL_FN_ADD && op != SKEL_FN_MAX) return fail(SKEL_ERR_UNSUPPORTED, "reduce: op must be ADD or MAX");
        if (!valid_handle(in)) return fail(SKEL_ERR_INVALID_ARG, "bad input handle");
        if (in->dtype != SKEL_F32 && in->dtype != SKEL_I32) return fail(SKEL_ERR_DTYPE, "reduce: float32 or int32 only");
        skel_handle ins[1] = {in};
        return reduce_common(SKEL_SK_REDUCE, -1, op, ins, 1, result_host, result_dev, (cudaStream_t)stream);
    });
}

int skel_mapreduce(skel_fn map_fn, skel_fn red_op, const skel_handle *ins, int nin, void *result_host,
                   skel_handle result_dev, void *stream)
{
    return guarded([&] {
        if (red_op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce: reduce op must be ADD");
        if (map_fn != SKEL_FN_MUL && map_fn != SKEL_FN_SQ) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce: map must be MUL or SQ");
        if (!ins || nin != (map_fn == SKEL_FN_MUL ? 2 : 1)) return fail(SKEL_ERR_INVALID_ARG, "mapreduce: wrong number of inputs");
        for (int k = 0; k < nin; ++k)
            if (!valid_handle(ins[k]) || ins[k]->dtype != SKEL_F32) return fail(SKEL_ERR_DTYPE, "mapreduce: float32 inputs");
        return reduce_common(SKEL_SK_MAPREDUCE, map_fn, red_op, ins, nin, result_host, result_dev, (cudaStream_t)stream);
    });
}

int skel_scan(skel_fn op, int inclusive, skel_handle in, skel_handle out, void *stream)
{
    return guarded([&] {
        if (op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "scan: op must be ADD");
        if (!valid_handle(in) || !valid_handle(out)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (in->dtype != out->dtype || (in->dtype != SKEL_F32 && in->dtype != SKEL_I32))
            return fail(SKEL_ERR_DTYPE, "scan: float32 or int32, same for input and output");
        if (in->n != out->n || in->ndim != out->ndim || in->shape[0] != out->shape[0])
            return fail(SKEL_ERR_SHAPE, "scan: input and output shapes differ");
        if (overlaps(in, out)) return fail(SKEL_ERR_INVALID_ARG, "scan: output must not alias the input");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<Operand> ops{{in, SKEL_READ}, {out, SKEL_WRITE}};
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        ScanLaunch sc{in->dtype, inclusive != 0, false, ops[0].ptr, ops[1].ptr, in->n,
                      in->ndim == 2 ? in->shape[1] : 0};
        // keyed by the total element count: the variants scan all rows in one
        // launch, so the work, not the row length, decides which is fastest
        // (a row length of 8192 once picked the one-block variant for 8192 rows)
        Context ctx{SKEL_SK_SCAN, inclusive ? 1 : 0, in->dtype, in->n, 0, res};
        return run_with_fallback(SKEL_SK_SCAN, ctx, [&](const Choice &c) { return launch_scan(sc, c, s); }, scan_def);
    });
}

int skel_mapoverlap(skel_fn fn, int radius, const float *weights, int nweights, skel_boundary boundary,
                    skel_handle in, skel_handle out, void *stream)
{
    return guarded([&] {
        return stencil_common(fn, radius, weights, nweights, boundary, in, out, (cudaStream_t)stream, false);
    });
}

int skel_mapoverlap_chain(skel_fn fn, const float *weights, int nweights, skel_boundary boundary, int steps,
                          skel_handle in, skel_handle tmp, skel_handle out, void *stream)
{
    return guarded([&] {
        if (!valid_handle(in) || !valid_handle(out) || (tmp && !valid_handle(tmp)))
            return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (steps < 1) return fail(SKEL_ERR_INVALID_ARG, "mapoverlap chain: steps must be >= 1");
        if (in->ndim != 2 || (fn != SKEL_FN_STENCIL5 && fn != SKEL_FN_STENCIL9))
            return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap chain: 2D STENCIL5 or STENCIL9");
        if (in->dtype != SKEL_F32 || out->dtype != SKEL_F32 || (tmp && tmp->dtype != SKEL_F32))
            return fail(SKEL_ERR_DTYPE, "mapoverlap chain: float32 only");
        auto same = [&](skel_handle h) { return h->ndim == 2 && h->shape[0] == in->shape[0] && h->shape[1] == in->shape[1]; };
        if (!same(out) || (tmp && !same(tmp))) return fail(SKEL_ERR_SHAPE, "mapoverlap chain: shapes differ");
        if (overlaps(in, out) || (tmp && (overlaps(tmp, in) || overlaps(tmp, out))))
            return fail(SKEL_ERR_INVALID_ARG, "mapoverlap chain: in, tmp and out must not overlap");
        if (boundary < SKEL_CLAMP || boundary > SKEL_PERIODIC) return fail(SKEL_ERR_INVALID_ARG, "unknown boundary");
        if (weights && nweights != 9) return fail(SKEL_ERR_SHAPE, "2D weights: need 9 values (3x3 row-major)");
        std::vector<float> wbuf;
        StencilLaunch st{};
        st.ndim = 2;
        st.radius = 1;
        st.boundary = boundary;
        st.transpose = false;
        st.rows = in->shape[0];
        st.cols = in->shape[1];
        st.taps5 = fn == SKEL_FN_STENCIL5;
        st.w = weights ? weights : default_weights(fn, 1, wbuf);
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<Operand> ops{{in, SKEL_READ}, {out, SKEL_WRITE}};
        if (tmp) ops.push_back({tmp, SKEL_WRITE});
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        if (in->n == 0) return (int)SKEL_OK;
        const float *src = static_cast<const float *>(ops[0].ptr);
        float *dout = static_cast<float *>(ops[1].ptr);
        float *dtmp = tmp ? static_cast<float *>(ops[2].ptr) : nullptr;
        Context ctx{SKEL_SK_CHAIN2D, fn, SKEL_F32, in->n, steps, res};
        return run_with_fallback(SKEL_SK_CHAIN2D, ctx, [&](const Choice &c) -> int {
            if (c.variant == 1) {
                StencilLaunch f = st;
                f.in = src;
                f.out = dout;
                return launch_stencil_chain_fused(f, steps, dtmp, c, s);
            }
            if (c.variant != 0) return fail(SKEL_ERR_INVALID_ARG, "mapoverlap chain: unknown variant");
            if (steps > 1 && !dtmp) return fail(SKEL_ERR_UNSUPPORTED, "mapoverlap chain: per-call steps need tmp");
            // per call: each step dispatched as a single 2D MapOverlap; the
            // last step writes out
            const float *cur = src;
            for (int k = 0; k < steps; ++k) {
                StencilLaunch one = st;
                one.in = cur;
                one.out = ((steps - 1 - k) % 2 == 0) ? dout : dtmp;
                Context c1{SKEL_SK_MAPOVERLAP2D, fn, SKEL_F32, in->n, 1, res};
                int r1 = run_with_fallback(SKEL_SK_MAPOVERLAP2D, c1,
                                           [&](const Choice &cc) { return launch_stencil(one, cc, s); }, st2_def);
                if (r1) return r1;
                cur = one.out;
            }
            return (int)SKEL_OK;
        }, chain_default);
    });
}

int skel_compose_map_stencil_sumsq(skel_fn map_fn, const double *params, int nparams, skel_fn stencil,
                                   const float *weights, int nweights, skel_boundary boundary, skel_handle in,
                                   void *result_host, skel_handle result_dev, void *stream)
{
    return guarded([&] {
        if (map_fn != SKEL_FN_TANH && map_fn != SKEL_FN_SQ && map_fn != SKEL_FN_SCALE && map_fn != SKEL_FN_COPY)
            return fail(SKEL_ERR_UNSUPPORTED, "composed chain: map must be TANH, SQ, SCALE or COPY");
        if (map_fn == SKEL_FN_SCALE && (!params || nparams < 1))
            return fail(SKEL_ERR_INVALID_ARG, "composed chain: SCALE needs params[0]");
        if (stencil != SKEL_FN_STENCIL5 && stencil != SKEL_FN_STENCIL9)
            return fail(SKEL_ERR_UNSUPPORTED, "composed chain: stencil must be STENCIL5 or STENCIL9");
        if (!valid_handle(in)) return fail(SKEL_ERR_INVALID_ARG, "bad input handle");
        if (in->ndim != 2 || in->dtype != SKEL_F32) return fail(SKEL_ERR_DTYPE, "composed chain: in must be 2D float32");
        if (boundary < SKEL_CLAMP || boundary > SKEL_PERIODIC) return fail(SKEL_ERR_INVALID_ARG, "unknown boundary");
        if (weights && nweights != 9) return fail(SKEL_ERR_SHAPE, "2D weights: need 9 values (3x3 row-major)");
        if (!result_host && !result_dev) return fail(SKEL_ERR_INVALID_ARG, "no result destination");
        if (result_dev && (!valid_handle(result_dev) || result_dev->n != 1 || result_dev->dtype != SKEL_F32))
            return fail(SKEL_ERR_SHAPE, "result container must hold 1 float32 element");
        if (result_dev && same_storage(result_dev, in)) return fail(SKEL_ERR_INVALID_ARG, "result aliases the input");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<Operand> ops{{in, SKEL_READ}};
        if (result_dev) ops.push_back({result_dev, SKEL_WRITE});
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        void *out = nullptr;
        if (result_dev) out = ops.back().ptr;
        else if ((rc = result_slot(s, &out))) return rc;
        const int64_t n = in->n;
        std::vector<float> wbuf;
        ComposeLaunch cl{map_fn, map_fn == SKEL_FN_SCALE ? (float)params[0] : 0.f, boundary,
                         weights ? weights : default_weights(stencil, 1, wbuf), stencil == SKEL_FN_STENCIL5,
                         static_cast<const float *>(ops[0].ptr), in->shape[0], in->shape[1]};
        const Allocator rec = current_allocator();
        // the sum of squares of the chain's last stage, over `len` values at v
        auto sumsq = [&](const float *v, int64_t len, int map) {
            ReduceLaunch r{SKEL_FN_ADD, map, SKEL_F32, v, nullptr, out, len};
            const int sk = map < 0 ? (int)SKEL_SK_REDUCE : (int)SKEL_SK_MAPREDUCE;
            Context c{sk, map < 0 ? (int)SKEL_FN_ADD : map, SKEL_F32, len, 0, 0};
            return run_with_fallback(sk, c, [&](const Choice &cc) { return launch_reduce(r, cc, s); }, reduce_def);
        };
        if (n == 0) {   // the empty sum: 0
            if ((rc = sumsq(nullptr, 0, SKEL_FN_SQ))) return rc;
            return result_host ? copy_result_to_host(result_host, out, 4, s) : (int)SKEL_OK;
        }
        Context ctx{SKEL_SK_COMPOSE, stencil, SKEL_F32, n, 1, res};
        rc = run_with_fallback(SKEL_SK_COMPOSE, ctx, [&](const Choice &c) -> int {
            if (c.variant == 1) {
                int64_t np = 0;
                int r1 = compose_fused_check(cl, c, &np);
                if (r1) return r1;
                float *parts = static_cast<float *>(dev_alloc(rec, (size_t)np * 4, s));
                if (!parts) return fail(SKEL_ERR_OOM, "composed chain: partial sums");
                r1 = launch_compose_fused(cl, c, parts, s);
                if (!r1) r1 = sumsq(parts, np, -1);
                dev_free(rec, parts, s);
                return r1;
            }
            if (c.variant != 0) return fail(SKEL_ERR_INVALID_ARG, "composed chain: unknown variant");
            // per call: Map -> MapOverlap -> MapReduce(sq, +), each dispatched
            float *t = static_cast<float *>(dev_alloc(rec, (size_t)n * 4, s));
            float *u = t ? static_cast<float *>(dev_alloc(rec, (size_t)n * 4, s)) : nullptr;
            int r1 = (t && u) ? (int)SKEL_OK : fail(SKEL_ERR_OOM, "composed chain: temporaries");
            if (!r1) {
                MapLaunch m{map_fn, cl.a, cl.in, nullptr, t, n};
                Context cm{SKEL_SK_MAP, map_fn, SKEL_F32, n, 0, 0};
                r1 = run_with_fallback(SKEL_SK_MAP, cm, [&](const Choice &cc) { return launch_map(m, cc, s); }, map_def);
            }
            if (!r1) {
                StencilLaunch st{};
                st.ndim = 2;
                st.radius = 1;
                st.boundary = boundary;
                st.w = cl.w;
                st.taps5 = cl.taps5;
                st.in = t;
                st.out = u;
                st.rows = cl.rows;
                st.cols = cl.cols;
                st.transpose = false;
                Context cs2{SKEL_SK_MAPOVERLAP2D, stencil, SKEL_F32, n, 1, 0};
                r1 = run_with_fallback(SKEL_SK_MAPOVERLAP2D, cs2,
                                       [&](const Choice &cc) { return launch_stencil(st, cc, s); }, st2_def);
            }
            if (!r1) r1 = sumsq(u, n, SKEL_FN_SQ);
            if (u) dev_free(rec, u, s);
            if (t) dev_free(rec, t, s);
            return r1;
        }, compose_default);
        if (rc) return rc;
        return result_host ? copy_result_to_host(result_host, out, 4, s) : (int)SKEL_OK;
    });
}

int skel_maparray(skel_fn fn, skel_handle whole, skel_handle elem, skel_handle out, void *stream)
{
    return guarded([&] {
        if (!valid_handle(whole) || !valid_handle(elem) || !valid_handle(out)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (whole->dtype != SKEL_F32 || out->dtype != SKEL_F32 || whole->ndim != 1 || out->ndim != 1)
            return fail(SKEL_ERR_DTYPE, "maparray: A and out must be 1D float32");
        int64_t n = 0;
        if (fn == SKEL_FN_GATHER) {
            if (elem->dtype != SKEL_I32 || elem->ndim != 1) return fail(SKEL_ERR_DTYPE, "gather: indices must be 1D int32");
            if (whole->n < 1 && elem->n > 0) return fail(SKEL_ERR_SHAPE, "gather: A must not be empty");
            n = elem->n;
        } else if (fn == SKEL_FN_ROWDOT) {
            if (elem->dtype != SKEL_F32 || elem->ndim != 2 || elem->shape[1] != whole->n)
                return fail(SKEL_ERR_SHAPE, "rowdot: B must be 2D float32 with as many columns as A has elements");
            n = elem->shape[0];
        } else {
            return fail(SKEL_ERR_UNSUPPORTED, "maparray: fn must be GATHER or ROWDOT");
        }
        if (out->n != n) return fail(SKEL_ERR_SHAPE, "maparray: out has the wrong length");
        if (overlaps(out, whole) || overlaps(out, elem)) return fail(SKEL_ERR_INVALID_ARG, "maparray: output aliases an input");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<Operand> ops{{whole, SKEL_READ}, {elem, SKEL_READ}, {out, SKEL_WRITE}};
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        if (n == 0) return (int)SKEL_OK;
        MapArrayLaunch ma{fn, (const float *)ops[0].ptr, whole->n, ops[1].ptr, (float *)ops[2].ptr, n};
        Context ctx{SKEL_SK_MAPARRAY, fn, SKEL_F32, fn == SKEL_FN_ROWDOT ? whole->n : n, 0, res};
        return run_with_fallback(SKEL_SK_MAPARRAY, ctx, [&](const Choice &c) { return launch_maparray(ma, c, s); }, ma_def);
    });
}

int skel_maparray_grid(skel_fn fn, skel_handle whole, skel_handle out, const double *params, int nparams,
                       void *stream)
{
    return guarded([&] {
        if (!valid_handle(whole) || !valid_handle(out)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (fn != SKEL_FN_COULOMB) return fail(SKEL_ERR_UNSUPPORTED, "maparray grid: fn must be COULOMB");
        if (whole->dtype != SKEL_F32 || out->dtype != SKEL_F32)
            return fail(SKEL_ERR_DTYPE, "coulomb: atoms and out must be float32");
        if (whole->ndim != 2 || whole->shape[1] != 4) return fail(SKEL_ERR_SHAPE, "coulomb: atoms must be (m, 4)");
        if (out->ndim != 2) return fail(SKEL_ERR_SHAPE, "coulomb: out must be 2D");
        if (!params || nparams != 2 || !(params[0] > 0.0))
            return fail(SKEL_ERR_INVALID_ARG, "coulomb: params must be {h > 0, z0}");
        if (overlaps(out, whole)) return fail(SKEL_ERR_INVALID_ARG, "coulomb: output aliases the atoms");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<Operand> ops{{whole, SKEL_READ}, {out, SKEL_WRITE}};
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        if (out->n == 0) return (int)SKEL_OK;
        CoulombLaunch cl{(const float *)ops[0].ptr, whole->shape[0], (float *)ops[1].ptr, out->shape[0], out->shape[1],
                         (float)params[0], (float)params[1]};
        Context ctx{SKEL_SK_MAPARRAY, SKEL_FN_COULOMB, SKEL_F32, out->n, 0, res};
        return run_with_fallback(SKEL_SK_MAPARRAY, ctx, [&](const Choice &c) { return launch_coulomb(cl, c, s); },
                                 maparray_default);
    });
}

}  // extern "C"

// ----------------------------------------------------------- batched ----
namespace {

int batched_prepare(skel_fn map_fn, skel_fn red_op, skel_fn scan_op, skel_handle values, skel_handle offsets,
                    skel_handle results, skel_handle scan_out, BatchedLaunch *b, std::vector<Operand> &ops)
{
    if (!valid_handle(values) || !valid_handle(offsets)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
    if (results && !valid_handle(results)) return fail(SKEL_ERR_INVALID_ARG, "bad results handle");
    if (scan_out && !valid_handle(scan_out)) return fail(SKEL_ERR_INVALID_ARG, "bad scan_out handle");
    if (!results && !scan_out) return fail(SKEL_ERR_INVALID_ARG, "batched: nothing to compute");
    if (results && (map_fn != SKEL_FN_SQ || red_op != SKEL_FN_ADD))
        return fail(SKEL_ERR_UNSUPPORTED, "batched: mapreduce must be (SQ, ADD)");
    if (scan_out && scan_op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "batched: scan op must be ADD");
    if (values->dtype != SKEL_F32 || offsets->dtype != SKEL_I64 || values->ndim != 1 || offsets->ndim != 1)
        return fail(SKEL_ERR_DTYPE, "batched: values 1D float32, offsets 1D int64");
    if (offsets->n < 1) return fail(SKEL_ERR_SHAPE, "batched: offsets needs B+1 >= 1 entries");
    const int64_t B = offsets->n - 1;
    if (results && (results->dtype != SKEL_F32 || results->n != B)) return fail(SKEL_ERR_SHAPE, "batched: results must be B float32");
    if (scan_out && (scan_out->dtype != SKEL_F32 || scan_out->n != values->n))
        return fail(SKEL_ERR_SHAPE, "batched: scan_out must match values");
    if (scan_out && overlaps(scan_out, values)) return fail(SKEL_ERR_INVALID_ARG, "batched: scan_out aliases values");
    ops.clear();
    ops.push_back({values, SKEL_READ});
    ops.push_back({offsets, SKEL_READ});
    if (results) ops.push_back({results, SKEL_WRITE});
    if (scan_out) ops.push_back({scan_out, SKEL_WRITE});
    b->want_reduce = results != nullptr;
    b->want_scan = scan_out != nullptr;
    b->B = B;
    b->total = values->n;
    return SKEL_OK;
}

void batched_bind(BatchedLaunch *b, std::vector<Operand> &ops)
{
    b->values = (const float *)ops[0].ptr;
    b->offsets = (const int64_t *)ops[1].ptr;
    size_t k = 2;
    b->results = b->want_reduce ? (float *)ops[k++].ptr : nullptr;
    b->scan_out = b->want_scan ? (float *)ops[k++].ptr : nullptr;
}

}  // namespace

struct skel_plan_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *scratch = nullptr;
    Allocator alloc{};
    cudaStream_t alloc_stream = nullptr;
};

extern "C" {

int skel_batched(skel_fn map_fn, skel_fn red_op, skel_fn scan_op, int inclusive, skel_handle values,
                 skel_handle offsets, skel_handle results, skel_handle scan_out, void *stream)
{
    return guarded([&] {
        BatchedLaunch b{};
        std::vector<Operand> ops;
        int rc = batched_prepare(map_fn, red_op, scan_op, values, offsets, results, scan_out, &b, ops);
        if (rc) return rc;
        b.inclusive = inclusive != 0;
        cudaStream_t s = (cudaStream_t)stream;
        int res = 0;
        if ((rc = acquire_all(ops, s, &res))) return rc;
        batched_bind(&b, ops);
        Context ctx{SKEL_SK_BATCHED, 0, SKEL_F32, b.total, 0, res};
        return run_with_fallback(SKEL_SK_BATCHED, ctx, [&](const Choice &c) {
            Scratch scr{};
            int r2 = get_scratch(s, batched_data_bytes(b, c), batched_word_count(b, c), &scr);
            if (r2) return r2;
            return launch_batched(b, c, scr.ctl, scr.words, scr.data, scr.epoch, s);
        }, bat_def);
    });
}

int skel_batched_plan_create(skel_fn map_fn, skel_fn red_op, skel_fn scan_op, int inclusive, skel_handle values,
                             skel_handle offsets, skel_handle results, skel_handle scan_out, void *stream,
                             skel_plan *plan)
{
    return guarded([&] {
        if (!plan) return fail(SKEL_ERR_INVALID_ARG, "plan is NULL");
        BatchedLaunch b{};
        std::vector<Operand> ops;
        int rc = batched_prepare(map_fn, red_op, scan_op, values, offsets, results, scan_out, &b, ops);
        if (rc) return rc;
        b.inclusive = inclusive != 0;
        cudaStream_t s = (cudaStream_t)stream;
        int res = 0;
        if ((rc = acquire_all(ops, s, &res))) return rc;
        batched_bind(&b, ops);
        Context ctx{SKEL_SK_BATCHED, 0, SKEL_F32, b.total, 0, res};
        bool forced = false;
        Choice c = select_variant(ctx, &forced);
        auto *p = new skel_plan_s();
        p->alloc = current_allocator();
        p->alloc_stream = s;
        const size_t nwords = (batched_word_count(b, c) + 31) & ~(size_t)31;
        const size_t total = sizeof(Control) + nwords * 8 + batched_data_bytes(b, c);
        p->scratch = dev_alloc(p->alloc, total, s);
        if (!p->scratch) { delete p; return fail(SKEL_ERR_OOM, "plan scratch allocation failed"); }
        cudaError_t e = cudaMemsetAsync(p->scratch, 0, total, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { dev_free(p->alloc, p->scratch, s); delete p; return fail_cuda(e, "plan scratch clear"); }
        cudaStream_t cap;
        SKEL_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        Control *ctl = static_cast<Control *>(p->scratch);
        uint64_t *words = reinterpret_cast<uint64_t *>(static_cast<unsigned char *>(p->scratch) + sizeof(Control));
        unsigned char *data = reinterpret_cast<unsigned char *>(words + nwords);
        // relaxed: the launcher queries occupancy (a host-side call) while capturing
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            // every replay starts from cleared look-back words and abort word
            // (the counters are reset by the kernels themselves; the error
            // word stays sticky), so all replays can use epoch 1
            e = cudaMemsetAsync(words, 0, nwords * 8, cap);
            if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->abort, 0, sizeof(uint32_t), cap);
            if (e == cudaSuccess) rc = launch_batched(b, c, ctl, words, data, 1u, cap);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e2;
            p->graph = g;
        }
        cudaStreamDestroy(cap);
        if (e == cudaSuccess && rc == SKEL_OK) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess || rc != SKEL_OK) {
            if (p->exec) cudaGraphExecDestroy(p->exec);
            if (p->graph) cudaGraphDestroy(p->graph);
            dev_free(p->alloc, p->scratch, s);
            delete p;
            return rc != SKEL_OK ? rc : fail_cuda(e, "graph capture of the batched launch");
        }
        record_last(SKEL_SK_BATCHED, c);
        *plan = p;
        return (int)SKEL_OK;
    });
}

int skel_plan_launch(skel_plan plan, void *stream)
{
    return guarded([&] {
        if (!plan || !plan->exec) return fail(SKEL_ERR_INVALID_ARG, "bad plan");
        SKEL_CUDA_TRY(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
        return (int)SKEL_OK;
    });
}

int skel_plan_destroy(skel_plan plan)
{
    return guarded([&] {
        if (!plan) return fail(SKEL_ERR_INVALID_ARG, "bad plan");
        cudaDeviceSynchronize();
        if (plan->exec) cudaGraphExecDestroy(plan->exec);
        if (plan->graph) cudaGraphDestroy(plan->graph);
        dev_free(plan->alloc, plan->scratch, plan->alloc_stream);
        delete plan;
        return (int)SKEL_OK;
    });
}

// ------------------------------------------------------------ backward --

int skel_map_bwd(skel_fn fn, const double *params, int nparams, const skel_handle *ins, int nin, skel_handle gout,
                 skel_handle *gins, void *stream)
{
    return skel_map_bwd_sum(fn, params, nparams, ins, nin, &gout, 1, gins, stream);
}

int skel_map_bwd_sum(skel_fn fn, const double *params, int nparams, const skel_handle *ins, int nin,
                     const skel_handle *gouts, int ngout, skel_handle *gins, void *stream)
{
    return guarded([&] {
        if (!gouts || ngout < 1 || ngout > 2) return fail(SKEL_ERR_INVALID_ARG, "map_bwd: one or two upstream gradients");
        const skel_handle gout = gouts[0];
        const int need = map_nin(fn);
        if (!need) return fail(SKEL_ERR_UNSUPPORTED, "map_bwd: function not offered");
        if (fn == SKEL_FN_MAX) return fail(SKEL_ERR_UNSUPPORTED, "map_bwd: MAX has no adjoint here");
        if (nin != need || !ins || !gins) return fail(SKEL_ERR_INVALID_ARG, "map_bwd: wrong number of inputs");
        if (map_needs_param(fn) && (!params || nparams < 1)) return fail(SKEL_ERR_INVALID_ARG, "map_bwd: needs params[0]");
        if (!valid_handle(gout) || gout->dtype != SKEL_F32) return fail(SKEL_ERR_INVALID_ARG, "bad gout");
        if (ngout == 2 && (!valid_handle(gouts[1]) || gouts[1]->dtype != SKEL_F32 || gouts[1]->n != gout->n))
            return fail(SKEL_ERR_SHAPE, "map_bwd: the second upstream gradient must match the first");
        const bool from_out = fn == SKEL_FN_TANH && params && nparams >= 1 && params[0] == 1.0;
        std::vector<Operand> ops;
        for (int k = 0; k < nin; ++k) {
            if (!valid_handle(ins[k]) || ins[k]->dtype != SKEL_F32 || ins[k]->n != gout->n)
                return fail(SKEL_ERR_SHAPE, "map_bwd: inputs must match gout");
            ops.push_back({ins[k], SKEL_READ});
        }
        ops.push_back({gout, SKEL_READ});
        if (ngout == 2) ops.push_back({gouts[1], SKEL_READ});
        int outs = 0;
        for (int k = 0; k < nin; ++k) {
            if (!gins[k]) continue;
            if (!valid_handle(gins[k]) || gins[k]->dtype != SKEL_F32 || gins[k]->n != gout->n)
                return fail(SKEL_ERR_SHAPE, "map_bwd: gradients must match gout");
            ops.push_back({gins[k], SKEL_WRITE});
            ++outs;
        }
        if (!outs) return (int)SKEL_OK;
        cudaStream_t s = (cudaStream_t)stream;
        int rc = acquire_all(ops, s, nullptr);
        if (rc) return rc;
        MapBwdLaunch m{};
        m.fn = fn;
        m.a = map_needs_param(fn) ? (float)params[0] : 0.f;
        m.tanh_from_output = from_out;
        m.in0 = (const float *)ops[0].ptr;
        m.in1 = nin == 2 ? (const float *)ops[1].ptr : nullptr;
        m.g = (const float *)ops[nin].ptr;
        m.g2 = ngout == 2 ? (const float *)ops[nin + 1].ptr : nullptr;
        size_t k = nin + ngout;
        m.gin0 = gins[0] ? (float *)ops[k++].ptr : nullptr;
        m.gin1 = (nin == 2 && gins[1]) ? (float *)ops[k++].ptr : nullptr;
        m.n = gout->n;
        return launch_map_bwd(m, s);
    });
}

int skel_reduce_bwd(skel_fn op, skel_handle gr, const float *gr_host, skel_handle gin, void *stream)
{
    return guarded([&] {
        if (op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "reduce_bwd: op must be ADD");
        if (!valid_handle(gin) || gin->dtype != SKEL_F32) return fail(SKEL_ERR_INVALID_ARG, "bad gin");
        if (!gr && !gr_host) return fail(SKEL_ERR_INVALID_ARG, "no upstream gradient");
        if (gr && (!valid_handle(gr) || gr->n != 1 || gr->dtype != SKEL_F32)) return fail(SKEL_ERR_SHAPE, "gr must be 1 float32");
        std::vector<Operand> ops;
        if (gr) ops.push_back({gr, SKEL_READ});
        ops.push_back({gin, SKEL_WRITE});
        cudaStream_t s = (cudaStream_t)stream;
        int rc = acquire_all(ops, s, nullptr);
        if (rc) return rc;
        MapBwdLaunch m{};
        m.fn = SKEL_FN_COPY;   // d(sum)/dx_i = 1: gin = gr broadcast
        m.g_scalar_dev = gr ? (const float *)ops[0].ptr : nullptr;
        m.g_scalar_host = gr ? 0.f : *gr_host;
        m.gin0 = (float *)ops.back().ptr;
        m.n = gin->n;
        return launch_map_bwd(m, s);
    });
}

int skel_mapreduce_bwd(skel_fn map_fn, skel_fn red_op, const skel_handle *ins, int nin, skel_handle gr,
                       const float *gr_host, skel_handle *gins, void *stream)
{
    return guarded([&] {
        if (red_op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce_bwd: reduce op must be ADD");
        if (map_fn != SKEL_FN_MUL && map_fn != SKEL_FN_SQ) return fail(SKEL_ERR_UNSUPPORTED, "mapreduce_bwd: map must be MUL or SQ");
        if (!ins || !gins || nin != (map_fn == SKEL_FN_MUL ? 2 : 1)) return fail(SKEL_ERR_INVALID_ARG, "mapreduce_bwd: wrong inputs");
        if (!gr && !gr_host) return fail(SKEL_ERR_INVALID_ARG, "no upstream gradient");
        if (gr && (!valid_handle(gr) || gr->n != 1 || gr->dtype != SKEL_F32)) return fail(SKEL_ERR_SHAPE, "gr must be 1 float32");
        std::vector<Operand> ops;
        for (int k = 0; k < nin; ++k) {
            if (!valid_handle(ins[k]) || ins[k]->dtype != SKEL_F32 || ins[k]->n != ins[0]->n)
                return fail(SKEL_ERR_SHAPE, "mapreduce_bwd: inputs must be float32 of equal length");
            ops.push_back({ins[k], SKEL_READ});
        }
        if (gr) ops.push_back({gr, SKEL_READ});
        int outs = 0;
        for (int k = 0; k < nin; ++k) {
            if (!gins[k]) continue;
            if (!valid_handle(gins[k]) || gins[k]->dtype != SKEL_F32 || gins[k]->n != ins[0]->n)
                return fail(SKEL_ERR_SHAPE, "mapreduce_bwd: gradients must match the inputs");
            ops.push_back({gins[k], SKEL_WRITE});
            ++outs;
        }
        if (!outs) return (int)SKEL_OK;
        cudaStream_t s = (cudaStream_t)stream;
        int rc = acquire_all(ops, s, nullptr);
        if (rc) return rc;
        MapBwdLaunch m{};
        m.fn = map_fn;
        m.in0 = (const float *)ops[0].ptr;
        m.in1 = nin == 2 ? (const float *)ops[1].ptr : nullptr;
        size_t k = nin;
        m.g_scalar_dev = gr ? (const float *)ops[k++].ptr : nullptr;
        m.g_scalar_host = gr ? 0.f : *gr_host;
        m.gin0 = gins[0] ? (float *)ops[k++].ptr : nullptr;
        m.gin1 = (nin == 2 && gins[1]) ? (float *)ops[k++].ptr : nullptr;
        m.n = ins[0]->n;
        return launch_map_bwd(m, s);
    });
}

int skel_scan_bwd(skel_fn op, int inclusive, skel_handle gout, skel_handle gin, void *stream)
{
    return guarded([&] {
        if (op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "scan_bwd: op must be ADD");
        if (!valid_handle(gout) || !valid_handle(gin)) return fail(SKEL_ERR_INVALID_ARG, "bad handle");
        if (gout->dtype != SKEL_F32 || gin->dtype != SKEL_F32) return fail(SKEL_ERR_DTYPE, "scan_bwd: float32 only");
        if (gout->n != gin->n || gout->ndim != gin->ndim || gout->shape[0] != gin->shape[0])
            return fail(SKEL_ERR_SHAPE, "scan_bwd: shapes differ");
        if (overlaps(gout, gin)) return fail(SKEL_ERR_INVALID_ARG, "scan_bwd: output aliases the input");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<Operand> ops{{gout, SKEL_READ}, {gin, SKEL_WRITE}};
        int res = 0;
        int rc = acquire_all(ops, s, &res);
        if (rc) return rc;
        ScanLaunch sc{SKEL_F32, inclusive != 0, true, ops[0].ptr, ops[1].ptr, gout->n,
                      gout->ndim == 2 ? gout->shape[1] : 0};
        // reverse scans have their own keys (fn 2: exclusive, 3: inclusive)
        Context ctx{SKEL_SK_SCAN, inclusive ? 3 : 2, SKEL_F32, gout->n, 0, res};   // total work, as forward
        return run_with_fallback(SKEL_SK_SCAN, ctx, [&](const Choice &c) { return launch_scan(sc, c, s); }, scan_def);
    });
}

int skel_mapoverlap_bwd(skel_fn fn, int radius, const float *weights, int nweights, skel_boundary boundary,
                        skel_handle gout, skel_handle gin, void *stream)
{
    return guarded([&] {
        return stencil_common(fn, radius, weights, nweights, boundary, gout, gin, (cudaStream_t)stream, true);
    });
}

// ------------------------------------------------------------ dispatch --

int skel_load_dispatch_table(const char *path) { return guarded([&] { return dispatch_load(path); }); }

int skel_dispatch_set(int skeleton, int fn, int dtype, int bucket, int radius, int residency, int variant,
                      int block, int ept, int tile)
{
    return guarded([&] {
        return dispatch_set(skeleton, fn, dtype, bucket, radius, residency, Choice{variant, block, ept, tile});
    });
}

int skel_dispatch_size(void) { return dispatch_size(); }

int skel_force_variant(int skeleton, int variant, int block, int ept, int tile)
{
    return guarded([&] { return force_variant(skeleton, Choice{variant, block, ept, tile}); });
}

int skel_last_variant(int skeleton, int *variant, int *block, int *ept, int *tile)
{
    return guarded([&] {
        Choice c;
        int rc = last_choice(skeleton, &c);
        if (rc) return rc;
        if (variant) *variant = c.variant;
        if (block) *block = c.block;
        if (ept) *ept = c.ept;
        if (tile) *tile = c.tile;
        return (int)SKEL_OK;
    });
}

int skel_variant_count(int skeleton)
{
    switch (skeleton) {
    case SKEL_SK_MAP: return map_variant_count();
    case SKEL_SK_REDUCE: case SKEL_SK_MAPREDUCE: return reduce_variant_count();
    case SKEL_SK_SCAN: return scan_variant_count();
    case SKEL_SK_MAPOVERLAP1D: return stencil_variant_count(1);
    case SKEL_SK_MAPOVERLAP2D: return stencil_variant_count(2);
    case SKEL_SK_MAPARRAY: return maparray_variant_count();
    case SKEL_SK_BATCHED: return batched_variant_count();
    case SKEL_SK_CHAIN2D: return chain_variant_count();
    case SKEL_SK_EDGE: return 3;
    case SKEL_SK_COMPOSE: return compose_variant_count();
    default: return 0;
    }
}

const char *skel_variant_name(int skeleton, int variant)
{
    switch (skeleton) {
    case SKEL_SK_MAP: return map_variant_name(variant);
    case SKEL_SK_REDUCE: case SKEL_SK_MAPREDUCE: return reduce_variant_name(variant);
    case SKEL_SK_SCAN: return scan_variant_name(variant);
    case SKEL_SK_MAPOVERLAP1D: return stencil_variant_name(1, variant);
    case SKEL_SK_MAPOVERLAP2D: return stencil_variant_name(2, variant);
    case SKEL_SK_MAPARRAY: return maparray_variant_name(variant);
    case SKEL_SK_BATCHED: return batched_variant_name(variant);
    case SKEL_SK_CHAIN2D: return chain_variant_name(variant);
    case SKEL_SK_COMPOSE: return compose_variant_name(variant);
    case SKEL_SK_EDGE: {
        static const char *names[] = {"copy", "chunked", "direct"};
        return variant >= 0 && variant < 3 ? names[variant] : "?";
    }
    default: return "?";
    }
}

// ------------------------------------------------------- device status --

int skel_check_device(void *stream)
{
    return guarded([&] {
        cudaStream_t s = (cudaStream_t)stream;
        SKEL_CUDA_TRY(cudaStreamSynchronize(s));
        uint32_t err = 0;
        if (Control *ctl = scratch_control(s)) {
            SKEL_CUDA_TRY(cudaMemcpy(&err, &ctl->error, sizeof(err), cudaMemcpyDeviceToHost));
            if (err) SKEL_CUDA_TRY(cudaMemset(&ctl->error, 0, sizeof(uint32_t)));
        }
        // the allocation-free scan records into its own static control block
        uint32_t err_static = 0;
        int rc = noalloc_take_status(&err_static);
        if (rc) return rc;
        err |= err_static;
        if (err) {
            if (err & kErrTimeout)
                return fail(SKEL_ERR_TIMEOUT, "a bounded device wait (scan look-back) gave up; results of that call are invalid");
            if (err & kErrInput)
                return fail(SKEL_ERR_INVALID_ARG, "batched offsets were not a valid CSR offset array; that call did nothing");
        }
        return (int)SKEL_OK;
    });
}

int skel_set_debug(int key, int64_t value) { return guarded([&] { return set_debug(key, value); }); }

// ------------------------------------------------------------- probes --

int skel_probe_empty_launches(int count, void *stream)
{
    return guarded([&] {
        if (count < 0) return fail(SKEL_ERR_INVALID_ARG, "probe: count must be >= 0");
        return probe_launch_empty(count, (cudaStream_t)stream);
    });
}

int skel_probe_l2_random(const float *table, int64_t m, int64_t reads, float *sink, int64_t *reads_made, void *stream)
{
    return guarded([&] {
        if (!table || !sink || !reads_made) return fail(SKEL_ERR_INVALID_ARG, "probe: NULL pointer");
        if (reads < 1) return fail(SKEL_ERR_INVALID_ARG, "probe: reads must be >= 1");
        int rc = probe_launch_l2_random(table, m, reads, sink, (cudaStream_t)stream);
        if (rc == SKEL_OK) *reads_made = probe_l2_random_reads(reads);
        return rc;
    });
}

int skel_probe_call_overhead(int calls, int64_t n, double *us_call, double *us_launch, void *stream)
{
    return guarded([&] {
        if (calls < 1 || n < 1 || !us_call || !us_launch) return fail(SKEL_ERR_INVALID_ARG, "probe: bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t shape[1] = {n};
        skel_handle x = nullptr, y = nullptr, o = nullptr;
        int rc = skel_container_create(SKEL_F32, 1, shape, &x);
        if (!rc) rc = skel_container_create(SKEL_F32, 1, shape, &y);
        if (!rc) rc = skel_container_create(SKEL_F32, 1, shape, &o);
        const double a = 2.5;
        const skel_handle ins[2] = {x, y};
        void *px = nullptr, *py = nullptr, *po = nullptr;
        if (!rc) rc = skel_container_device_ptr(x, SKEL_WRITE, stream, &px);     // device-valid operands
        if (!rc) rc = skel_container_device_ptr(y, SKEL_WRITE, stream, &py);
        if (!rc) rc = skel_container_device_ptr(o, SKEL_WRITE, stream, &po);
        for (int k = 0; k < 10 && !rc; ++k) rc = skel_map(SKEL_FN_AXPY, &a, 1, ins, 2, o, stream);
        if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "probe sync");
        // the whole call: argument checks, table lookup, coherence steps, launch
        auto t0 = std::chrono::steady_clock::now();
        for (int k = 0; k < calls && !rc; ++k) rc = skel_map(SKEL_FN_AXPY, &a, 1, ins, 2, o, stream);
        auto t1 = std::chrono::steady_clock::now();
        if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "probe sync");
        // the same kernel launched directly with the choice the call made
        Choice c{};
        if (!rc) rc = last_choice(SKEL_SK_MAP, &c);
        MapLaunch m{SKEL_FN_AXPY, (float)a, (const float *)px, (const float *)py, (float *)po, n};
        auto t2 = std::chrono::steady_clock::now();
        for (int k = 0; k < calls && !rc; ++k) rc = launch_map(m, c, s);
        auto t3 = std::chrono::steady_clock::now();
        if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "probe sync");
        for (skel_handle h : {x, y, o})
            if (h) skel_container_destroy(h);
        if (rc) return rc;
        *us_call = std::chrono::duration<double, std::micro>(t1 - t0).count() / calls;
        *us_launch = std::chrono::duration<double, std::micro>(t3 - t2).count() / calls;
        return (int)SKEL_OK;
    });
}

}  // extern "C"
