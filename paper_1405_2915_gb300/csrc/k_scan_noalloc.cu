// Allocation-free scan (skel_scan_noalloc): the single-pass look-back scan
// over raw device pointers, with its scratch -- the control block (tile
// ticket, finished-block counter, status word, abort tag, look-back tag) and
// the look-back descriptor words -- in a file-scope static device array
// instead of allocated memory.  The array is part of the loaded module: every
// device that loads the library holds it until the process exits, and every
// call shares it.
//
// The look-back tag of a call lives in the array too: each block reads it
// when it starts, and the block that finishes last advances it (and clears
// the descriptor words when the 8-bit tag space is used up).  A call
// therefore needs no host-side state besides the array's address, and the
// tag of every call follows from the calls before it in stream order.
#include <map>
#include <mutex>

#include "scan_tile.cuh"

namespace skel {
namespace {

using dev::LookbackDesc;
using dev::ScanTypes;
using dev::TileMap;

constexpr int kBlock = 256;
constexpr int kV = 4;                                   // 16 elements per thread
constexpr int kTile = kBlock * 4 * kV;                  // 4096 elements per tile
constexpr int64_t kMaxTiles = SKEL_SCAN_NOALLOC_MAX_N / kTile;
constexpr size_t kWordsBytes = 2 * kMaxTiles * sizeof(uint64_t);   // aggregate + prefix word per tile

// 256-byte control block followed by the descriptor words (512 KiB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(Control) + kWordsBytes];

template <class T, bool INCL>
__global__ void __launch_bounds__(kBlock)
scan_noalloc_kernel(const T *__restrict__ in, T *__restrict__ out, int64_t n, int64_t ntiles, unsigned char *scratch,
                    int64_t skip_tile, uint64_t limit_ns, bool vec_ok)
{
    using CT = typename ScanTypes<T>::CT;
    __shared__ T smem[kBlock / 32 + 1];
    __shared__ int64_t s_tile;
    __shared__ uint32_t s_epoch;
    __shared__ int s_last;
    __shared__ CT s_prefix;
    Control *ctl = reinterpret_cast<Control *>(scratch);
    uint64_t *words = reinterpret_cast<uint64_t *>(scratch + sizeof(Control));
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(&ctl->ticket, 1u);
        if ((int64_t)t == ntiles - 1) ctl->ticket = 0u;   // last ticket: every block has drawn; ready for the next call
        s_tile = t;
        // the tag the previous call left, plus one: 1..kMaxEpoch (no block of
        // this call changes it before every block has read it, below)
        s_epoch = dev::ld_volatile(&ctl->epoch) + 1u;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    const uint32_t epoch = s_epoch;
    TileMap m;
    m.base = tile * kTile;
    m.len = n - m.base < kTile ? n - m.base : kTile;
    m.rev = false;
    m.vec = vec_ok && m.len == kTile;
    T v[kV][4];
    dev::tile_load<T, kBlock, kV>(in, m, v);
    const T agg = dev::tile_scan_local<T, INCL, kBlock, kV>(v, smem);
    if (threadIdx.x < 32) {
        const LookbackDesc d{words, words + kMaxTiles};
        const CT p = dev::lookback<CT>(tile, 0, (CT)agg, d, epoch, ctl, limit_ns, tile != skip_tile);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
    dev::tile_add_prefix<T, kV>(v, dev::to_elem<T>(s_prefix));
    dev::tile_store<T, kBlock, kV>(out, m, v);
    // This block's look-back reads are done (warp 0 finished them before the
    // barrier above).  The block that finishes last therefore knows that no
    // block of this call reads the tag or the words any more: it advances the
    // tag for the next call, and when the tag space is used up it clears the
    // words and the abort tag and restarts at 1.
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->done, 1u) == (uint32_t)(ntiles - 1);
    }
    __syncthreads();
    if (s_last) {
        if (epoch >= kMaxEpoch) {
            uint4 *w4 = reinterpret_cast<uint4 *>(words);
            for (size_t i = threadIdx.x; i < kWordsBytes / sizeof(uint4); i += kBlock) w4[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (threadIdx.x == 0) {
            ctl->done = 0u;
            if (epoch >= kMaxEpoch) {
                ctl->abort = 0u;
                ctl->epoch = 0u;
            } else {
                ctl->epoch = epoch;
            }
        }
    }
}

// Per-device state: the array's device address.
struct DevState {
    unsigned char *scratch = nullptr;
};
std::mutex g_mu;
std::map<int, DevState> g_dev;

// Once per device, with that device current: look up the array's address.
// A host-side reference to g_noalloc_scratch is only a stand-in symbol, not
// a device address, so it is never passed to a kernel.
int setup(int dev, cudaStream_t s, DevState **out)
{
    DevState &st = g_dev[dev];
    if (!st.scratch) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "skel_scan_noalloc: cudaGetSymbolAddress of the static scratch");
        // the array is zero at load; clear it once more so that a tile
        // ticket or word left by nothing can never be read (no allocation)
        e = cudaMemsetAsync(p, 0, sizeof(g_noalloc_scratch), s);
        if (e != cudaSuccess) return fail_cuda(e, "skel_scan_noalloc: clearing the static scratch");
        st.scratch = static_cast<unsigned char *>(p);
    }
    *out = &st;
    return SKEL_OK;
}

template <class T>
int run(int inclusive, const void *in, void *out, int64_t n, unsigned char *scratch, cudaStream_t s)
{
    const int64_t ntiles = ceil_div(n, kTile);
    const bool vec_ok = aligned16(in) && aligned16(out);
    const DebugKnobs k = debug_knobs();
    if (inclusive)
        launch_kernel(scan_noalloc_kernel<T, true>, (unsigned)ntiles, kBlock, 0, s, static_cast<const T *>(in),
                      static_cast<T *>(out), n, ntiles, scratch, k.scan_skip_publish_tile, k.wait_limit_ns, vec_ok);
    else
        launch_kernel(scan_noalloc_kernel<T, false>, (unsigned)ntiles, kBlock, 0, s, static_cast<const T *>(in),
                      static_cast<T *>(out), n, ntiles, scratch, k.scan_skip_publish_tile, k.wait_limit_ns, vec_ok);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "skel_scan_noalloc launch");
}

}  // namespace

int noalloc_take_status(uint32_t *err)
{
    *err = 0;
    int dev = 0;
    SKEL_CUDA_TRY(cudaGetDevice(&dev));
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_dev.find(dev);
        if (it != g_dev.end()) scratch = it->second.scratch;
    }
    if (!scratch) return SKEL_OK;
    uint32_t *word = &reinterpret_cast<Control *>(scratch)->error;
    SKEL_CUDA_TRY(cudaMemcpy(err, word, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (*err) SKEL_CUDA_TRY(cudaMemset(word, 0, sizeof(uint32_t)));
    return SKEL_OK;
}

}  // namespace skel

using namespace skel;

extern "C" int skel_scan_noalloc(skel_fn op, int inclusive, skel_dtype dtype, const void *in, void *out, int64_t n,
                                 void *stream)
{
    try {
        clear_error();
        if (op != SKEL_FN_ADD) return fail(SKEL_ERR_UNSUPPORTED, "skel_scan_noalloc: op must be ADD");
        if (dtype != SKEL_F32 && dtype != SKEL_I32) return fail(SKEL_ERR_DTYPE, "skel_scan_noalloc: float32 or int32 only");
        if (n < 0) return fail(SKEL_ERR_SHAPE, "skel_scan_noalloc: n must be >= 0");
        if (n > SKEL_SCAN_NOALLOC_MAX_N)
            return fail(SKEL_ERR_SHAPE, "skel_scan_noalloc: n exceeds SKEL_SCAN_NOALLOC_MAX_N (2^27 elements), the "
                                        "capacity of its static scratch; use skel_scan");
        if (n == 0) return SKEL_OK;
        if (!in || !out) return fail(SKEL_ERR_INVALID_ARG, "skel_scan_noalloc: NULL pointer");
        const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
        if (a < b + 4 * n && b < a + 4 * n) return fail(SKEL_ERR_INVALID_ARG, "skel_scan_noalloc: out overlaps in");
        cudaStream_t s = (cudaStream_t)stream;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return fail_cuda(e, "skel_scan_noalloc: cudaGetDevice");
        std::lock_guard<std::mutex> lk(g_mu);
        DevState *st = nullptr;
        int rc = setup(dev, s, &st);
        if (rc) return rc;
        return dtype == SKEL_F32 ? run<float>(inclusive, in, out, n, st->scratch, s)
                                 : run<uint32_t>(inclusive, in, out, n, st->scratch, s);
    } catch (...) {
        return fail(SKEL_ERR_INVALID_ARG, "skel_scan_noalloc: unexpected exception");
    }
}
