// Allocation-free scan (skel_scan_noalloc): the single-pass look-back scan
// over raw device pointers, with its scratch -- the control block (tile ticket,
// abort tag) and the look-back descriptor words -- in a file-scope static
// device array instead of allocated memory.  The array is part of the loaded
// module: every device that loads the library holds it until the process
// exits, and every call shares it.
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
                    uint32_t epoch, uint64_t limit_ns, bool vec_ok)
{
    using CT = typename ScanTypes<T>::CT;
    __shared__ T smem[kBlock / 32 + 1];
    __shared__ int64_t s_tile;
    __shared__ CT s_prefix;
    Control *ctl = reinterpret_cast<Control *>(scratch);
    uint64_t *words = reinterpret_cast<uint64_t *>(scratch + sizeof(Control));
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(&ctl->ticket, 1u);
        if ((int64_t)t == ntiles - 1) ctl->ticket = 0u;   // last ticket: every block has drawn; ready for the next call
        s_tile = t;
    }
    __syncthreads();
    const int64_t tile = s_tile;
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
        const CT p = dev::lookback<CT>(tile, 0, (CT)agg, d, epoch, ctl, limit_ns, true);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
    dev::tile_add_prefix<T, kV>(v, dev::to_elem<T>(s_prefix));
    dev::tile_store<T, kBlock, kV>(out, m, v);
}

// Per-device state: the array's device address and the epoch counter of
// the descriptor words.
struct DevState {
    unsigned char *scratch = nullptr;
    uint32_t epoch = 0;
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
        st.epoch = 0;
    }
    *out = &st;
    return SKEL_OK;
}

template <class T>
int run(int inclusive, const void *in, void *out, int64_t n, unsigned char *scratch, uint32_t epoch,
        cudaStream_t s)
{
    const int64_t ntiles = ceil_div(n, kTile);
    const bool vec_ok = aligned16(in) && aligned16(out);
    const uint64_t limit = debug_knobs().wait_limit_ns;
    if (inclusive)
        launch_kernel(scan_noalloc_kernel<T, true>, (unsigned)ntiles, kBlock, 0, s, static_cast<const T *>(in),
                      static_cast<T *>(out), n, ntiles, scratch, epoch, limit, vec_ok);
    else
        launch_kernel(scan_noalloc_kernel<T, false>, (unsigned)ntiles, kBlock, 0, s, static_cast<const T *>(in),
                      static_cast<T *>(out), n, ntiles, scratch, epoch, limit, vec_ok);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "skel_scan_noalloc launch");
}

}  // namespace
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
        st->epoch += 1;
        if (st->epoch > kMaxEpoch) {   // tag space used up: clear the words and the abort tag, restart
            st->epoch = 1;
            e = cudaMemsetAsync(st->scratch + sizeof(Control), 0, kWordsBytes, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(&reinterpret_cast<Control *>(st->scratch)->abort, 0, sizeof(uint32_t), s);
            if (e != cudaSuccess) return fail_cuda(e, "skel_scan_noalloc: clearing the static scratch");
        }
        return dtype == SKEL_F32 ? run<float>(inclusive, in, out, n, st->scratch, st->epoch, s)
                                 : run<uint32_t>(inclusive, in, out, n, st->scratch, st->epoch, s);
    } catch (...) {
        return fail(SKEL_ERR_INVALID_ARG, "skel_scan_noalloc: unexpected exception");
    }
}
