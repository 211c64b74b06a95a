// Measurement probes: kernels that compute no skeleton but measure the
// hardware ceilings the skeletons are judged against on this GPU.
//
//   probe_empty        an empty kernel: back-to-back launches of it give the
//                      launch floor of a call made of k dependent launches
//                      (the latency bound of the small MapReduce).
//   probe_l2_random    random 4-byte reads from a table that stays in L2
//                      (MapArray gather's access pattern without its index
//                      and output streams): the L2's random-sector rate, the
//                      roofline of the gather.  Indices come from a per-thread
//                      generator in registers, so no HBM stream competes.
#include "common.cuh"

namespace skel {
namespace {

__global__ void probe_empty() {}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Each thread makes `per_thread` reads in batches of 8 independent loads;
// the sum is written only if it equals a value it cannot take (NaN never
// equals itself), so the loads stay live without an output stream.
__global__ void __launch_bounds__(256) probe_l2_random(const float *__restrict__ A, uint32_t mask, int per_thread,
                                                       uint64_t seed, float *__restrict__ sink)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // per-thread stream: a 64-bit linear congruential step (Knuth's MMIX
    // constants) from a hashed start; the index is the state's high bits
    uint64_t x = mix64(seed + (tid + 1) * 0x9E3779B97F4A7C15ull);
    float acc = 0.f;
    for (int r = 0; r < per_thread; r += 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            v[k] = __ldg(A + ((uint32_t)(x >> 32) & mask));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += v[k];
    }
    if (acc != acc) *sink = acc;
}

}  // namespace

int probe_launch_empty(int count, cudaStream_t s)
{
    for (int k = 0; k < count; ++k) launch_kernel(probe_empty, 1, 32, 0, s);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "probe_empty launch");
}

int probe_launch_l2_random(const float *table, int64_t m, int64_t reads, float *sink, cudaStream_t s)
{
    if (m < 1 || (m & (m - 1)) || m > (int64_t(1) << 31))
        return fail(SKEL_ERR_SHAPE, "probe: table length must be a power of two <= 2^31");
    const int block = 256;
    const int64_t blocks = (int64_t)device_info().sms * 8;          // one full wave at 8 blocks per SM
    const int64_t threads = blocks * block;
    int64_t per = ceil_div(reads, threads);
    per = ceil_div(per, 8) * 8;
    if (per > (int64_t(1) << 30)) return fail(SKEL_ERR_SHAPE, "probe: too many reads");
    launch_kernel(probe_l2_random, (unsigned)blocks, block, 0, s, table, (uint32_t)(m - 1), (int)per,
                  (uint64_t)0x1405291500ull, sink);
    cudaError_t e = cudaPeekAtLastError();
    return e == cudaSuccess ? SKEL_OK : fail_cuda(cudaGetLastError(), "probe_l2_random launch");
}

int64_t probe_l2_random_reads(int64_t reads)
{
    const int64_t threads = (int64_t)device_info().sms * 8 * 256;
    return ceil_div(ceil_div(reads, threads), 8) * 8 * threads;
}

}  // namespace skel
