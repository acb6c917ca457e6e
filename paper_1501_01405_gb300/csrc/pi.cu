// Monte Carlo pi (paper, Section 5.1, first model): points in the unit
// square counted when they fall in the quarter disc.  Draw k of replication
// `rep` uses words 2(k mod 2), 2(k mod 2)+1 of Philox block (c0 = 0,
// c1 = k div 2) as integer coordinates x, y in [0, 2^32); it is inside iff
// x^2 + y^2 < 2^64, tested exactly as x^2 <= (2^64 - 1) - y^2.
//
// Draws are independent, so a replication is split over CTAs of 2^16 draws
// (a 10^7-draw replication spreads over ~150 CTAs, i.e. the whole GPU even
// for one replication); each CTA reduces its count (warp reduction, then
// shared memory) and adds it to the replication's counter with one 64-bit
// atomic -- integer addition, so the result does not depend on the order.
#include "common.cuh"

namespace mrip {
namespace {

constexpr int kPiThreads = 256;
constexpr long long kPiChunk = 1LL << 16;  // draws per CTA (even)

__device__ __forceinline__ uint32_t inside(uint32_t x, uint32_t y) {
    const unsigned long long x2 = static_cast<unsigned long long>(x) * x;
    const unsigned long long y2 = static_cast<unsigned long long>(y) * y;
    return x2 <= ~y2 ? 1u : 0u;
}

__global__ void __launch_bounds__(kPiThreads) pi_kernel(long long n_draws, long long chunks, long long rep0,
                                                        const __grid_constant__ RoundKeys rk,
                                                        unsigned long long* __restrict__ hits) {
    __shared__ uint32_t part[kPiThreads / 32];
    const long long rep = blockIdx.x / chunks;
    const long long start = (blockIdx.x - rep * chunks) * kPiChunk;
    const long long end = min(start + kPiChunk, n_draws);
    const uint32_t c3 = stream_word(0u, 0u);
    uint32_t cnt = 0;
    for (long long b = start / 2 + threadIdx.x; 2 * b < end; b += kPiThreads) {
        const uint4 w = philox(0u, static_cast<uint32_t>(b), static_cast<uint32_t>(rep0 + rep), c3, rk);
        cnt += inside(w.x, w.y);
        if (2 * b + 1 < end) cnt += inside(w.z, w.w);
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int i = 0; i < kPiThreads / 32; ++i) tot += part[i];
        atomicAdd(hits + rep, tot);
    }
}

}  // namespace
}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_pi_simulate(int64_t rep0, int64_t n_reps, int64_t n_draws, uint64_t seed,
                                        int64_t* d_hits, void* stream) {
    if (rep0 < 0 || n_reps < 0 || n_draws < 0) return fail(MRIP_EINVAL, "mrip_pi_simulate: negative size");
    if (rep0 + n_reps > 0x100000000ll || n_draws > (1LL << 33))
        return fail(MRIP_EINVAL, "mrip_pi_simulate: replication indices < 2^32, n_draws <= 2^33");
    if (n_reps == 0) return MRIP_OK;
    if (!d_hits) return fail(MRIP_EINVAL, "mrip_pi_simulate: null output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d_hits, 0, static_cast<size_t>(n_reps) * sizeof(int64_t), st);
    if (e != cudaSuccess) return cuda_status(e, "mrip_pi_simulate: clear");
    if (n_draws == 0) return MRIP_OK;
    const long long chunks = (n_draws + kPiChunk - 1) / kPiChunk;
    if (chunks * n_reps > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_pi_simulate: too many draws in total");
    pi_kernel<<<static_cast<unsigned>(chunks * n_reps), kPiThreads, 0, st>>>(
        n_draws, chunks, rep0, expand_key(seed), reinterpret_cast<unsigned long long*>(d_hits));
    return launch_status("mrip_pi_simulate");
}
