// Throughput of the widening 32 x 32 -> 64-bit multiply on this GPU: the
// unit that bounds the Philox4x32-10 stream (two such products per round).
// The measured rate is the denominator of a roofline for kernels whose work
// is Philox blocks; the nominal alternatives (issue slots, 64 multiply
// results per SM-clock) are derived from unit counts, this one is timed.
//
// Each thread runs kChains independent chains a <- hi(a M) ^ lo(a M) (one
// widening multiply and one logic operation per step), so the multiply unit,
// not latency, is the limit at full occupancy; the chains' final values are
// folded into one word per thread and stored so that nothing is dead code.
#include "common.cuh"

namespace mrip {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) mul_wide_probe(uint32_t seed, int iters, uint32_t* sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + 977u * (blockIdx.x * kProbeThreads + threadIdx.x) + 131u * k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            uint32_t hi, lo;
            mul_wide_u32(a[k], 0xD2511F53u, hi, lo);
            a[k] = hi ^ lo;
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x ^= a[k];
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = x;
}

}  // namespace
}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_probe_mul_wide(double* warp_products_per_s, void* stream) {
    if (!warp_products_per_s) return fail(MRIP_EINVAL, "mrip_probe_mul_wide: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = sm_count() * (2048 / kProbeThreads);  // every SM full
    const int iters = 4096;
    uint32_t* sink = static_cast<uint32_t*>(scratch(static_cast<size_t>(blocks) * kProbeThreads * 4, 5));
    if (!sink) return fail(MRIP_ENOMEM, "mrip_probe_mul_wide: scratch allocation failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    mul_wide_probe<<<blocks, kProbeThreads, 0, st>>>(1u, iters / 8, sink);  // warm-up
    cudaEventRecord(e0, st);
    mul_wide_probe<<<blocks, kProbeThreads, 0, st>>>(2u, iters, sink);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e, "mrip_probe_mul_wide");
    const double warps = static_cast<double>(blocks) * kProbeThreads / 32.0;
    *warp_products_per_s = warps * iters * kChains / (ms * 1e-3);
    return MRIP_OK;
}
