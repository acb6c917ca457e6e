// Shared device helpers of the MRIP engine: the Philox4x32-10 stream, the
// 53-bit uniform and exponential variates, launch plumbing and the library's
// error state.  Written for sm_103a (GB300).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mrip.h"

namespace mrip {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The ten round keys are
// fixed per seed, so the host expands them once and every kernel reads them
// from its parameter bank (uniform across the grid, no registers).
// ---------------------------------------------------------------------------
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline RoundKeys expand_key(uint64_t seed) {
    RoundKeys rk;
    uint32_t a = static_cast<uint32_t>(seed);
    uint32_t b = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = a;
        rk.k1[r] = b;
        a += 0x9E3779B9u;  // Weyl increments of the key schedule
        b += 0xBB67AE85u;
    }
    return rk;
}

// One Philox4x32 round: products of (0xD2511F53, x0) and (0xCD9E8D57, x2);
// high halves xored with the other words and the round key; low halves
// moved to positions 1 and 3.
__host__ __device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                                      uint32_t& x3, uint32_t ka, uint32_t kb) {
#ifdef __CUDA_ARCH__
    const uint32_t p0_lo = 0xD2511F53u * x0;
    const uint32_t p0_hi = __umulhi(0xD2511F53u, x0);
    const uint32_t p1_lo = 0xCD9E8D57u * x2;
    const uint32_t p1_hi = __umulhi(0xCD9E8D57u, x2);
#else
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * x0;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * x2;
    const uint32_t p0_lo = static_cast<uint32_t>(p0), p0_hi = static_cast<uint32_t>(p0 >> 32);
    const uint32_t p1_lo = static_cast<uint32_t>(p1), p1_hi = static_cast<uint32_t>(p1 >> 32);
#endif
    x0 = p1_hi ^ x1 ^ ka;
    x1 = p1_lo;
    x2 = p0_hi ^ x3 ^ kb;
    x3 = p0_lo;
}

__host__ __device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, rk.k0[r], rk.k1[r]);
    return make_uint4(c0, c1, c2, c3);
}

// Counter word 3: stream tag in the top byte, design point below.
__host__ __device__ __forceinline__ uint32_t stream_word(uint32_t tag, uint32_t dp) {
    return (tag << 24) | dp;
}

// u = (top 53 bits of hi:lo) * 2^-53, exact in double.
__device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
    const unsigned long long bits = (static_cast<unsigned long long>(hi) << 32) | lo;
    return __ull2double_rn(bits >> 11) * 0x1p-53;
}

// Exponential variate by inversion, -log(1 - u) / rate, IEEE divide.
__device__ __forceinline__ double expo_div(double u, double rate) {
    return -log(1.0 - u) / rate;
}

// Bernoulli threshold floor(p 2^32) for p in [0, 1) -- exact in double.
// Values outside [0, 1) (or NaN) are clamped to the nearest end.
__host__ __device__ __forceinline__ uint32_t threshold32(double p) {
    if (!(p > 0.0)) return 0u;
    if (p >= 1.0) return 0xFFFFFFFFu;
    return static_cast<uint32_t>(floor(p * 4294967296.0));
}

// ---------------------------------------------------------------------------
// Host-side error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
mrip_status fail(mrip_status code, const std::string& msg);
mrip_status cuda_status(cudaError_t e, const char* what);
mrip_status launch_status(const char* what);

// Scratch memory shared by the stage entry points of one device: grows on
// demand, never shrinks, freed at exit.
void* scratch(size_t bytes, int slot);
int* device_error_flags();
int sm_count();

inline unsigned ceil_div_u(long long a, long long b) {
    return static_cast<unsigned>((a + b - 1) / b);
}

}  // namespace mrip
