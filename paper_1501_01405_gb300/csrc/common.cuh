// Shared device helpers of the MRIP engine: the Philox4x32-10 stream, the
// 53-bit uniform and exponential variates, launch plumbing and the library's
// error state.  Written for sm_103a (GB300).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mrip.h"

namespace mrip {

// A named NVTX range for the lifetime of the object (host timeline; profilers
// can attribute and filter the kernels a call launches by it).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Bounds checks of a debug build (-DMRIP_DEBUG).
//
// MRIP_CHECK(cond, site, index) guards one access: in a release build it is
// the constant true and the compiler drops it; in a debug build a false
// cond records (site, index) in this translation unit's record -- the first
// failure since the record was last read wins -- and evaluates to false, so
// the caller skips (or clamps) the access.  Nothing traps, asserts or waits.
// Sites are numbered per file (forest fire 1xx, queues 2xx, walk 3xx,
// network 4xx, control variate 5xx, area walk 6xx, statistics 7xx); the
// host reads and clears the records with mrip_debug_checks.
// ---------------------------------------------------------------------------
#ifdef MRIP_DEBUG
static __device__ unsigned long long g_check_first;

__device__ __forceinline__ bool check_record(bool ok, unsigned site, long long index) {
    if (!ok) {
        const unsigned long long rec =
            (static_cast<unsigned long long>(site) << 40) | (static_cast<unsigned long long>(index) & ((1ull << 40) - 1));
        atomicCAS(&g_check_first, 0ull, rec);
    }
    return ok;
}

#define MRIP_CHECK(cond, site, index) \
    (::mrip::check_record(static_cast<bool>(cond), (site), static_cast<long long>(index)))

// The host half of a unit's record: read it and put it back to zero.
#define MRIP_DEBUG_UNIT(name)                                                       \
    namespace mrip {                                                                \
    mrip_status debug_take_##name(unsigned long long* rec) {                        \
        const unsigned long long zero = 0;                                          \
        cudaError_t e = cudaMemcpyFromSymbol(rec, g_check_first, sizeof(*rec));     \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_first, &zero, sizeof(zero)); \
        return e == cudaSuccess ? MRIP_OK : cuda_status(e, "debug checks: " #name); \
    }                                                                               \
    }
#else
#define MRIP_CHECK(cond, site, index) true
#define MRIP_DEBUG_UNIT(name)
#endif

// Bytes of dynamic shared memory this launch was given (the PTX special
// register), for the debug checks of dynamically sized shared arrays.
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

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

// The full 64-bit product of two 32-bit words as one widening multiply
// (mul.wide.u32), both halves from one instruction.
__host__ __device__ __forceinline__ void mul_wide_u32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
#ifdef __CUDA_ARCH__
    unsigned long long r;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(b));
#else
    const uint64_t r = static_cast<uint64_t>(a) * b;
#endif
    hi = static_cast<uint32_t>(r >> 32);
    lo = static_cast<uint32_t>(r);
}

// One Philox4x32 round: products of (0xD2511F53, x0) and (0xCD9E8D57, x2);
// high halves xored with the other words and the round key; low halves
// moved to positions 1 and 3.
__host__ __device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                                      uint32_t& x3, uint32_t ka, uint32_t kb) {
#ifdef __CUDA_ARCH__
    uint32_t p0_lo, p0_hi, p1_lo, p1_hi;
    mul_wide_u32(0xD2511F53u, x0, p0_hi, p0_lo);
    mul_wide_u32(0xCD9E8D57u, x2, p1_hi, p1_lo);
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

// ---------------------------------------------------------------------------
// Exponential variates without the FP64 log.
//
// GB300's FP64 pipe retires about 2 FMAs per SM per clock, its integer pipes
// over 40 multiplies, so -log(1 - u) is evaluated in 64-bit fixed point
// (Tang's table-driven reduction, ACM TOMS 16(4), 1990, carried out in
// integers).  With 1 - u = K 2^-53, K in [1, 2^53], K = 2^e M, M in [1, 2):
//   -log(1 - u) = (53 - e) ln 2 - ln M,
//   ln M = ln c_j + log1p(r),  r = M / c_j - 1,  |r| < 2^-13,
// c_j the centre of the j-th of 4096 slices of [1, 2) (j = the 12 bits after
// the leading one), 1/c_j stored as a 63-bit fraction, ln c_j as a 64-bit
// fraction.  log1p(r) = r - r^2/2 + r^2 (r/3 - r^2/4) (the r^5 term is below
// 2^-67): r in 64-bit fixed point; r^2 from r's top 32 bits and one cross
// product (two 32x32 multiplies instead of a signed 64x64 high product, to
// 2^-64); the bracket and its product with r^2 in 32-bit pieces (one wide
// multiply), since their weight is below 2^-40; ln c_j + log1p(r) is summed
// and rounded once, unsigned; n ln 2 comes rounded from a 64-entry table.  The result carries an
// absolute error below 2^-56 (2^-57.0 in an exhaustive check of slice edges
// and centres at every exponent) before its one rounding to double, i.e.
// within about an ulp for -log(1 - u) > 1/16 and far below the ulp of any
// sum it enters.
// ---------------------------------------------------------------------------
constexpr int kLogSliceBits = 12;
constexpr int kLogSlices = 1 << kLogSliceBits;

struct __align__(16) LogSlice {
    unsigned long long inv;  // round(2^63 / c_j)
    unsigned long long lnc;  // round(-ln(inv 2^-63) 2^64) = ln c_j to 2^-64
};

struct LogTable {
    const LogSlice* slice;            // kLogSlices entries, device memory
    const unsigned long long* nln2;   // [n] = round(n ln 2 * 2^57), n = 0..63, device memory
    unsigned long long ln2_q64;       // round(ln 2 * 2^64)
};

// Table for the current device (built and uploaded on first use; call it
// outside stream capture before the first launch that needs it).
mrip_status log_table(LogTable* out);

// High 64 bits of a 64 x 64-bit product, short by 0, 1 or 2 units: of the
// four 32 x 32 partial products the lowest is dropped and the two middle ones
// enter by their high halves only (one wide multiply and two high products).
__device__ __forceinline__ unsigned long long umul64hi_trunc(unsigned long long a, unsigned long long b) {
    const uint32_t ah = static_cast<uint32_t>(a >> 32), al = static_cast<uint32_t>(a);
    const uint32_t bh = static_cast<uint32_t>(b >> 32), bl = static_cast<uint32_t>(b);
    return static_cast<unsigned long long>(ah) * bh + __umulhi(ah, bl) + __umulhi(al, bh);
}

// -log(K 2^-53) * 2^57 for K in [1, 2^53] (the result is below 53 ln 2 < 2^5.2,
// so it fits a signed 64-bit word).
__device__ __forceinline__ unsigned long long neg_log_q57(unsigned long long K, const LogTable& tab) {
    const int lz = __clzll(K);
    const unsigned long long m = K << lz;                   // bit 63 set: M = m 2^-63
    const unsigned long long n = static_cast<unsigned long long>(lz - 10);  // 53 - e
    const int j = static_cast<int>((m >> (63 - kLogSliceBits)) & (kLogSlices - 1));
    const ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2*>(tab.slice) + j);
    // m inv = 2^126 (1 + r); r 2^64 = (m inv - 2^126) >> 62 to 2^-60 (the
    // truncated high product is short by at most 2 units of 2^-62), |r 2^64| < 2^51
    const unsigned long long hi = umul64hi_trunc(m, e.x);
    const long long R = static_cast<long long>((hi - (1ULL << 62)) << 2);
    const int a = static_cast<int>(R >> 20);       // r 2^44, |a| < 2^31
    const int rho = static_cast<int>(R & 0xFFFFF);  // R = a 2^20 + rho
    // r^2 2^64 = (a^2 + a rho 2^-19) 2^-24 + rho^2 2^-64 (< 2^-24, dropped); < 2^38
    const long long r2 =
        (static_cast<long long>(a) * a + ((static_cast<long long>(a) * rho) >> 19)) >> 24;
    const int q = __mulhi(a, 1431655766) - static_cast<int>(r2 >> 22);  // (r/3 - r^2/4) 2^44
    const long long tail = (static_cast<long long>(static_cast<int>(r2 >> 7)) * q) >> 37;  // r^2 q 2^64
    const long long l1p = R - (r2 >> 1) + tail;                          // log1p(r) 2^64
    // ln M 2^64 + 2^6: below 2^64 (ln M < ln 2) and, the roundings being a
    // few units, never below zero, so the unsigned sum does not wrap
    const unsigned long long s64 = e.y + static_cast<unsigned long long>(l1p) + 64u;
    const unsigned long long nln2 = __ldg(tab.nln2 + n);  // n ln2 2^57, rounded (n <= 53)
    // No clamp is needed: for n >= 1 the exact result is at least
    // -ln(1 - 2^-53) (16 units) and the error below 2^-56 (2 units); for
    // n = 0 (K = 2^53, M = 1) s64 is 2^6 plus an error of a few units of
    // 2^-64, so s64 >> 7 = 0 = nln2.
    return nln2 - (s64 >> 7);
}

// Exponential variate from words (lo, hi): -log(1 - u) * inv_rate_q57 where
// inv_rate_q57 = 2^-57 / rate.
__device__ __forceinline__ double expo_fast(uint32_t lo, uint32_t hi, const LogTable& tab,
                                            double inv_rate_q57) {
    const unsigned long long bits = (static_cast<unsigned long long>(hi) << 32) | lo;
    const unsigned long long K = (1ULL << 53) - (bits >> 11);
    return __ull2double_rn(neg_log_q57(K, tab)) * inv_rate_q57;
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
