// Library runtime: thread-local error state, per-device scratch memory,
// device error flags, and the random-stream stage entry points
// (mrip_philox, mrip_expo).
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace mrip {

namespace {
thread_local std::string g_last_error;

struct DeviceScratch {
    void* ptr[8] = {nullptr};
    size_t bytes[8] = {0};
    int* flags = nullptr;
    int sms = 0;
    LogSlice* log_slices = nullptr;
};
std::mutex g_scratch_mutex;
std::vector<DeviceScratch> g_scratch;

DeviceScratch& dev_scratch() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (static_cast<int>(g_scratch.size()) <= dev) g_scratch.resize(dev + 1);
    return g_scratch[dev];
}
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

mrip_status fail(mrip_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

mrip_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MRIP_OK;
    return fail(MRIP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

mrip_status launch_status(const char* what) { return cuda_status(cudaGetLastError(), what); }

void* scratch(size_t bytes, int slot) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch& d = dev_scratch();
    if (d.bytes[slot] >= bytes && d.ptr[slot]) return d.ptr[slot];
    if (d.ptr[slot]) {
        cudaDeviceSynchronize();  // the old buffer may still be in use
        cudaFree(d.ptr[slot]);
        d.ptr[slot] = nullptr;
        d.bytes[slot] = 0;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    if (cudaMalloc(&d.ptr[slot], want) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    d.bytes[slot] = want;
    return d.ptr[slot];
}

int* device_error_flags() {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch& d = dev_scratch();
    if (!d.flags) {
        if (cudaMalloc(&d.flags, 16 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            d.flags = nullptr;
            return nullptr;
        }
        cudaMemset(d.flags, 0, 16 * sizeof(int));
    }
    return d.flags;
}

namespace {
// 1/c_j and ln c_j for the slices of [1, 2), from the host's long-double
// logarithm (64-bit or wider mantissa).
void build_log_slices(std::vector<LogSlice>& t) {
    t.resize(kLogSlices);
    for (int j = 0; j < kLogSlices; ++j) {
        const long double c = 1.0L + (static_cast<long double>(j) + 0.5L) / static_cast<long double>(kLogSlices);
        const unsigned long long inv =
            static_cast<unsigned long long>(ldexpl(1.0L / c, 63) + 0.5L);
        const long double ic = ldexpl(static_cast<long double>(inv), -63);
        const long double lnc = -logl(ic);
        t[j].inv = inv;
        t[j].lnc = static_cast<unsigned long long>(ldexpl(lnc, 64) + 0.5L);
    }
}
}  // namespace

mrip_status log_table(LogTable* out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch& d = dev_scratch();
    const unsigned long long ln2_q64 = static_cast<unsigned long long>(ldexpl(logl(2.0L), 64) + 0.5L);
    if (!d.log_slices) {
        std::vector<LogSlice> t;
        build_log_slices(t);
        // n ln2 2^57 rounded, from the 128-bit product n * round(ln2 2^64)
        std::vector<unsigned long long> nln2(64);
        for (unsigned n = 0; n < 64; ++n) {
            const unsigned __int128 prod = static_cast<unsigned __int128>(n) * ln2_q64 + 64u;
            nln2[n] = static_cast<unsigned long long>(prod >> 7);
        }
        const size_t slice_bytes = t.size() * sizeof(LogSlice);
        LogSlice* p = nullptr;
        cudaError_t e = cudaMalloc(&p, slice_bytes + nln2.size() * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemcpy(p, t.data(), slice_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(reinterpret_cast<char*>(p) + slice_bytes, nln2.data(),
                           nln2.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (p) cudaFree(p);
            return cuda_status(e, "log table upload");
        }
        d.log_slices = p;
    }
    out->slice = d.log_slices;
    out->nln2 = reinterpret_cast<const unsigned long long*>(d.log_slices + kLogSlices);
    out->ln2_q64 = ln2_q64;
    return MRIP_OK;
}

int sm_count() {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DeviceScratch& d = dev_scratch();
    if (d.sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (d.sms <= 0) d.sms = 1;
    }
    return d.sms;
}

// ---------------------------------------------------------------------------
// Random-stream stages
// ---------------------------------------------------------------------------
__global__ void philox_kernel(const uint4* __restrict__ ctr, const uint2* __restrict__ key,
                              long long n, uint4* __restrict__ out) {
    long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    uint4 c = ctr[i];
    uint2 k = key[i];
    uint32_t a = k.x, b = k.y;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c.x, c.y, c.z, c.w, a, b);
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    out[i] = c;
}

__global__ void expo_kernel(const uint32_t* __restrict__ lo, const uint32_t* __restrict__ hi,
                            const double* __restrict__ rate, long long n, double* __restrict__ u_out,
                            double* __restrict__ e_out, LogTable tab) {
    long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    if (u_out) u_out[i] = u53(lo[i], hi[i]);
    if (e_out) e_out[i] = expo_fast(lo[i], hi[i], tab, 0x1p-57 / rate[i]);
}

}  // namespace mrip

using namespace mrip;

extern "C" const char* mrip_last_error(void) { return g_last_error.c_str(); }

extern "C" mrip_status mrip_philox(const uint32_t* d_ctr, const uint32_t* d_key, int64_t n,
                                   uint32_t* d_out, void* stream) {
    if (n < 0) return fail(MRIP_EINVAL, "mrip_philox: n < 0");
    if (n == 0) return MRIP_OK;
    if (!d_ctr || !d_key || !d_out) return fail(MRIP_EINVAL, "mrip_philox: null pointer");
    if ((reinterpret_cast<uintptr_t>(d_ctr) | reinterpret_cast<uintptr_t>(d_out)) & 15u ||
        reinterpret_cast<uintptr_t>(d_key) & 7u)
        return fail(MRIP_EINVAL, "mrip_philox: misaligned buffer (ctr/out need 16 B, key 8 B)");
    philox_kernel<<<ceil_div_u(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(d_ctr), reinterpret_cast<const uint2*>(d_key), n,
        reinterpret_cast<uint4*>(d_out));
    return launch_status("mrip_philox");
}

extern "C" mrip_status mrip_expo(const uint32_t* d_lo, const uint32_t* d_hi, const double* d_rate,
                                 int64_t n, double* d_u, double* d_e, void* stream) {
    if (n < 0) return fail(MRIP_EINVAL, "mrip_expo: n < 0");
    if (n == 0) return MRIP_OK;
    if (!d_lo || !d_hi || (d_e && !d_rate)) return fail(MRIP_EINVAL, "mrip_expo: null pointer");
    LogTable tab;
    mrip_status s = log_table(&tab);
    if (s != MRIP_OK) return s;
    expo_kernel<<<ceil_div_u(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_lo, d_hi, d_rate, n, d_u, d_e, tab);
    return launch_status("mrip_expo");
}

#ifdef MRIP_DEBUG
namespace mrip {
namespace {
// One deliberately failed check (site 999, index 12345): no access is
// guarded by it, it only exercises the record.
__global__ void debug_selftest_kernel() { (void)MRIP_CHECK(threadIdx.x != 0, 999, 12345); }
}  // namespace
mrip_status debug_take_runtime(unsigned long long* rec);
mrip_status debug_take_forest_fire(unsigned long long* rec);
mrip_status debug_take_queues(unsigned long long* rec);
mrip_status debug_take_walk(unsigned long long* rec);
mrip_status debug_take_mlp(unsigned long long* rec);
mrip_status debug_take_cv(unsigned long long* rec);
mrip_status debug_take_area_walk(unsigned long long* rec);
mrip_status debug_take_stats(unsigned long long* rec);
}  // namespace mrip
#endif

extern "C" mrip_status mrip_debug_checks(int32_t* enabled, uint64_t* first) {
    if (!enabled || !first) return fail(MRIP_EINVAL, "mrip_debug_checks: null argument");
    *first = 0;
#ifdef MRIP_DEBUG
    *enabled = 1;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e, "mrip_debug_checks");
    using Take = mrip_status (*)(unsigned long long*);
    const Take units[] = {debug_take_runtime, debug_take_forest_fire, debug_take_queues,
                          debug_take_walk,    debug_take_mlp,         debug_take_cv,
                          debug_take_area_walk, debug_take_stats};
    for (Take take : units) {  // every unit is read (and cleared); the first record is kept
        unsigned long long rec = 0;
        const mrip_status s = take(&rec);
        if (s != MRIP_OK) return s;
        if (*first == 0) *first = rec;
    }
#else
    *enabled = 0;
#endif
    return MRIP_OK;
}

extern "C" mrip_status mrip_debug_selftest(void) {
#ifdef MRIP_DEBUG
    debug_selftest_kernel<<<1, 32>>>();
    return launch_status("mrip_debug_selftest");
#else
    return fail(MRIP_EINVAL, "mrip_debug_selftest: not a debug build");
#endif
}

extern "C" mrip_status mrip_check_device_flags(void) {
    int* flags = device_error_flags();
    if (!flags) return fail(MRIP_ENOMEM, "device error flags: allocation failed");
    int host[16];
    cudaError_t e = cudaMemcpy(host, flags, sizeof(host), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e, "mrip_check_device_flags");
    if (host[0] != 0) {
        cudaMemset(flags, 0, sizeof(host));
        return fail(MRIP_ESTEPCAP, "a replication reached its step cap (its output is -1)");
    }
    return MRIP_OK;
}

MRIP_DEBUG_UNIT(runtime)
