// Per-design-point statistics of the replication outputs (paper, Section 1:
// the replication mean and a CLT confidence interval) and the Student-t
// critical value.
//
// Device: one CTA per design point and slice of at most 4,096 replications
// computes the slice's (n, mean, M2) by the two-pass definition in a fixed
// summation order; a second kernel merges the slices' triples
// in slice order with Chan, Golub and LeVeque's pairwise formula (1979), so
// the result does not depend on scheduling.
//
// Host: t_{(1+conf)/2, df} from Abramowitz & Stegun 26.7.3/26.7.4 (finite
// series in cos^2(theta) for integer df), evaluated innermost-first
// (Horner) in double-double, and solved by a bracketed Newton iteration
// whose density comes from lgamma.
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace mrip {
namespace {

constexpr int kStatsThreads = 256;
constexpr int kGroups = kStatsThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Sum of a warp's values into lane 0 (fixed shuffle tree).
__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(kFull, a, off);
    return a;
}

// The 8 warp totals in a fixed pairwise order.
__device__ __forceinline__ double total8(const double* g) {
    return ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]));
}

// One CTA per (design point, slice of replications): (n, mean, M2) of the
// slice by the corrected two-pass algorithm (Chan, Golub, LeVeque 1983):
// m = (sum of x) / n, then with d = x - m the exact mean is m + (sum d) / n
// and M2 = sum d^2 - (sum d)^2 / n; the corrections cancel the first-order
// effect of the rounding of m (data with a large mean and a small spread).
// Thread t sums the slice's elements t, t + 256, ... in order; a warp
// shuffle tree and a fixed sum of the 8 warp totals finish each pass.
// (Welford's one-pass update with a Chan merge tree across the threads gives
// the same moments but puts a dependent FP64 division on every element and
// two on every tree level; on GB300's narrow FP64 pipe that chain was the
// kernel's whole latency: 12.3k cycles for 32 values and 45k for 4,096,
// against 4.8k and 11k for the two passes.)  With one slice out[dp] gets
// (n, m + (sum d) / n, M2); otherwise part[dp][slice] gets the mean as the
// unrounded pair (n, m, M2, (sum d) / n) for the slice merge.
template <typename T>
__global__ void __launch_bounds__(kStatsThreads) stats_kernel(const T* __restrict__ x, long long n_reps,
                                                              int slices, double* __restrict__ out) {
    __shared__ double gsum[kGroups], gsq[kGroups], gdev[kGroups];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long dp = blockIdx.x / slices;
    const long long sl = blockIdx.x - dp * slices;
    const long long per = (n_reps + slices - 1) / slices;
    const long long lo = sl * per;
    const long long hi = lo + per < n_reps ? lo + per : n_reps;
    const long long n = hi > lo ? hi - lo : 0;
    const double inv_n = n > 0 ? 1.0 / static_cast<double>(n) : 0.0;
    const T* row = x + dp * n_reps;
    if (!MRIP_CHECK(lo >= 0 && hi <= n_reps, 701, sl)) return;  // CTA-uniform
    double a = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kStatsThreads) a += static_cast<double>(row[i]);
    a = warp_sum(a);
    if (lane == 0) gsum[warp] = a;
    __syncthreads();
    const double mean = n > 0 ? total8(gsum) / static_cast<double>(n) : 0.0;
    double q = 0.0, c = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kStatsThreads) {
        const double d = static_cast<double>(row[i]) - mean;
        q += d * d;
        c += d;
    }
    q = warp_sum(q);
    c = warp_sum(c);
    if (lane == 0) {
        gsq[warp] = q;
        gdev[warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double sd = total8(gdev);
        double m2 = total8(gsq) - sd * sd * inv_n;
        if (m2 < 0.0) m2 = 0.0;
        if (slices == 1) {
            double* o = out + 3 * blockIdx.x;
            o[0] = static_cast<double>(n);
            o[1] = mean + sd * inv_n;
            o[2] = m2;
        } else {
            double* o = out + 4 * blockIdx.x;
            o[0] = static_cast<double>(n);
            o[1] = mean;
            o[2] = m2;
            o[3] = sd * inv_n;
        }
    }
}

// Slices of one design point merged in slice order by Chan's formula, the
// running mean kept as an unevaluated pair hi + lo (Knuth's two-sum) so that
// the difference of two slice means keeps the bits their rounding to one
// double would lose.
__global__ void stats_merge_kernel(const double* __restrict__ part, int n_dp, int slices,
                                   double* __restrict__ out) {
    const int dp = blockIdx.x * blockDim.x + threadIdx.x;
    if (dp >= n_dp) return;
    const double* p = part + static_cast<long long>(dp) * slices * 4;
    double n = p[0], mh = p[1], m2 = p[2], ml = p[3];
    for (int s = 1; s < slices; ++s) {
        const double nb = p[4 * s], bh = p[4 * s + 1], m2b = p[4 * s + 2], bl = p[4 * s + 3];
        if (nb == 0.0) continue;
        if (n == 0.0) {
            n = nb;
            mh = bh;
            m2 = m2b;
            ml = bl;
            continue;
        }
        const double nn = n + nb;
        const double delta = (bh - mh) + (bl - ml);
        const double t = ml + delta * (nb / nn);
        const double sh = mh + t;  // two-sum of mh and t
        const double v = sh - mh;
        const double sl = (mh - (sh - v)) + (t - v);
        m2 = m2 + m2b + delta * delta * (n * nb / nn);
        mh = sh;
        ml = sl;
        n = nn;
    }
    out[3 * dp] = n;
    out[3 * dp + 1] = mh + ml;
    out[3 * dp + 2] = m2;
}

// ---------------------------------------------------------------------------
// Host double-double arithmetic (Dekker / Knuth error-free transformations)
// ---------------------------------------------------------------------------
struct DD {
    double hi, lo;
};
inline DD dd(double x) { return DD{x, 0.0}; }
inline DD two_sum(double a, double b) {
    const double s = a + b;
    const double v = s - a;
    return DD{s, (a - (s - v)) + (b - v)};
}
inline DD renorm(double hi, double lo) {
    const double s = hi + lo;
    return DD{s, lo - (s - hi)};
}
inline DD add(DD a, DD b) {
    DD s = two_sum(a.hi, b.hi);
    return renorm(s.hi, s.lo + a.lo + b.lo);
}
inline DD mul(DD a, DD b) {
    const double p = a.hi * b.hi;
    const double e = std::fma(a.hi, b.hi, -p);
    return renorm(p, e + (a.hi * b.lo + a.lo * b.hi));
}
inline DD quot(DD a, DD b) {
    const double q1 = a.hi / b.hi;
    const DD r = add(a, mul(b, dd(-q1)));
    const double q2 = r.hi / b.hi;
    return renorm(q1, q2);
}

// P(|T| <= t), t >= 0, nu >= 1 integer.
DD two_sided(double t, long long nu) {
    const double fnu = static_cast<double>(nu);
    const DD t2 = mul(dd(t), dd(t));
    const DD c2 = quot(dd(fnu), add(dd(fnu), t2));  // cos^2(theta)
    const double s = t / std::sqrt(fnu + t * t);    // sin(theta)
    const double theta = std::atan2(t, std::sqrt(fnu));
    if (nu % 2 == 1) {
        DD inner = dd(1.0);
        for (long long k = (nu - 3) / 2; k >= 1; --k) {
            const DD r = quot(dd(2.0 * k), dd(2.0 * k + 1.0));
            inner = add(dd(1.0), mul(mul(r, c2), inner));
        }
        DD series = dd(0.0);
        if (nu >= 3) series = mul(dd(std::sqrt(c2.hi + c2.lo)), inner);
        const DD body = add(dd(theta), mul(dd(s), series));
        return mul(body, quot(dd(2.0), dd(M_PI)));
    }
    DD inner = dd(1.0);
    for (long long k = (nu - 2) / 2; k >= 1; --k) {
        const DD r = quot(dd(2.0 * k - 1.0), dd(2.0 * k));
        inner = add(dd(1.0), mul(mul(r, c2), inner));
    }
    return mul(dd(s), inner);
}

// P(T > t) for t >= 0.
double upper_tail(double t, long long nu) {
    const DD a = two_sided(t, nu);
    const DD one_minus = add(dd(1.0), DD{-a.hi, -a.lo});
    return 0.5 * (one_minus.hi + one_minus.lo);
}

double density(double t, long long nu) {
    const double fnu = static_cast<double>(nu);
    const double lg = std::lgamma(0.5 * (fnu + 1.0)) - std::lgamma(0.5 * fnu) -
                      0.5 * std::log(fnu * M_PI) - 0.5 * (fnu + 1.0) * std::log1p(t * t / fnu);
    return std::exp(lg);
}

}  // namespace

double t_critical_uncached(double conf, long long df) {
    const double tail = (1.0 - conf) / 2.0;
    double lo = 0.0, hi = 1.0;
    while (upper_tail(hi, df) > tail) {
        lo = hi;
        hi *= 2.0;
    }
    double t = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double g = upper_tail(t, df) - tail;  // decreasing in t
        if (g > 0.0)
            lo = t;
        else
            hi = t;
        double next = t + g / density(t, df);
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        if (next == t || hi - lo <= 0.0) break;
        if (std::fabs(next - t) <= 0x1p-60 * t) {
            t = next;
            break;
        }
        t = next;
    }
    return t;
}

// The series has about df/2 terms per evaluation and the solve takes a few
// dozen evaluations, so large df cost milliseconds; repeated runs of one
// experiment ask for the same (conf, df), so results are kept (bounded).
double t_critical(double conf, long long df) {
    static std::mutex mu;
    static std::map<std::pair<double, long long>, double> cache;
    const std::pair<double, long long> key(conf, df);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const double t = t_critical_uncached(conf, df);
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() >= 4096) cache.clear();
    cache.emplace(key, t);
    return t;
}

// Replications per slice: few design points with many replications would
// otherwise run on a few SMs (GB300's FP64 pipe is narrow: each value costs
// two loads and three FP64 operations).
constexpr long long kStatsSlice = 4096;

int stats_slices(int32_t n_dp, int64_t n_reps) {
    long long s = (n_reps + kStatsSlice - 1) / kStatsSlice;
    if (s < 1) s = 1;
    if (s > 256) s = 256;
    if (static_cast<long long>(n_dp) * s > 0x7FFFFFFFll) s = 1;
    return static_cast<int>(s);
}

size_t stats_scratch_bytes(int32_t n_dp, int64_t n_reps) {
    const int s = stats_slices(n_dp, n_reps);
    return s > 1 ? static_cast<size_t>(n_dp) * s * 4 * sizeof(double) : 0;
}

template <typename T>
mrip_status stats_reduce_t(const T* d_x, int32_t n_dp, int64_t n_reps, double* d_out, double* d_part,
                           cudaStream_t st) {
    if (n_dp == 0) return MRIP_OK;
    const int slices = stats_slices(n_dp, n_reps);
    if (slices == 1) {
        stats_kernel<T><<<n_dp, kStatsThreads, 0, st>>>(d_x, n_reps, 1, d_out);
        return launch_status("stats reduce");
    }
    if (!d_part) return fail(MRIP_ENOMEM, "stats reduce: no partials buffer");
    stats_kernel<T><<<static_cast<unsigned>(static_cast<long long>(n_dp) * slices), kStatsThreads, 0, st>>>(
        d_x, n_reps, slices, d_part);
    stats_merge_kernel<<<(n_dp + 127) / 128, 128, 0, st>>>(d_part, n_dp, slices, d_out);
    return launch_status("stats reduce");
}

mrip_status stats_reduce_double(const double* d_x, int32_t n_dp, int64_t n_reps, double* d_out,
                                cudaStream_t st, double* d_part) {
    return stats_reduce_t<double>(d_x, n_dp, n_reps, d_out, d_part, st);
}

mrip_status stats_reduce_int64(const int64_t* d_x, int32_t n_dp, int64_t n_reps, double* d_out,
                               cudaStream_t st, double* d_part) {
    return stats_reduce_t<long long>(reinterpret_cast<const long long*>(d_x), n_dp, n_reps, d_out, d_part,
                                     st);
}

void finalize_one(double n, double mean, double m2, double conf, mrip_stat* out) {
    out->n = static_cast<int64_t>(n);
    out->mean = mean;
    if (n < 2.0) {
        out->var = NAN;
        out->half_width = NAN;
        out->t_crit = NAN;
        return;
    }
    out->var = m2 / (n - 1.0);
    out->t_crit = t_critical(conf, static_cast<long long>(n) - 1);
    out->half_width = out->t_crit * std::sqrt(out->var / n);
}

}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_stats_reduce(const double* d_x, int32_t n_dp, int64_t n_reps,
                                         double* d_out, void* stream) {
    if (n_dp < 0 || n_reps < 0) return fail(MRIP_EINVAL, "mrip_stats_reduce: negative size");
    if (n_dp > 0 && (!d_out || (n_reps > 0 && !d_x))) return fail(MRIP_EINVAL, "mrip_stats_reduce: null pointer");
    const size_t need = stats_scratch_bytes(n_dp, n_reps);
    double* part = need ? static_cast<double*>(scratch(need, 3)) : nullptr;
    if (need && !part) return fail(MRIP_ENOMEM, "mrip_stats_reduce: scratch allocation failed");
    return stats_reduce_double(d_x, n_dp, n_reps, d_out, static_cast<cudaStream_t>(stream), part);
}

extern "C" mrip_status mrip_stats_reduce_i64(const int64_t* d_x, int32_t n_dp, int64_t n_reps,
                                             double* d_out, void* stream) {
    if (n_dp < 0 || n_reps < 0) return fail(MRIP_EINVAL, "mrip_stats_reduce_i64: negative size");
    if (n_dp > 0 && (!d_out || (n_reps > 0 && !d_x))) return fail(MRIP_EINVAL, "mrip_stats_reduce_i64: null pointer");
    const size_t need = stats_scratch_bytes(n_dp, n_reps);
    double* part = need ? static_cast<double*>(scratch(need, 3)) : nullptr;
    if (need && !part) return fail(MRIP_ENOMEM, "mrip_stats_reduce_i64: scratch allocation failed");
    return stats_reduce_int64(d_x, n_dp, n_reps, d_out, static_cast<cudaStream_t>(stream), part);
}

extern "C" mrip_status mrip_stats_finalize(const double* nmm2, int32_t n_dp, double conf,
                                           mrip_stat* out) {
    if (n_dp < 0 || (n_dp > 0 && (!nmm2 || !out)))
        return fail(MRIP_EINVAL, "mrip_stats_finalize: bad arguments");
    if (!(conf > 0.0 && conf < 1.0)) return fail(MRIP_EINVAL, "mrip_stats_finalize: conf in (0, 1)");
    // every design point of a run shares n: compute t once per distinct n
    double last_n = -1.0, last_t = NAN;
    for (int32_t i = 0; i < n_dp; ++i) {
        const double n = nmm2[3 * i];
        if (n >= 2.0 && n == last_n) {
            out[i].n = static_cast<int64_t>(n);
            out[i].mean = nmm2[3 * i + 1];
            out[i].var = nmm2[3 * i + 2] / (n - 1.0);
            out[i].t_crit = last_t;
            out[i].half_width = last_t * std::sqrt(out[i].var / n);
            continue;
        }
        finalize_one(n, nmm2[3 * i + 1], nmm2[3 * i + 2], conf, &out[i]);
        last_n = n;
        last_t = out[i].t_crit;
    }
    return MRIP_OK;
}

extern "C" mrip_status mrip_t_crit(double conf, int64_t df, double* out) {
    if (!out) return fail(MRIP_EINVAL, "mrip_t_crit: null output");
    if (!(conf > 0.0 && conf < 1.0) || df < 1) return fail(MRIP_EINVAL, "mrip_t_crit: conf in (0,1), df >= 1");
    *out = t_critical(conf, df);
    return MRIP_OK;
}

extern "C" mrip_status mrip_stats_merge(const double* parts, int32_t n_parts, int32_t n_dp, double* out) {
    if (n_parts < 1 || n_dp < 0 || (n_dp > 0 && (!parts || !out)))
        return fail(MRIP_EINVAL, "mrip_stats_merge: need n_parts >= 1, n_dp >= 0 and buffers");
    for (int32_t d = 0; d < n_dp; ++d) {
        double n = 0.0, mean = 0.0, m2 = 0.0;
        for (int32_t p = 0; p < n_parts; ++p) {
            const double* t = parts + (static_cast<size_t>(p) * n_dp + d) * 3;
            const double nb = t[0];
            if (!(nb >= 0.0)) return fail(MRIP_EINVAL, "mrip_stats_merge: negative count");
            if (nb == 0.0) continue;
            if (n == 0.0) {
                n = nb;
                mean = t[1];
                m2 = t[2];
                continue;
            }
            const double tot = n + nb;
            const double delta = t[1] - mean;
            mean = mean + delta * (nb / tot);
            m2 = m2 + t[2] + delta * delta * (n * nb / tot);
            n = tot;
        }
        out[3 * d] = n;
        out[3 * d + 1] = mean;
        out[3 * d + 2] = m2;
    }
    return MRIP_OK;
}

MRIP_DEBUG_UNIT(stats)
