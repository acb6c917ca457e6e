// Per-design-point statistics of the replication outputs (paper, Section 1:
// the replication mean and a CLT confidence interval) and the Student-t
// critical value.
//
// Device: one CTA per design point and slice of at most 4,096 replications.
// Thread t runs Welford's update over the slice's replications t, t + B, ...;
// the CTA merges the (n, mean, M2) triples pairwise in a fixed tree (Chan,
// Golub, LeVeque 1979) and a second kernel merges the slices in order, so
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

__device__ __forceinline__ void chan_merge(double& na, double& ma, double& m2a, double nb, double mb,
                                           double m2b) {
    const double n = na + nb;
    if (nb == 0.0) return;
    if (na == 0.0) {
        na = nb;
        ma = mb;
        m2a = m2b;
        return;
    }
    const double delta = mb - ma;
    ma = ma + delta * (nb / n);
    m2a = m2a + m2b + delta * delta * (na * nb / n);
    na = n;
}

// One CTA per (design point, slice of replications): Welford per thread over
// the slice, then the CTA's fixed merge tree.  With one slice the triple goes
// straight to out[dp]; otherwise to part[dp][slice].
template <typename T>
__global__ void __launch_bounds__(kStatsThreads) stats_kernel(const T* __restrict__ x, long long n_reps,
                                                              int slices, double* __restrict__ out) {
    __shared__ double sn[kStatsThreads], sm[kStatsThreads], s2[kStatsThreads];
    const long long dp = blockIdx.x / slices;
    const long long sl = blockIdx.x - dp * slices;
    const long long per = (n_reps + slices - 1) / slices;
    const long long lo = sl * per;
    const long long hi = lo + per < n_reps ? lo + per : n_reps;
    const T* row = x + dp * n_reps;
    double n = 0.0, mean = 0.0, m2 = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kStatsThreads) {
        const double v = static_cast<double>(row[i]);
        n += 1.0;
        const double d = v - mean;
        mean += d / n;
        m2 += d * (v - mean);
    }
    sn[threadIdx.x] = n;
    sm[threadIdx.x] = mean;
    s2[threadIdx.x] = m2;
    __syncthreads();
    for (int stride = kStatsThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            double a = sn[threadIdx.x], b = sm[threadIdx.x], c = s2[threadIdx.x];
            chan_merge(a, b, c, sn[threadIdx.x + stride], sm[threadIdx.x + stride],
                       s2[threadIdx.x + stride]);
            sn[threadIdx.x] = a;
            sm[threadIdx.x] = b;
            s2[threadIdx.x] = c;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = out + 3 * blockIdx.x;
        o[0] = sn[0];
        o[1] = sm[0];
        o[2] = s2[0];
    }
}

// Slices of one design point merged in slice order.
__global__ void stats_merge_kernel(const double* __restrict__ part, int n_dp, int slices,
                                   double* __restrict__ out) {
    const int dp = blockIdx.x * blockDim.x + threadIdx.x;
    if (dp >= n_dp) return;
    const double* p = part + static_cast<long long>(dp) * slices * 3;
    double n = p[0], mean = p[1], m2 = p[2];
    for (int s = 1; s < slices; ++s) chan_merge(n, mean, m2, p[3 * s], p[3 * s + 1], p[3 * s + 2]);
    out[3 * dp] = n;
    out[3 * dp + 1] = mean;
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
// otherwise run on a few SMs (the FP64 Welford update is ~14 FP64 operations
// per value on GB300's narrow FP64 pipe).
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
    return s > 1 ? static_cast<size_t>(n_dp) * s * 3 * sizeof(double) : 0;
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
    if (n_dp > 0 && (!d_x || !d_out)) return fail(MRIP_EINVAL, "mrip_stats_reduce: null pointer");
    const size_t need = stats_scratch_bytes(n_dp, n_reps);
    double* part = need ? static_cast<double*>(scratch(need, 3)) : nullptr;
    if (need && !part) return fail(MRIP_ENOMEM, "mrip_stats_reduce: scratch allocation failed");
    return stats_reduce_double(d_x, n_dp, n_reps, d_out, static_cast<cudaStream_t>(stream), part);
}

extern "C" mrip_status mrip_stats_reduce_i64(const int64_t* d_x, int32_t n_dp, int64_t n_reps,
                                             double* d_out, void* stream) {
    if (n_dp < 0 || n_reps < 0) return fail(MRIP_EINVAL, "mrip_stats_reduce_i64: negative size");
    if (n_dp > 0 && (!d_x || !d_out)) return fail(MRIP_EINVAL, "mrip_stats_reduce_i64: null pointer");
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
