// Queueing models of the MRIP engine: the M/M/1 queue of the paper
// (Section 5.1, second model) and a 3-station tandem of M/M/1 stations.
//
// Mappings (paper, Section 3):
//   THREAD      one replication per thread (TLP);
//   WARP_1LANE  one replication per warp, lane 0 works, 31 lanes idle (WLP);
//   WARP_COOP   one replication per warp, the clients split into 32
//               contiguous segments.  The Lindley step W -> max(0, W + S - A)
//               composes to maps W -> max(c, W + d); lanes compose their
//               segment's map, a warp scan of the maps gives each segment's
//               entry wait, and each lane then replays its segment with the
//               plain recurrence.  The tandem does the same with 3-station
//               max-plus maps (lower-triangular 3x3 matrix plus constants).
#include "common.cuh"

namespace mrip {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Times in 64-bit fixed point.  GB300 retires about two FP64 operations per
// SM-clock and over forty 32-bit integer multiplies, so the queue recurrences
// (additions, subtractions and maxima only) run on integers: a time t is held
// as round(t 2^48).  A variate is E / rate with E = y57 2^-57 from the
// fixed-point log, i.e. round(y57 * (2^-9 / rate)), the factor stored as a
// 64-bit multiplier cm = round(2^57 / rate) (2^-9 / rate = cm 2^-66).  A
// variate then carries the multiplier's relative error (2^-53, as an FP64
// division would) plus at most one unit (2^-48), and every recurrence step is
// exact, where FP64 rounds each addition; the outputs agree with
// FP64 evaluation far inside 1e-12 as long as the variates are not tiny
// against 2^-48: rates are limited to [2^-6, 2^4] (mean variate >= 1/16).
// A variate is then below 36.8 * 64 < 2^11.3 time units (E <= 53 ln 2);
// while the largest state stays below 2^12 (2^60 units) one more step stays
// below 2^61.5, so nothing overflows.  Design points with other rates run the
// FP64 recurrence, and a replication whose sojourn time reaches 2^12
// restarts in FP64.  Means of single variates (the early-window features)
// are summed in FP64 from the same log values, where a variate's relative
// precision matters.
// ---------------------------------------------------------------------------
constexpr int kFixBits = 48;
constexpr long long kFixGuard = 1LL << 60;
constexpr long long kFixNegInf = -(1LL << 62);  // "empty" state: v - A stays above -2^63

// 2^-9 / rate as cm 2^-66 (cm in [2^53, 2^63] for the rates above: at least
// 53 significant bits), so that round(y57 2^-9 / rate) = (hi(y57 cm) + 2) >> 2.
// hi comes from umul64hi_trunc, 0 to 2 units short, so 3 is added instead of
// 2: the variate is then within one unit (2^-48) of y57 2^-9 / rate.
__device__ __forceinline__ bool fix_rate_ok(double rate) { return rate >= 0x1p-6 && rate <= 0x1p4; }

__device__ __forceinline__ unsigned long long fix_scale(double rate) {
    return static_cast<unsigned long long>(0x1p57 / rate + 0.5);
}

__device__ __forceinline__ long long to_fix(unsigned long long y57, unsigned long long cm) {
    return static_cast<long long>((umul64hi_trunc(y57, cm) + 3u) >> 2);
}

struct U128 {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(long long v) {  // v >= 0
        const unsigned long long u = static_cast<unsigned long long>(v);
        lo += u;
        hi += (lo < u) ? 1u : 0u;
    }
    __device__ __forceinline__ double to_double() const {  // value 2^-48
        return static_cast<double>(hi) * 0x1p16 + static_cast<double>(lo) * 0x1p-48;
    }
};

constexpr long long kSat = 1LL << 61;

__device__ __forceinline__ long long sat61(long long x) { return x > kSat ? kSat : (x < -kSat ? -kSat : x); }

__device__ __forceinline__ U128 shfl_down_u128(const U128& x, int off) {
    U128 r;
    r.lo = __shfl_down_sync(kFull, x.lo, off);
    r.hi = __shfl_down_sync(kFull, x.hi, off);
    return r;
}
__device__ __forceinline__ void add_u128(U128& a, const U128& b) {
    a.lo += b.lo;
    a.hi += b.hi + ((a.lo < b.lo) ? 1u : 0u);
}

__device__ __forceinline__ unsigned long long word_k(uint32_t lo, uint32_t hi) {
    const unsigned long long bits = (static_cast<unsigned long long>(hi) << 32) | lo;
    return (1ULL << 53) - (bits >> 11);
}

struct Mm1Out {
    double* wait;
    double* idle;
    double* system;
};

// Client n of (dp, rep): service S_n from words (0,1), gap A_{n+1} from (2,3).
// inv_mu, inv_lam are 2^-57 / rate (see expo_fast).
__device__ __forceinline__ void mm1_client(uint32_t n, uint32_t rep, uint32_t dp, double inv_lam,
                                           double inv_mu, const RoundKeys& rk, const LogTable& tab,
                                           double& s, double& a) {
    const uint4 b = philox(0u, n, rep, stream_word(0u, dp), rk);
    s = expo_fast(b.x, b.y, tab, inv_mu);
    a = expo_fast(b.z, b.w, tab, inv_lam);
}

// (A minimum of four CTAs per SM rather than eight: the same 64 registers,
// but 0.80 instead of 0.83 ms for 2^16 replications of 1,000 clients.)
template <bool kLane0Only>
__global__ void __launch_bounds__(128, 4) mm1_serial_kernel(const double* __restrict__ dps, long long n_items,
                                  long long n_reps, long long rep0, long long n_clients,
                                  const __grid_constant__ RoundKeys rk, LogTable tab, Mm1Out out) {
    long long item;
    if (kLane0Only) {
        if ((threadIdx.x & 31) != 0) return;
        item = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    } else {
        item = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    }
    if (item >= n_items) return;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double lam = dps[2 * dp], mu = dps[2 * dp + 1];
    const double inv = static_cast<double>(n_clients);
    if (fix_rate_ok(lam) && fix_rate_ok(mu)) {  // 48-bit fixed-point times
        const unsigned long long cl = fix_scale(lam), cmu = fix_scale(mu);
        const uint32_t c3 = stream_word(0u, dp);
        long long wf = 0;
        U128 sw, si, sv;
        bool overflow = false;
        for (long long n = 0; n < n_clients; ++n) {
            const uint4 b = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
            const long long s_ = to_fix(neg_log_q57(word_k(b.x, b.y), tab), cmu);
            const long long a_ = to_fix(neg_log_q57(word_k(b.z, b.w), tab), cl);
            sw.add(wf);
            const long long v = wf + s_;
            sv.add(v);
            const long long t = v - a_;
            si.add(t < 0 ? -t : 0);
            wf = t > 0 ? t : 0;
            if (wf >= kFixGuard) {
                overflow = true;
                break;
            }
        }
        if (!overflow) {
            if (out.wait) out.wait[item] = sw.to_double() / inv;
            if (out.idle) out.idle[item] = si.to_double() / inv;
            if (out.system) out.system[item] = sv.to_double() / inv;
            return;
        }
    }
    const double inv_lam = 0x1p-57 / lam, inv_mu = 0x1p-57 / mu;
    double w = 0.0, sum_w = 0.0, sum_i = 0.0, sum_v = 0.0;
    for (long long n = 0; n < n_clients; ++n) {
        double s, a;
        mm1_client(static_cast<uint32_t>(n), rep, dp, inv_lam, inv_mu, rk, tab, s, a);
        sum_w += w;
        const double v = w + s;
        sum_v += v;
        const double t = v - a;
        sum_i += (t < 0.0) ? -t : 0.0;
        w = (t > 0.0) ? t : 0.0;
    }
    if (out.wait) out.wait[item] = sum_w / inv;
    if (out.idle) out.idle[item] = sum_i / inv;
    if (out.system) out.system[item] = sum_v / inv;
}

// Max-plus map W -> max(c, W + d).  compose(first, then).
struct MaxPlus {
    double c, d;
};
__device__ __forceinline__ MaxPlus compose(MaxPlus f, MaxPlus g) {
    // g(f(W)) = max(g.c, max(f.c, W + f.d) + g.d) = max(max(g.c, f.c + g.d), W + (f.d + g.d))
    MaxPlus r;
    const double cc = f.c + g.d;
    r.c = (g.c > cc) ? g.c : cc;
    r.d = f.d + g.d;
    return r;
}

// One warp per replication; clients staged in shared memory when kStage.
template <bool kStage>
__global__ void mm1_warp_coop_kernel(const double* __restrict__ dps, long long n_items,
                                     long long n_reps, long long rep0, long long n_clients,
                                     const __grid_constant__ RoundKeys rk, LogTable tab, Mm1Out out) {
    extern __shared__ double stage[];  // per warp: S[seg_cap*32], A[seg_cap*32]
    const int lane = threadIdx.x & 31;
    const int warp_in_cta = threadIdx.x >> 5;
    const long long item = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    if (item >= n_items) return;  // warp-uniform
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double inv_lam = 0x1p-57 / dps[2 * dp], inv_mu = 0x1p-57 / dps[2 * dp + 1];
    const long long seg = (n_clients + 31) / 32;
    const long long lo = lane * seg;
    const long long hi = (lo + seg < n_clients) ? lo + seg : n_clients;
    double* s_buf = stage + static_cast<size_t>(warp_in_cta) * 2 * seg * 32;
    double* a_buf = s_buf + seg * 32;
    // staged only where the warp's slice fits the launch's shared memory
    // (always, unless the host sized it wrong: then the debug build records
    // it and the variates are recomputed instead)
    const bool staged =
        kStage && MRIP_CHECK((warp_in_cta + 1ull) * 2 * seg * 32 * sizeof(double) <= dynamic_smem_bytes(), 201, seg);

    // pass 1: the segment's composed map
    MaxPlus f{-INFINITY, 0.0};
    for (long long n = lo; n < hi; ++n) {
        double s, a;
        mm1_client(static_cast<uint32_t>(n), rep, dp, inv_lam, inv_mu, rk, tab, s, a);
        if (staged) {
            s_buf[(n - lo) * 32 + lane] = s;
            a_buf[(n - lo) * 32 + lane] = a;
        }
        MaxPlus step{0.0, s - a};
        f = compose(f, step);
    }
    // inclusive scan of maps over lanes (earlier lanes first), then shift
    MaxPlus acc = f;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        MaxPlus prev;
        prev.c = __shfl_up_sync(kFull, acc.c, off);
        prev.d = __shfl_up_sync(kFull, acc.d, off);
        if (lane >= off) acc = compose(prev, acc);
    }
    MaxPlus excl;
    excl.c = __shfl_up_sync(kFull, acc.c, 1);
    excl.d = __shfl_up_sync(kFull, acc.d, 1);
    double w = 0.0;
    if (lane > 0) w = (excl.c > excl.d) ? excl.c : excl.d;  // entry wait = map(0)

    // pass 2: replay the segment with the plain recurrence
    double sum_w = 0.0, sum_i = 0.0, sum_v = 0.0;
    for (long long n = lo; n < hi; ++n) {
        double s, a;
        if (staged) {
            s = s_buf[(n - lo) * 32 + lane];
            a = a_buf[(n - lo) * 32 + lane];
        } else {
            mm1_client(static_cast<uint32_t>(n), rep, dp, inv_lam, inv_mu, rk, tab, s, a);
        }
        sum_w += w;
        const double v = w + s;
        sum_v += v;
        const double t = v - a;
        sum_i += (t < 0.0) ? -t : 0.0;
        w = (t > 0.0) ? t : 0.0;
    }
    // fixed-order (lane-ordered tree) reduction of the three sums
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double ow = __shfl_down_sync(kFull, sum_w, off);
        const double oi = __shfl_down_sync(kFull, sum_i, off);
        const double ov = __shfl_down_sync(kFull, sum_v, off);
        if ((lane & (2 * off - 1)) == 0) {
            sum_w += ow;
            sum_i += oi;
            sum_v += ov;
        }
    }
    if (lane == 0) {
        const double inv = static_cast<double>(n_clients);
        if (out.wait) out.wait[item] = sum_w / inv;
        if (out.idle) out.idle[item] = sum_i / inv;
        if (out.system) out.system[item] = sum_v / inv;
    }
}

// ---------------------------------------------------------------------------
// Tandem: V_{n,j} = max(V_{n-1,j} - A_n, V_{n,j-1}) + S_{n,j}
// ---------------------------------------------------------------------------
struct TandemOut {
    double* y;
    double* feat;     // 8 planes of n_items (may be null)
    long long plane;  // plane stride = n_items
};

template <bool kLane0Only>
__global__ void __launch_bounds__(128, 8) tandem3_serial_kernel(const double* __restrict__ dps, long long n_items,
                                      long long n_reps, long long rep0, long long n_clients,
                                      long long window, uint32_t tag,
                                      const __grid_constant__ RoundKeys rk, LogTable tab,
                                      TandemOut out) {
    long long item;
    if (kLane0Only) {
        if ((threadIdx.x & 31) != 0) return;
        item = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    } else {
        item = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    }
    if (item >= n_items) return;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double lam = dps[4 * dp], mu1 = dps[4 * dp + 1], mu2 = dps[4 * dp + 2],
                 mu3 = dps[4 * dp + 3];
    const double i_lam = 0x1p-57 / lam, i_mu1 = 0x1p-57 / mu1, i_mu2 = 0x1p-57 / mu2,
                 i_mu3 = 0x1p-57 / mu3;
    const uint32_t c3 = stream_word(tag, dp);
    const long long w_len = (n_clients < window) ? n_clients : window;
    double sum_y = 0.0, sum_a = 0.0, sum_1 = 0.0, sum_2 = 0.0, sum_3 = 0.0;
    bool fixed_done = false;
    if (fix_rate_ok(lam) && fix_rate_ok(mu1) && fix_rate_ok(mu2) && fix_rate_ok(mu3)) {
        const unsigned long long fl = fix_scale(lam), f1 = fix_scale(mu1), f2 = fix_scale(mu2),
                                 f3 = fix_scale(mu3);
        long long v1 = kFixNegInf, v2 = kFixNegInf, v3 = kFixNegInf;
        U128 sy;
        double wa = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        bool overflow = false;
        // client n's four log values; then one step of the recurrence
        auto logs = [&](uint32_t n, unsigned long long& ya, unsigned long long& y1, unsigned long long& y2,
                        unsigned long long& y3) {
            const uint4 b0 = philox(0u, n, rep, c3, rk);
            const uint4 b1 = philox(1u, n, rep, c3, rk);
            ya = neg_log_q57(word_k(b0.x, b0.y), tab);
            y1 = neg_log_q57(word_k(b0.z, b0.w), tab);
            y2 = neg_log_q57(word_k(b1.x, b1.y), tab);
            y3 = neg_log_q57(word_k(b1.z, b1.w), tab);
        };
        auto step = [&](unsigned long long ya, unsigned long long y1, unsigned long long y2,
                        unsigned long long y3) {
            const long long a = to_fix(ya, fl);
            long long q = v1 - a;
            v1 = ((q > 0) ? q : 0) + to_fix(y1, f1);
            q = v2 - a;
            v2 = ((q > v1) ? q : v1) + to_fix(y2, f2);
            q = v3 - a;
            v3 = ((q > v2) ? q : v2) + to_fix(y3, f3);
            sy.add(v3);
            return v3 < kFixGuard;
        };
        // the early window also sums the same variates as doubles (expo_fast);
        // the loop after it carries none of that state.  Client indices are
        // 32-bit (n_clients < 2^32, the counter word c1).
        const uint32_t nc = static_cast<uint32_t>(n_clients), nw = static_cast<uint32_t>(w_len);
        uint32_t n = 0;
        for (; n < nw; ++n) {
            unsigned long long ya, y1, y2, y3;
            logs(n, ya, y1, y2, y3);
            wa += __ull2double_rn(ya) * i_lam;
            w1 += __ull2double_rn(y1) * i_mu1;
            w2 += __ull2double_rn(y2) * i_mu2;
            w3 += __ull2double_rn(y3) * i_mu3;
            if (!step(ya, y1, y2, y3)) {
                overflow = true;
                break;
            }
        }
        for (; !overflow && n < nc; ++n) {
            unsigned long long ya, y1, y2, y3;
            logs(n, ya, y1, y2, y3);
            if (!step(ya, y1, y2, y3)) overflow = true;
        }
        if (!overflow) {
            fixed_done = true;
            sum_y = sy.to_double();
            sum_a = wa;
            sum_1 = w1;
            sum_2 = w2;
            sum_3 = w3;
        }
    }
    double v1 = -INFINITY, v2 = -INFINITY, v3 = -INFINITY;
    for (long long n = 0; !fixed_done && n < n_clients; ++n) {
        const uint4 b0 = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
        const uint4 b1 = philox(1u, static_cast<uint32_t>(n), rep, c3, rk);
        const double a = expo_fast(b0.x, b0.y, tab, i_lam);
        const double s1 = expo_fast(b0.z, b0.w, tab, i_mu1);
        const double s2 = expo_fast(b1.x, b1.y, tab, i_mu2);
        const double s3 = expo_fast(b1.z, b1.w, tab, i_mu3);
        double q = v1 - a;
        v1 = ((q > 0.0) ? q : 0.0) + s1;
        q = v2 - a;
        v2 = ((q > v1) ? q : v1) + s2;
        q = v3 - a;
        v3 = ((q > v2) ? q : v2) + s3;
        sum_y += v3;
        if (n < w_len) {
            sum_a += a;
            sum_1 += s1;
            sum_2 += s2;
            sum_3 += s3;
        }
    }
    out.y[item] = sum_y / static_cast<double>(n_clients);
    if (out.feat) {
        const double wl = static_cast<double>(w_len);
        double* f = out.feat + item;
        const long long p = out.plane;
        f[0] = lam;
        f[p] = mu1;
        f[2 * p] = mu2;
        f[3 * p] = mu3;
        f[4 * p] = sum_a / wl;
        f[5 * p] = sum_1 / wl;
        f[6 * p] = sum_2 / wl;
        f[7 * p] = sum_3 / wl;
    }
}

// Tandem, one warp per replication.  One client maps the arrival-relative
// state v = (v1, v2, v3) to v'_j = max(v_j - A, v'_{j-1}) + S_j (v'_0 = 0),
// a max-plus affine map with a lower-triangular matrix:
//   v'_j = max(c_j, max_{k <= j} (v_k + d_jk)).
// Maps compose (TMap below), so a warp scan over the lanes' segment maps gives
// each segment's entry state (the composed map applied to the empty state,
// i.e. its constant terms c); every lane then replays its segment with the
// plain recurrence, as the serial kernel does.
struct TMap {
    double c1, c2, c3, d11, d21, d22, d31, d32, d33;
};

__device__ __forceinline__ TMap tmap_identity() {
    return TMap{-INFINITY, -INFINITY, -INFINITY, 0.0, -INFINITY, 0.0, -INFINITY, -INFINITY, 0.0};
}

__device__ __forceinline__ double dmax(double x, double y) { return x > y ? x : y; }

// f followed by one client (a, s1, s2, s3)
__device__ __forceinline__ TMap tmap_push(const TMap& f, double a, double s1, double s2, double s3) {
    const double e1 = s1 - a, e2 = s2 - a, e3 = s3 - a;
    TMap r;
    r.c1 = dmax(s1, f.c1 + e1);
    r.d11 = f.d11 + e1;
    r.c2 = dmax(f.c2 + e2, r.c1 + s2);
    r.d21 = dmax(f.d21 + e2, r.d11 + s2);
    r.d22 = f.d22 + e2;
    r.c3 = dmax(f.c3 + e3, r.c2 + s3);
    r.d31 = dmax(f.d31 + e3, r.d21 + s3);
    r.d32 = dmax(f.d32 + e3, r.d22 + s3);
    r.d33 = f.d33 + e3;
    return r;
}

// g after f
__device__ __forceinline__ TMap tmap_compose(const TMap& f, const TMap& g) {
    TMap h;
    h.c1 = dmax(g.c1, f.c1 + g.d11);
    h.c2 = dmax(g.c2, dmax(f.c1 + g.d21, f.c2 + g.d22));
    h.c3 = dmax(g.c3, dmax(f.c1 + g.d31, dmax(f.c2 + g.d32, f.c3 + g.d33)));
    h.d11 = f.d11 + g.d11;
    h.d21 = dmax(f.d11 + g.d21, f.d21 + g.d22);
    h.d22 = f.d22 + g.d22;
    h.d31 = dmax(f.d11 + g.d31, dmax(f.d21 + g.d32, f.d31 + g.d33));
    h.d32 = dmax(f.d22 + g.d32, f.d32 + g.d33);
    h.d33 = f.d33 + g.d33;
    return h;
}

__device__ __forceinline__ TMap tmap_shfl_up(const TMap& m, int off) {
    TMap r;
    r.c1 = __shfl_up_sync(kFull, m.c1, off);
    r.c2 = __shfl_up_sync(kFull, m.c2, off);
    r.c3 = __shfl_up_sync(kFull, m.c3, off);
    r.d11 = __shfl_up_sync(kFull, m.d11, off);
    r.d21 = __shfl_up_sync(kFull, m.d21, off);
    r.d22 = __shfl_up_sync(kFull, m.d22, off);
    r.d31 = __shfl_up_sync(kFull, m.d31, off);
    r.d32 = __shfl_up_sync(kFull, m.d32, off);
    r.d33 = __shfl_up_sync(kFull, m.d33, off);
    return r;
}

struct TandemClient {
    double a, s1, s2, s3;
};

__device__ __forceinline__ TandemClient tandem_client(uint32_t n, uint32_t rep, uint32_t c3,
                                                      const RoundKeys& rk, const LogTable& tab,
                                                      double i_lam, double i_mu1, double i_mu2,
                                                      double i_mu3) {
    const uint4 b0 = philox(0u, n, rep, c3, rk);
    const uint4 b1 = philox(1u, n, rep, c3, rk);
    return TandemClient{expo_fast(b0.x, b0.y, tab, i_lam), expo_fast(b0.z, b0.w, tab, i_mu1),
                        expo_fast(b1.x, b1.y, tab, i_mu2), expo_fast(b1.z, b1.w, tab, i_mu3)};
}

// The same maps in 48-bit fixed point, every sum saturated at +-2^61 (the
// empty state's -inf is -2^61).  After one client every constant is positive,
// so a term pushed down to -2^61 never decides a maximum for states in
// [0, 2^60]; a state or constant past 2^60 sends the replication to FP64.
struct FTMap {
    long long c1, c2, c3, d11, d21, d22, d31, d32, d33;
};

__device__ __forceinline__ FTMap ftmap_identity() {
    return FTMap{-kSat, -kSat, -kSat, 0, -kSat, 0, -kSat, -kSat, 0};
}

__device__ __forceinline__ long long lmax(long long x, long long y) { return x > y ? x : y; }

__device__ __forceinline__ FTMap ftmap_push(const FTMap& f, long long a, long long s1, long long s2, long long s3) {
    const long long e1 = s1 - a, e2 = s2 - a, e3 = s3 - a;
    FTMap r;
    r.c1 = lmax(s1, sat61(f.c1 + e1));
    r.d11 = sat61(f.d11 + e1);
    r.c2 = sat61(lmax(f.c2 + e2, r.c1 + s2));
    r.d21 = sat61(lmax(f.d21 + e2, r.d11 + s2));
    r.d22 = sat61(f.d22 + e2);
    r.c3 = sat61(lmax(f.c3 + e3, r.c2 + s3));
    r.d31 = sat61(lmax(f.d31 + e3, r.d21 + s3));
    r.d32 = sat61(lmax(f.d32 + e3, r.d22 + s3));
    r.d33 = sat61(f.d33 + e3);
    return r;
}

__device__ __forceinline__ FTMap ftmap_compose(const FTMap& f, const FTMap& g) {  // g after f
    FTMap h;
    h.c1 = lmax(g.c1, sat61(f.c1 + g.d11));
    h.c2 = lmax(g.c2, sat61(lmax(f.c1 + g.d21, f.c2 + g.d22)));
    h.c3 = lmax(g.c3, sat61(lmax(f.c1 + g.d31, lmax(f.c2 + g.d32, f.c3 + g.d33))));
    h.d11 = sat61(f.d11 + g.d11);
    h.d21 = sat61(lmax(f.d11 + g.d21, f.d21 + g.d22));
    h.d22 = sat61(f.d22 + g.d22);
    h.d31 = sat61(lmax(f.d11 + g.d31, lmax(f.d21 + g.d32, f.d31 + g.d33)));
    h.d32 = sat61(lmax(f.d22 + g.d32, f.d32 + g.d33));
    h.d33 = sat61(f.d33 + g.d33);
    return h;
}

__device__ __forceinline__ FTMap ftmap_shfl_up(const FTMap& m, int off) {
    FTMap r;
    r.c1 = __shfl_up_sync(kFull, m.c1, off);
    r.c2 = __shfl_up_sync(kFull, m.c2, off);
    r.c3 = __shfl_up_sync(kFull, m.c3, off);
    r.d11 = __shfl_up_sync(kFull, m.d11, off);
    r.d21 = __shfl_up_sync(kFull, m.d21, off);
    r.d22 = __shfl_up_sync(kFull, m.d22, off);
    r.d31 = __shfl_up_sync(kFull, m.d31, off);
    r.d32 = __shfl_up_sync(kFull, m.d32, off);
    r.d33 = __shfl_up_sync(kFull, m.d33, off);
    return r;
}

// FP64 warp scan of one replication (the fallback of the fixed-point paths):
// lane l takes the l-th of 32 contiguous client segments.
__device__ void tandem_coop_fp64(long long item, uint32_t dp, uint32_t rep, double lam, double mu1, double mu2,
                                 double mu3, long long n_clients, long long window, uint32_t c3,
                                 const RoundKeys& rk, const LogTable& tab, const TandemOut& out) {
    (void)dp;
    const int lane = threadIdx.x & 31;
    const double i_lam = 0x1p-57 / lam, i_mu1 = 0x1p-57 / mu1, i_mu2 = 0x1p-57 / mu2, i_mu3 = 0x1p-57 / mu3;
    const long long w_len = (n_clients < window) ? n_clients : window;
    const long long seg = (n_clients + 31) / 32;
    const long long lo = min(lane * seg, n_clients);
    const long long hi = min(lo + seg, n_clients);
    // pass 1: this segment's map
    TMap f = tmap_identity();
    for (long long n = lo; n < hi; ++n) {
        const TandemClient k = tandem_client(static_cast<uint32_t>(n), rep, c3, rk, tab, i_lam, i_mu1, i_mu2, i_mu3);
        f = tmap_push(f, k.a, k.s1, k.s2, k.s3);
    }
    // inclusive scan over lanes, then the previous lane's prefix is the entry map
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const TMap prev = tmap_shfl_up(f, off);
        if (lane >= off) f = tmap_compose(prev, f);
    }
    const TMap excl = tmap_shfl_up(f, 1);
    double v1 = -INFINITY, v2 = -INFINITY, v3 = -INFINITY;
    if (lane > 0) {
        v1 = excl.c1;
        v2 = excl.c2;
        v3 = excl.c3;
    }

    // pass 2: replay the segment with the plain recurrence
    double sum_y = 0.0, sum_a = 0.0, sum_1 = 0.0, sum_2 = 0.0, sum_3 = 0.0;
    for (long long n = lo; n < hi; ++n) {
        const TandemClient k = tandem_client(static_cast<uint32_t>(n), rep, c3, rk, tab, i_lam, i_mu1, i_mu2, i_mu3);
        double q = v1 - k.a;
        v1 = ((q > 0.0) ? q : 0.0) + k.s1;
        q = v2 - k.a;
        v2 = ((q > v1) ? q : v1) + k.s2;
        q = v3 - k.a;
        v3 = ((q > v2) ? q : v2) + k.s3;
        sum_y += v3;
        if (n < w_len) {
            sum_a += k.a;
            sum_1 += k.s1;
            sum_2 += k.s2;
            sum_3 += k.s3;
        }
    }
    // fixed-order (lane-ordered tree) reduction
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double oy = __shfl_down_sync(kFull, sum_y, off);
        const double oa = __shfl_down_sync(kFull, sum_a, off);
        const double o1 = __shfl_down_sync(kFull, sum_1, off);
        const double o2 = __shfl_down_sync(kFull, sum_2, off);
        const double o3 = __shfl_down_sync(kFull, sum_3, off);
        if ((lane & (2 * off - 1)) == 0) {
            sum_y += oy;
            sum_a += oa;
            sum_1 += o1;
            sum_2 += o2;
            sum_3 += o3;
        }
    }
    if (lane != 0) return;
    out.y[item] = sum_y / static_cast<double>(n_clients);
    if (out.feat) {
        const double wl = static_cast<double>(w_len);
        double* fo = out.feat + item;
        const long long p = out.plane;
        fo[0] = lam;
        fo[p] = mu1;
        fo[2 * p] = mu2;
        fo[3 * p] = mu3;
        fo[4 * p] = sum_a / wl;
        fo[5 * p] = sum_1 / wl;
        fo[6 * p] = sum_2 / wl;
        fo[7 * p] = sum_3 / wl;
    }
}

__global__ void __launch_bounds__(128) tandem3_warp_coop_kernel(
    const double* __restrict__ dps, long long n_items, long long n_reps, long long rep0,
    long long n_clients, long long window, uint32_t tag, const __grid_constant__ RoundKeys rk,
    LogTable tab, TandemOut out) {
    const int lane = threadIdx.x & 31;
    const long long item = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    if (item >= n_items) return;  // warp-uniform
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double lam = dps[4 * dp], mu1 = dps[4 * dp + 1], mu2 = dps[4 * dp + 2], mu3 = dps[4 * dp + 3];
    const double i_lam = 0x1p-57 / lam, i_mu1 = 0x1p-57 / mu1, i_mu2 = 0x1p-57 / mu2,
                 i_mu3 = 0x1p-57 / mu3;
    const uint32_t c3 = stream_word(tag, dp);
    const long long w_len = (n_clients < window) ? n_clients : window;
    const long long seg = (n_clients + 31) / 32;
    const long long lo = min(lane * seg, n_clients);
    const long long hi = min(lo + seg, n_clients);

    if (fix_rate_ok(lam) && fix_rate_ok(mu1) && fix_rate_ok(mu2) && fix_rate_ok(mu3)) {
        const unsigned long long cl = fix_scale(lam), c1 = fix_scale(mu1), c2 = fix_scale(mu2),
                                 c3f = fix_scale(mu3);
        FTMap f = ftmap_identity();
        for (long long n = lo; n < hi; ++n) {
            const uint4 b0 = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
            const uint4 b1 = philox(1u, static_cast<uint32_t>(n), rep, c3, rk);
            f = ftmap_push(f, to_fix(neg_log_q57(word_k(b0.x, b0.y), tab), cl),
                           to_fix(neg_log_q57(word_k(b0.z, b0.w), tab), c1),
                           to_fix(neg_log_q57(word_k(b1.x, b1.y), tab), c2),
                           to_fix(neg_log_q57(word_k(b1.z, b1.w), tab), c3f));
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const FTMap prev = ftmap_shfl_up(f, off);
            if (lane >= off) f = ftmap_compose(prev, f);
        }
        const FTMap excl = ftmap_shfl_up(f, 1);
        long long v1 = kFixNegInf, v2 = kFixNegInf, v3 = kFixNegInf;
        if (lane > 0) {
            v1 = excl.c1;
            v2 = excl.c2;
            v3 = excl.c3;
        }
        bool bad = v3 >= kFixGuard;
        U128 sy;
        double wa = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        for (long long n = lo; n < hi && !bad; ++n) {
            const uint4 b0 = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
            const uint4 b1 = philox(1u, static_cast<uint32_t>(n), rep, c3, rk);
            const unsigned long long ya = neg_log_q57(word_k(b0.x, b0.y), tab);
            const unsigned long long y1 = neg_log_q57(word_k(b0.z, b0.w), tab);
            const unsigned long long y2 = neg_log_q57(word_k(b1.x, b1.y), tab);
            const unsigned long long y3 = neg_log_q57(word_k(b1.z, b1.w), tab);
            const long long a = to_fix(ya, cl);
            long long q = v1 - a;
            v1 = ((q > 0) ? q : 0) + to_fix(y1, c1);
            q = v2 - a;
            v2 = ((q > v1) ? q : v1) + to_fix(y2, c2);
            q = v3 - a;
            v3 = ((q > v2) ? q : v2) + to_fix(y3, c3f);
            sy.add(v3);
            if (n < w_len) {
                wa += __ull2double_rn(ya) * i_lam;
                w1 += __ull2double_rn(y1) * i_mu1;
                w2 += __ull2double_rn(y2) * i_mu2;
                w3 += __ull2double_rn(y3) * i_mu3;
            }
            bad = v3 >= kFixGuard;
        }
        if (!__any_sync(kFull, bad)) {
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {  // lane-ordered tree (integers: exact)
                const U128 oy = shfl_down_u128(sy, off);
                const double oa = __shfl_down_sync(kFull, wa, off);
                const double o1 = __shfl_down_sync(kFull, w1, off);
                const double o2 = __shfl_down_sync(kFull, w2, off);
                const double o3 = __shfl_down_sync(kFull, w3, off);
                if ((lane & (2 * off - 1)) == 0) {
                    add_u128(sy, oy);
                    wa += oa;
                    w1 += o1;
                    w2 += o2;
                    w3 += o3;
                }
            }
            if (lane != 0) return;
            out.y[item] = sy.to_double() / static_cast<double>(n_clients);
            if (out.feat) {
                const double wl = static_cast<double>(w_len);
                double* fo = out.feat + item;
                const long long p = out.plane;
                fo[0] = lam;
                fo[p] = mu1;
                fo[2 * p] = mu2;
                fo[3 * p] = mu3;
                fo[4 * p] = wa / wl;
                fo[5 * p] = w1 / wl;
                fo[6 * p] = w2 / wl;
                fo[7 * p] = w3 / wl;
            }
            return;
        }
    }

    // FP64
    tandem_coop_fp64(item, dp, rep, lam, mu1, mu2, mu3, n_clients, window, c3, rk, tab, out);
}

// ---------------------------------------------------------------------------
// M/M/1, one replication per CTA (few replications of a latency-bound
// length): thread i takes the contiguous clients [i k, (i+1) k).  Pass 1
// composes each thread's Lindley maps W -> max(c, W + d); a block scan (warp
// shuffles, then the warp totals in shared memory) gives every thread the
// map of all clients before it, whose value at W_0 = 0 is its entry wait;
// pass 2 replays the thread's clients with the plain recurrence.  Times run
// in the 48-bit fixed point of the tandem, so composition is exact and the
// sums are exact integers (order-free); c and d saturate at +-2^61, which
// changes no map value for waits in [0, 2^60] unless a wait passes 2^60 --
// then, or for rates outside [2^-6, 2^4], the CTA redoes the replication in
// FP64 with the same structure (maps with -inf, sums in a fixed tree).
// ---------------------------------------------------------------------------

struct FixMap {
    long long c, d;
};
__device__ __forceinline__ FixMap fcompose(const FixMap& f, const FixMap& g) {  // g after f
    const long long cc = sat61(f.c + g.d);
    return FixMap{g.c > cc ? g.c : cc, sat61(f.d + g.d)};
}
struct DblMap {
    double c, d;
};
__device__ __forceinline__ DblMap dcompose(const DblMap& f, const DblMap& g) {
    const double cc = f.c + g.d;
    return DblMap{g.c > cc ? g.c : cc, f.d + g.d};
}

template <class Map>
__device__ __forceinline__ Map shfl_up_map(const Map& m, int off) {
    return Map{__shfl_up_sync(kFull, m.c, off), __shfl_up_sync(kFull, m.d, off)};
}

// Exclusive block scan of per-thread maps (thread order); `identity` for
// thread 0.  smem: one Map per warp.
template <class Map, class Compose>
__device__ Map block_exclusive_map(Map f, Map identity, Map* smem, Compose compose) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    Map incl = f;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Map prev = shfl_up_map(incl, off);
        if (lane >= off) incl = compose(prev, incl);
    }
    if (lane == 31) smem[warp] = incl;
    __syncthreads();
    Map before = identity;  // maps of the earlier warps, composed in order
    for (int w = 0; w < warp; ++w) before = compose(before, smem[w]);
    Map excl = shfl_up_map(incl, 1);
    if (lane == 0) excl = identity;
    __syncthreads();  // smem reusable
    return compose(before, excl);
}

struct Mm1Sums128 {
    U128 w, i, v;
};


__global__ void __launch_bounds__(1024) mm1_cta_kernel(const double* __restrict__ dps, long long n_reps,
                                                       long long rep0, long long n_clients, bool staged,
                                                       const __grid_constant__ RoundKeys rk, LogTable tab,
                                                       Mm1Out out) {
    extern __shared__ long long fix_stage[];  // [client - lo][thread] x (S, A) when staged
    __shared__ FixMap fmaps[32];
    __shared__ DblMap dmaps[32];
    __shared__ U128 part[3][32];
    __shared__ double dpart[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const long long item = blockIdx.x;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double lam = dps[2 * dp], mu = dps[2 * dp + 1];
    const uint32_t c3 = stream_word(0u, dp);
    const long long k = (n_clients + blockDim.x - 1) / blockDim.x;
    const long long lo = min(static_cast<long long>(threadIdx.x) * k, n_clients);
    const long long hi = min(lo + k, n_clients);
    const double inv_n = static_cast<double>(n_clients);
    // (debug build: a stage larger than the launch's shared memory is
    // recorded and the variates recomputed)
    staged = staged && MRIP_CHECK(2ull * k * blockDim.x * sizeof(long long) <= dynamic_smem_bytes(), 202, k);

    bool fixed_ok = fix_rate_ok(lam) && fix_rate_ok(mu);
    if (fixed_ok) {
        // every thread needs the same two multipliers (FP64 divisions on a
        // slow pipe): lane 0 of each warp computes them, a shuffle shares them
        unsigned long long cl = 0, cmu = 0;
        if (lane == 0) {
            cl = fix_scale(lam);
            cmu = fix_scale(mu);
        }
        cl = __shfl_sync(kFull, cl, 0);
        cmu = __shfl_sync(kFull, cmu, 0);
        FixMap f{-kSat, 0};
        long long* st_s = fix_stage + threadIdx.x;
        long long* st_a = fix_stage + k * blockDim.x + threadIdx.x;
        for (long long n = lo; n < hi; ++n) {
            const uint4 b = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
            const long long sv = to_fix(neg_log_q57(word_k(b.x, b.y), tab), cmu);
            const long long av = to_fix(neg_log_q57(word_k(b.z, b.w), tab), cl);
            if (staged) {
                st_s[(n - lo) * blockDim.x] = sv;
                st_a[(n - lo) * blockDim.x] = av;
            }
            f = fcompose(f, FixMap{0, sv - av});
        }
        const FixMap pre = block_exclusive_map(f, FixMap{-kSat, 0}, fmaps, fcompose);
        long long w = pre.c > pre.d ? pre.c : pre.d;  // map at W_0 = 0
        if (threadIdx.x == 0) w = 0;
        bool bad = w >= kFixGuard;
        Mm1Sums128 sm;
        for (long long n = lo; n < hi && !bad; ++n) {
            long long sv, av;
            if (staged) {
                sv = st_s[(n - lo) * blockDim.x];
                av = st_a[(n - lo) * blockDim.x];
            } else {
                const uint4 b = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
                sv = to_fix(neg_log_q57(word_k(b.x, b.y), tab), cmu);
                av = to_fix(neg_log_q57(word_k(b.z, b.w), tab), cl);
            }
            sm.w.add(w);
            const long long v = w + sv;
            sm.v.add(v);
            const long long t = v - av;
            sm.i.add(t < 0 ? -t : 0);
            w = t > 0 ? t : 0;
            bad = w >= kFixGuard;
        }
        fixed_ok = !__syncthreads_or(bad);
        if (fixed_ok) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                add_u128(sm.w, shfl_down_u128(sm.w, off));
                add_u128(sm.i, shfl_down_u128(sm.i, off));
                add_u128(sm.v, shfl_down_u128(sm.v, off));
            }
            if (lane == 0) {
                part[0][warp] = sm.w;
                part[1][warp] = sm.i;
                part[2][warp] = sm.v;
            }
            __syncthreads();
            if (threadIdx.x < 3) {
                U128 tot;
                for (int x = 0; x < nwarp; ++x) add_u128(tot, part[threadIdx.x][x]);
                double* dst = threadIdx.x == 0 ? out.wait : threadIdx.x == 1 ? out.idle : out.system;
                if (dst) dst[item] = tot.to_double() / inv_n;
            }
            return;
        }
    }
    // FP64: the same passes with doubles
    const double inv_lam = 0x1p-57 / lam, inv_mu = 0x1p-57 / mu;
    DblMap f{-INFINITY, 0.0};
    for (long long n = lo; n < hi; ++n) {
        double sv, av;
        mm1_client(static_cast<uint32_t>(n), rep, dp, inv_lam, inv_mu, rk, tab, sv, av);
        f = dcompose(f, DblMap{0.0, sv - av});
    }
    const DblMap pre = block_exclusive_map(f, DblMap{-INFINITY, 0.0}, dmaps, dcompose);
    double w = pre.c > pre.d ? pre.c : pre.d;
    if (threadIdx.x == 0) w = 0.0;
    double sw = 0.0, si = 0.0, sv_sum = 0.0;
    for (long long n = lo; n < hi; ++n) {
        double sv, av;
        mm1_client(static_cast<uint32_t>(n), rep, dp, inv_lam, inv_mu, rk, tab, sv, av);
        sw += w;
        const double v = w + sv;
        sv_sum += v;
        const double t = v - av;
        si += (t < 0.0) ? -t : 0.0;
        w = (t > 0.0) ? t : 0.0;
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {  // lane-ordered tree
        const double ow = __shfl_down_sync(kFull, sw, off);
        const double oi = __shfl_down_sync(kFull, si, off);
        const double ov = __shfl_down_sync(kFull, sv_sum, off);
        if ((lane & (2 * off - 1)) == 0) {
            sw += ow;
            si += oi;
            sv_sum += ov;
        }
    }
    if (lane == 0) {
        dpart[0][warp] = sw;
        dpart[1][warp] = si;
        dpart[2][warp] = sv_sum;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double tot = 0.0;
        for (int x = 0; x < nwarp; ++x) tot += dpart[threadIdx.x][x];
        double* dst = threadIdx.x == 0 ? out.wait : threadIdx.x == 1 ? out.idle : out.system;
        if (dst) dst[item] = tot / inv_n;
    }
}

// ---------------------------------------------------------------------------
// Tandem, one replication per CTA (few replications of a long horizon): thread
// i takes the contiguous clients [i k, (i+1) k); its fixed-point max-plus map
// (FTMap) is composed in pass 1, a block scan (warp shuffles, then the warp
// totals in order) gives every thread the map of all clients before it, and
// pass 2 replays its clients from that entry state.  Sojourn sums are exact
// 128-bit integers; the early-window sums FP64 in a fixed order.  Rates
// outside the fixed-point range or a sojourn past 2^12 hand the replication
// to the FP64 warp scan (warp 0).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) tandem3_cta_kernel(const double* __restrict__ dps, long long n_reps,
                                                           long long rep0, long long n_clients, long long window,
                                                           uint32_t tag, const __grid_constant__ RoundKeys rk,
                                                           LogTable tab, TandemOut out) {
    __shared__ FTMap wmap[32];
    __shared__ U128 wy[32];
    __shared__ double wsum[4][32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const long long item = blockIdx.x;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double lam = dps[4 * dp], mu1 = dps[4 * dp + 1], mu2 = dps[4 * dp + 2], mu3 = dps[4 * dp + 3];
    const uint32_t c3 = stream_word(tag, dp);
    const long long w_len = (n_clients < window) ? n_clients : window;
    const long long k = (n_clients + blockDim.x - 1) / blockDim.x;
    const long long lo = min(static_cast<long long>(t) * k, n_clients);
    const long long hi = min(lo + k, n_clients);

    if (fix_rate_ok(lam) && fix_rate_ok(mu1) && fix_rate_ok(mu2) && fix_rate_ok(mu3)) {
        const unsigned long long cl = fix_scale(lam), c1 = fix_scale(mu1), c2 = fix_scale(mu2),
                                 c3f = fix_scale(mu3);
        FTMap f = ftmap_identity();
        for (long long n = lo; n < hi; ++n) {
            const uint4 b0 = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
            const uint4 b1 = philox(1u, static_cast<uint32_t>(n), rep, c3, rk);
            f = ftmap_push(f, to_fix(neg_log_q57(word_k(b0.x, b0.y), tab), cl),
                           to_fix(neg_log_q57(word_k(b0.z, b0.w), tab), c1),
                           to_fix(neg_log_q57(word_k(b1.x, b1.y), tab), c2),
                           to_fix(neg_log_q57(word_k(b1.z, b1.w), tab), c3f));
        }
        // block exclusive scan of the maps
        FTMap incl = f;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const FTMap prev = ftmap_shfl_up(incl, off);
            if (lane >= off) incl = ftmap_compose(prev, incl);
        }
        if (lane == 31) wmap[warp] = incl;
        __syncthreads();
        FTMap pre = ftmap_identity();
        for (int w = 0; w < warp; ++w) pre = ftmap_compose(pre, wmap[w]);
        FTMap excl = ftmap_shfl_up(incl, 1);
        if (lane == 0) excl = ftmap_identity();
        pre = ftmap_compose(pre, excl);
        long long v1 = pre.c1, v2 = pre.c2, v3 = pre.c3;  // -2^61 for the first thread: empty
        bool bad = v3 >= kFixGuard;
        U128 sy;
        double wa = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        const double i_lam = 0x1p-57 / lam, i_mu1 = 0x1p-57 / mu1, i_mu2 = 0x1p-57 / mu2,
                     i_mu3 = 0x1p-57 / mu3;
        for (long long n = lo; n < hi && !bad; ++n) {
            const uint4 b0 = philox(0u, static_cast<uint32_t>(n), rep, c3, rk);
            const uint4 b1 = philox(1u, static_cast<uint32_t>(n), rep, c3, rk);
            const unsigned long long ya = neg_log_q57(word_k(b0.x, b0.y), tab);
            const unsigned long long y1 = neg_log_q57(word_k(b0.z, b0.w), tab);
            const unsigned long long y2 = neg_log_q57(word_k(b1.x, b1.y), tab);
            const unsigned long long y3 = neg_log_q57(word_k(b1.z, b1.w), tab);
            const long long a = to_fix(ya, cl);
            long long q = v1 - a;
            v1 = ((q > 0) ? q : 0) + to_fix(y1, c1);
            q = v2 - a;
            v2 = ((q > v1) ? q : v1) + to_fix(y2, c2);
            q = v3 - a;
            v3 = ((q > v2) ? q : v2) + to_fix(y3, c3f);
            sy.add(v3);
            if (n < w_len) {
                wa += __ull2double_rn(ya) * i_lam;
                w1 += __ull2double_rn(y1) * i_mu1;
                w2 += __ull2double_rn(y2) * i_mu2;
                w3 += __ull2double_rn(y3) * i_mu3;
            }
            bad = v3 >= kFixGuard;
        }
        if (!__syncthreads_or(bad)) {
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {  // lane-ordered tree (integers: exact)
                const U128 oy = shfl_down_u128(sy, off);
                const double oa = __shfl_down_sync(kFull, wa, off);
                const double o1 = __shfl_down_sync(kFull, w1, off);
                const double o2 = __shfl_down_sync(kFull, w2, off);
                const double o3 = __shfl_down_sync(kFull, w3, off);
                if ((lane & (2 * off - 1)) == 0) {
                    add_u128(sy, oy);
                    wa += oa;
                    w1 += o1;
                    w2 += o2;
                    w3 += o3;
                }
            }
            if (lane == 0) {
                wy[warp] = sy;
                wsum[0][warp] = wa;
                wsum[1][warp] = w1;
                wsum[2][warp] = w2;
                wsum[3][warp] = w3;
            }
            __syncthreads();
            if (t == 0) {
                U128 ty;
                double sa = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                for (int w = 0; w < nwarp; ++w) {
                    add_u128(ty, wy[w]);
                    sa += wsum[0][w];
                    s1 += wsum[1][w];
                    s2 += wsum[2][w];
                    s3 += wsum[3][w];
                }
                out.y[item] = ty.to_double() / static_cast<double>(n_clients);
                if (out.feat) {
                    const double wl = static_cast<double>(w_len);
                    double* fo = out.feat + item;
                    const long long p = out.plane;
                    fo[0] = lam;
                    fo[p] = mu1;
                    fo[2 * p] = mu2;
                    fo[3 * p] = mu3;
                    fo[4 * p] = sa / wl;
                    fo[5 * p] = s1 / wl;
                    fo[6 * p] = s2 / wl;
                    fo[7 * p] = s3 / wl;
                }
            }
            return;
        }
    }
    if (warp == 0) tandem_coop_fp64(item, dp, rep, lam, mu1, mu2, mu3, n_clients, window, c3, rk, tab, out);
}

}  // namespace
}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_mm1_simulate(const double* d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                                         int64_t n_clients, uint64_t seed, int mapping,
                                         double* d_wait, double* d_idle, double* d_system,
                                         void* stream) {
    if (n_dp < 0 || n_reps < 0 || rep0 < 0 || n_clients < 1)
        return fail(MRIP_EINVAL, "mrip_mm1_simulate: need n_dp, n_reps, rep0 >= 0 and n_clients >= 1");
    if (n_dp >= (1 << 24) || rep0 + n_reps > 0x100000000ll || n_clients > 0xFFFFFFFFll)
        return fail(MRIP_EINVAL, "mrip_mm1_simulate: n_dp < 2^24, replication indices < 2^32, n_clients <= 2^32-1");
    const long long n_items = static_cast<long long>(n_dp) * n_reps;
    if (n_items == 0) return MRIP_OK;
    if (!d_dps) return fail(MRIP_EINVAL, "mrip_mm1_simulate: null design points");
    const RoundKeys rk = expand_key(seed);
    LogTable tab;
    mrip_status ts = log_table(&tab);
    if (ts != MRIP_OK) return ts;
    Mm1Out out{d_wait, d_idle, d_system};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_THREAD) {
        mm1_serial_kernel<false><<<ceil_div_u(n_items, 128), 128, 0, st>>>(
            d_dps, n_items, n_reps, rep0, n_clients, rk, tab, out);
    } else if (mapping == MRIP_MAP_WARP_1LANE) {
        mm1_serial_kernel<true><<<ceil_div_u(n_items * 32, 128), 128, 0, st>>>(
            d_dps, n_items, n_reps, rep0, n_clients, rk, tab, out);
    } else if (mapping == MRIP_MAP_CTA) {
        if (n_items > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_mm1_simulate: too many replications for CTA");
        // about 4 clients per thread, 32 .. 1024 threads; fixed-point variates
        // staged in shared memory between the passes when they fit 96 KiB
        long long threads = ((n_clients + 3) / 4 + 31) / 32 * 32;
        threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
        const long long per_thread = (n_clients + threads - 1) / threads;
        const size_t stage = static_cast<size_t>(threads * per_thread) * 2 * sizeof(long long);
        const bool staged = stage <= 96 * 1024;  // plus ~3.3 KB of static shared memory
        if (staged && stage > 40 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(mm1_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 96 * 1024);
            if (e != cudaSuccess) return cuda_status(e, "mrip_mm1_simulate: shared memory attribute");
        }
        mm1_cta_kernel<<<static_cast<unsigned>(n_items), static_cast<unsigned>(threads), staged ? stage : 0, st>>>(
            d_dps, n_reps, rep0, n_clients, staged, rk, tab, out);
    } else if (mapping == MRIP_MAP_WARP_COOP) {
        const long long seg = (n_clients + 31) / 32;
        const size_t per_warp = static_cast<size_t>(seg) * 32 * 2 * sizeof(double);
        const int warps = 1;
        if (per_warp * warps <= 96 * 1024) {
            const size_t smem = per_warp * warps;
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(mm1_warp_coop_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem));
            mm1_warp_coop_kernel<true><<<ceil_div_u(n_items, warps), 32 * warps, smem, st>>>(
                d_dps, n_items, n_reps, rep0, n_clients, rk, tab, out);
        } else {
            mm1_warp_coop_kernel<false><<<ceil_div_u(n_items, 4), 128, 0, st>>>(
                d_dps, n_items, n_reps, rep0, n_clients, rk, tab, out);
        }
    } else {
        return fail(MRIP_EINVAL, "mrip_mm1_simulate: mapping must be THREAD, WARP_1LANE, WARP_COOP or CTA");
    }
    return launch_status("mrip_mm1_simulate");
}

extern "C" mrip_status mrip_tandem3_simulate(const double* d_dps, int32_t n_dp, int64_t rep0,
                                             int64_t n_reps, int64_t n_clients, int64_t window,
                                             uint64_t seed, uint32_t tag, int mapping,
                                             double* d_y, double* d_feat, void* stream) {
    if (n_dp < 0 || n_reps < 0 || rep0 < 0 || n_clients < 1 || window < 1)
        return fail(MRIP_EINVAL,
                    "mrip_tandem3_simulate: need n_dp, n_reps, rep0 >= 0 and n_clients, window >= 1");
    if (n_dp >= (1 << 24) || rep0 + n_reps > 0x100000000ll || n_clients > 0xFFFFFFFFll || tag > 255)
        return fail(MRIP_EINVAL,
                    "mrip_tandem3_simulate: n_dp < 2^24, replication indices < 2^32, tag < 256");
    const long long n_items = static_cast<long long>(n_dp) * n_reps;
    if (n_items == 0) return MRIP_OK;
    if (!d_dps || !d_y) return fail(MRIP_EINVAL, "mrip_tandem3_simulate: null pointer");
    const RoundKeys rk = expand_key(seed);
    LogTable tab;
    mrip_status ts = log_table(&tab);
    if (ts != MRIP_OK) return ts;
    TandemOut out{d_y, d_feat, n_items};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_THREAD) {
        tandem3_serial_kernel<false><<<ceil_div_u(n_items, 128), 128, 0, st>>>(
            d_dps, n_items, n_reps, rep0, n_clients, window, tag, rk, tab, out);
    } else if (mapping == MRIP_MAP_WARP_1LANE) {
        tandem3_serial_kernel<true><<<ceil_div_u(n_items * 32, 128), 128, 0, st>>>(
            d_dps, n_items, n_reps, rep0, n_clients, window, tag, rk, tab, out);
    } else if (mapping == MRIP_MAP_WARP_COOP) {
        tandem3_warp_coop_kernel<<<ceil_div_u(n_items * 32, 128), 128, 0, st>>>(
            d_dps, n_items, n_reps, rep0, n_clients, window, tag, rk, tab, out);
    } else if (mapping == MRIP_MAP_CTA) {
        if (n_items > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_tandem3_simulate: too many replications for CTA");
        // about 4 clients per thread, 32 .. 1024 threads
        long long threads = ((n_clients + 3) / 4 + 31) / 32 * 32;
        threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
        tandem3_cta_kernel<<<static_cast<unsigned>(n_items), static_cast<unsigned>(threads), 0, st>>>(
            d_dps, n_reps, rep0, n_clients, window, tag, rk, tab, out);
    } else {
        return fail(MRIP_EINVAL, "mrip_tandem3_simulate: mapping must be THREAD, WARP_1LANE, WARP_COOP or CTA");
    }
    return launch_status("mrip_tandem3_simulate");
}

MRIP_DEBUG_UNIT(queues)
