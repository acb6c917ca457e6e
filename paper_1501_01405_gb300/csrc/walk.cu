// L1-exit random walk: the uneven-length workload.  A simple random walk on
// Z^2 starts at the origin; tau is the number of moves until |x| + |y| = R.
// It adapts the random-walk model of the paper (Section 5.1, third model),
// whose WLP-versus-TLP comparison is the paper's central experiment
// (Section 5.3); stopping times vary over orders of magnitude, which is
// what the persistent work-stealing mapping is for.
//
// Move m reads the 2-bit field (m mod 64) of Philox block (c0 = 0,
// c1 = m div 64): word (m mod 64) div 16, bits 2 (m mod 16) and up.  Sixteen
// moves of one word are applied at once (their net displacement by popcount)
// whenever the walker is more than 16 away from the boundary; otherwise
// move by move with an exit check.  Both paths give the same walk.
//
// Mappings:
//   PERSISTENT  #SM x k CTAs; each warp takes chunks of replications from a
//               global ticket (atomicAdd) and refills a lane as soon as its
//               walker exits, so lanes stay busy despite uneven lengths;
//               words that may cross the boundary are walked by the whole
//               warp (walk_block_warp), so one lane near the boundary does
//               not serialise the other 31; when the ticket runs out, a
//               warp finishes its last walkers with all 32 lanes on one
//               walker at a time (walk_tail_coop, 2,048 moves per
//               round).  Default launch: one CTA of 32 warps per SM,
//               chunks of 16.
//   THREAD      one replication per thread (TLP), no refill.
//   WARP_1LANE  one replication per warp, lane 0 only (the paper's WLP).
//   WARP_COOP   one replication per warp: the 32 lanes take 32 consecutive
//               16-move words, a warp scan of their displacements gives each
//               lane's start, and a ballot finds the first exit.
#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"

namespace mrip {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kEven = 0x55555555u;

struct WalkJob {
    const int32_t* radius;  // by processing position k
    const int32_t* dp_of;   // design point by processing position k
    long long n_reps;
    long long rep0;         // replication index of output column 0
    long long total;
    long long max_steps;
    long long chunk;
    unsigned long long reps_magic;  // ceil(2^64 / n_reps) for n_reps >= 2 (0 for n_reps = 1)
    int64_t* tau;
    unsigned long long* ticket;
    int* err;
};

// Net displacement of the 16 moves packed in w.
__device__ __forceinline__ void word_displacement(uint32_t w, int& dx, int& dy) {
    const uint32_t sgn = w & kEven;
    const uint32_t axis = (w >> 1) & kEven;
    const int nx = __popc(~axis & kEven);
    dx = nx - 2 * __popc(~axis & sgn);
    dy = (16 - nx) - 2 * __popc(axis & sgn);
}

// Apply the 16 moves of w one by one from (x, y); returns the 1-based index
// of the exiting move, or 0 (then (x, y) is the end point).
__device__ __forceinline__ int word_steps(uint32_t w, int R, int& x, int& y) {
#pragma unroll 4
    for (int s = 0; s < 16; ++s) {
        const uint32_t f = (w >> (2 * s)) & 3u;
        const int step = 1 - 2 * static_cast<int>(f & 1u);
        if (f & 2u)
            y += step;
        else
            x += step;
        if (abs(x) + abs(y) >= R) return s + 1;
    }
    return 0;
}

// Advance through the 64 moves of one block; true on exit (m = tau).
__device__ __forceinline__ bool walk_block(const uint4 b, int R, int& x, int& y, long long& m) {
    const uint32_t words[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t w = words[k];
        if (abs(x) + abs(y) + 16 < R) {
            int dx, dy;
            word_displacement(w, dx, dy);
            x += dx;
            y += dy;
            m += 16;
        } else {
            const int e = word_steps(w, R, x, y);
            if (e) {
                m += e;
                return true;
            }
            m += 16;
        }
    }
    return false;
}

// Warp-convergent block step for the persistent mapping, in the diagonal
// coordinates u = x + y, v = x - y (|x| + |y| = max(|u|, |v|); a move changes
// u by +1 iff its bit 0 is clear and v by +1 iff its two bits agree).  Per
// 16-move word, a lane whose walker cannot leave within the word -- u plus
// the word's +1 steps in u below R, u minus its -1 steps above -R, the same
// for v -- applies the word at once (popcounts).  The other lanes' words are
// then walked by the whole warp, two lanes at a time: each half-warp takes
// one walker's 16 moves, one per lane, a 16-lane scan gives the positions
// and a ballot the first exit.
// This keeps the per-move work off the warp when one lane of 32 is near the
// boundary, which (with stopping times spread over orders of magnitude) is
// most of the time.  `live`: the lane has a walker; on return `done` marks
// walkers that exited in this block, `exit_at` (1..64) the exiting move
// within it.
//
// The no-exit test: u's positions within the word lie between u - mu and
// u - mu + 16 (mu its -1 steps), so with t = u - mu the word is safe in u iff
// -R < t < R - 16, i.e. t + R - 1 in [0, 2R - 17): one unsigned compare
// against lim = max(2R - 17, 0) (R <= 8: never safe).  The same for v.
__device__ __forceinline__ uint32_t walk_safe_limit(int R) { return R > 8 ? static_cast<uint32_t>(2 * R - 17) : 0u; }

__device__ __forceinline__ void walk_block_warp(const uint4 b, bool live, int R, uint32_t lim, int& u, int& v,
                                                int& exit_at, bool& done) {
    const int lane = threadIdx.x & 31;
    const uint32_t words[4] = {b.x, b.y, b.z, b.w};
    done = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t w = words[k];
        const int mu = __popc(w & kEven), mv = __popc((w ^ (w >> 1)) & kEven);  // -1 steps of u, of v
        const int tu = u - mu, tv = v - mv;
        const bool going = live && !done;
        const bool safe = static_cast<uint32_t>(tu + (R - 1)) < lim && static_cast<uint32_t>(tv + (R - 1)) < lim;
        if (going && safe) {
            u = tu + (16 - mu);
            v = tv + (16 - mv);
        }
        unsigned near = __ballot_sync(kFull, going && !safe);
        while (near) {  // two walkers per pass: lanes 0..15 and 16..31
            const int src0 = __ffs(near) - 1;
            near &= near - 1;
            int src1 = -1;
            if (near) {
                src1 = __ffs(near) - 1;
                near &= near - 1;
            }
            const int src = (lane >= 16 && src1 >= 0) ? src1 : src0;
            const uint32_t ws = __shfl_sync(kFull, w, src);
            const int us = __shfl_sync(kFull, u, src), vs = __shfl_sync(kFull, v, src);
            const int rs = __shfl_sync(kFull, R, src);
            const uint32_t f = (ws >> (2 * (lane & 15))) & 3u;
            int du = 1 - 2 * static_cast<int>(f & 1u);
            int dv = 1 - 2 * static_cast<int>((f ^ (f >> 1)) & 1u);
#pragma unroll
            for (int off = 1; off < 16; off <<= 1) {
                const int pu = __shfl_up_sync(kFull, du, off, 16);
                const int pv = __shfl_up_sync(kFull, dv, off, 16);
                if ((lane & 15) >= off) {
                    du += pu;
                    dv += pv;
                }
            }
            const unsigned hits = __ballot_sync(kFull, max(abs(us + du), abs(vs + dv)) >= rs);
            const int tu0 = __shfl_sync(kFull, du, 15), tv0 = __shfl_sync(kFull, dv, 15);
            const int tu1 = __shfl_sync(kFull, du, 31), tv1 = __shfl_sync(kFull, dv, 31);
            const bool me0 = lane == src0, me1 = lane == src1;
            if (me0 || me1) {
                const unsigned h = me0 ? (hits & 0xFFFFu) : (hits >> 16);
                if (h) {
                    exit_at = 16 * k + __ffs(h);
                    done = true;
                } else {
                    u += me0 ? tu0 : tu1;
                    v += me0 ? tv0 : tv1;
                }
            }
        }
    }
}

// Tail of the persistent mapping: once no replications are left to take and
// at most kTailLanes lanes of a warp still walk, the warp finishes those
// walkers one at a time, all 32 lanes on one walker.  Per round the walker
// advances 2,048 moves: lane l takes block blk + l (64 moves), a warp scan of
// the blocks' u and v displacements gives each block's start, a block that
// may reach the boundary is taken word by word (a word that may reach it
// move by move), and a ballot picks the first exit.  In the lane-parallel
// loop a walker makes 64 moves per warp round, so the longest walkers (the
// exit time has an exponential tail) would otherwise set the launch's length.
constexpr int kTailLanes = 16;

// Whole walk from (u, v) after blk blocks; returns tau, or -1 past max_steps.
// Warp-uniform arguments; every lane returns the same value.
__device__ long long walk_tail_coop(int u, int v, uint32_t blk, int R, uint32_t lim, uint32_t rep, uint32_t c3,
                                    long long max_steps, const RoundKeys& rk) {
    const int lane = threadIdx.x & 31;
    // the same no-exit test as walk_block_warp, over 64 moves: t + R - 1 in [0, 2R - 65)
    const uint32_t lim64 = R > 32 ? static_cast<uint32_t>(2 * R - 65) : 0u;
    while (true) {
        const uint4 b = philox(0u, blk + static_cast<uint32_t>(lane), rep, c3, rk);
        const uint32_t words[4] = {b.x, b.y, b.z, b.w};
        int mu = 0, mv = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            mu += __popc(words[k] & kEven);
            mv += __popc((words[k] ^ (words[k] >> 1)) & kEven);
        }
        const int du = 64 - 2 * mu, dv = 64 - 2 * mv;
        int su = du, sv = dv;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int pu = __shfl_up_sync(kFull, su, off), pv = __shfl_up_sync(kFull, sv, off);
            if (lane >= off) {
                su += pu;
                sv += pv;
            }
        }
        int pu = u + su - du, pv = v + sv - dv;  // position before this lane's block
        int e = 0;
        if (!(static_cast<uint32_t>(pu - mu + (R - 1)) < lim64 && static_cast<uint32_t>(pv - mv + (R - 1)) < lim64)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (e) break;
                const uint32_t w = words[k];
                const int wu = __popc(w & kEven), wv = __popc((w ^ (w >> 1)) & kEven);
                if (static_cast<uint32_t>(pu - wu + (R - 1)) < lim && static_cast<uint32_t>(pv - wv + (R - 1)) < lim) {
                    pu += 16 - 2 * wu;
                    pv += 16 - 2 * wv;
                    continue;
                }
                for (int s = 0; s < 16; ++s) {
                    const uint32_t f = (w >> (2 * s)) & 3u;
                    pu += (f & 1u) ? -1 : 1;
                    pv += ((f ^ (f >> 1)) & 1u) ? -1 : 1;
                    if (max(abs(pu), abs(pv)) >= R) {
                        e = 16 * k + s + 1;
                        break;
                    }
                }
            }
        }
        const unsigned ex = __ballot_sync(kFull, e != 0);
        if (ex) {
            const int first = __ffs(ex) - 1;
            const long long tau = 64LL * (static_cast<long long>(blk) + first) + __shfl_sync(kFull, e, first);
            return tau > max_steps ? -1 : tau;
        }
        // blocks past the cap are never used (and blk + 32 stays below 2^32)
        if (64LL * blk + 2048 >= max_steps) return -1;
        u += __shfl_sync(kFull, su, 31);
        v += __shfl_sync(kFull, sv, 31);
        blk += 32;
    }
}

// g div n_reps without a 64-bit division: hi(g * ceil(2^64 / n_reps)) exceeds
// g / n_reps by less than g / 2^64 < 1, so it is the quotient or one more,
// which the remainder's sign tells.
__device__ __forceinline__ void decode(const WalkJob& job, long long g, int& R, uint32_t& dp,
                                       uint32_t& rep, long long& out) {
    long long k = g;
    if (job.reps_magic) {
        k = static_cast<long long>(__umul64hi(static_cast<unsigned long long>(g), job.reps_magic));
        if (g - k * job.n_reps < 0) --k;
    }
    long long r = g - k * job.n_reps;
    // (debug build: the division and the tables must give a replication of
    // this launch and an output row inside it; a bad one is recorded and
    // replaced by item 0)
    if (!MRIP_CHECK(g >= 0 && g < job.total && r >= 0 && r < job.n_reps, 301, g)) {
        k = 0;
        r = 0;
    }
    rep = static_cast<uint32_t>(job.rep0 + r);
    R = job.radius[k];
    dp = static_cast<uint32_t>(job.dp_of[k]);
    out = static_cast<long long>(dp) * job.n_reps + r;
    if (!MRIP_CHECK(out < job.total && R >= 1, 302, out)) {
        out = 0;
        R = 1;
    }
}

// Whole replication on one thread (THREAD and WARP_1LANE mappings).
__device__ void walk_serial(const WalkJob& job, long long g, const RoundKeys& rk) {
    int R;
    uint32_t dp, rep;
    long long out;
    decode(job, g, R, dp, rep, out);
    int x = 0, y = 0;
    long long m = 0;
    const uint32_t c3 = stream_word(0u, dp);
    while (true) {
        const uint4 b = philox(0u, static_cast<uint32_t>(m >> 6), rep, c3, rk);
        if (walk_block(b, R, x, y, m)) {
            if (m > job.max_steps) break;
            job.tau[out] = m;
            return;
        }
        if (m >= job.max_steps) break;
    }
    job.tau[out] = -1;
    atomicExch(job.err, 1);
}

template <bool kLane0Only>
__global__ void walk_serial_kernel(WalkJob job, const __grid_constant__ RoundKeys rk) {
    long long g;
    if (kLane0Only) {
        if ((threadIdx.x & 31) != 0) return;
        g = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    } else {
        g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    }
    if (g >= job.total) return;
    walk_serial(job, g, rk);
}

__global__ void __launch_bounds__(1024) walk_persistent_kernel(WalkJob job, const __grid_constant__ RoundKeys rk) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    bool active = false;
    int u = 0, v = 0, R = 1;
    uint32_t lim = 0, blk = 0;  // blk: Philox block index, the walker has made 64 blk moves
    long long out = 0;
    uint32_t dp = 0, rep = 0, c3 = 0;
    long long next = 0, end = 0;  // warp-uniform range of the current chunk
    bool exhausted = false;       // warp-uniform
    while (true) {
        unsigned need = __ballot_sync(kFull, !active);
        while (need && !exhausted) {
            if (next >= end) {
                unsigned long long start = 0;
                if (lane == 0) start = atomicAdd(job.ticket, static_cast<unsigned long long>(job.chunk));
                start = __shfl_sync(kFull, start, 0);
                if (static_cast<long long>(start) >= job.total) {
                    exhausted = true;
                    break;
                }
                next = static_cast<long long>(start);
                end = next + job.chunk < job.total ? next + job.chunk : job.total;
            }
            const long long g = next + __popc(need & below);
            const bool take = ((need >> lane) & 1u) && g < end;
            if (take) {
                decode(job, g, R, dp, rep, out);
                c3 = stream_word(0u, dp);
                lim = walk_safe_limit(R);
                u = 0;
                v = 0;
                blk = 0;
                active = true;
            }
            const unsigned took = __ballot_sync(kFull, take);
            next += __popc(took);
            need &= ~took;
        }
        const unsigned act = __ballot_sync(kFull, active);
        if (!act) break;
        if (exhausted && __popc(act) <= kTailLanes) {
            for (unsigned rest = act; rest; rest &= rest - 1) {
                const int src = __ffs(rest) - 1;
                const long long tau = walk_tail_coop(
                    __shfl_sync(kFull, u, src), __shfl_sync(kFull, v, src), __shfl_sync(kFull, blk, src),
                    __shfl_sync(kFull, R, src), __shfl_sync(kFull, lim, src), __shfl_sync(kFull, rep, src),
                    __shfl_sync(kFull, c3, src), job.max_steps, rk);
                if (lane == src) {
                    job.tau[out] = tau;
                    if (tau < 0) atomicExch(job.err, 1);
                }
            }
            break;
        }
        const uint4 b = philox(0u, blk, rep, c3, rk);
        bool done;
        int exit_at = 0;
        walk_block_warp(b, active, R, lim, u, v, exit_at, done);
        if (active) {
            if (done) {
                const long long m = 64LL * blk + exit_at;
                if (m > job.max_steps) {
                    job.tau[out] = -1;
                    atomicExch(job.err, 1);
                } else {
                    job.tau[out] = m;
                }
                active = false;
            } else if (64LL * blk + 64 >= job.max_steps) {  // so blk stays below 2^32 (max_steps <= 2^38)
                job.tau[out] = -1;
                atomicExch(job.err, 1);
                active = false;
            } else {
                ++blk;
            }
        }
    }
}

// One replication per warp; lanes cover 512 consecutive moves per round.
__global__ void walk_warp_coop_kernel(WalkJob job, const __grid_constant__ RoundKeys rk) {
    const int lane = threadIdx.x & 31;
    const long long g = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    if (g >= job.total) return;  // warp-uniform
    int R;
    uint32_t dp, rep;
    long long out;
    decode(job, g, R, dp, rep, out);
    const uint32_t c3 = stream_word(0u, dp);
    int px = 0, py = 0;  // warp-uniform position before the round
    long long m = 0;     // warp-uniform move count before the round (multiple of 512)
    long long result = -1;
    while (m < job.max_steps) {
        const uint4 b = philox(0u, static_cast<uint32_t>((m >> 6) + (lane >> 2)), rep, c3, rk);
        const int sel = lane & 3;
        const uint32_t w = sel == 0 ? b.x : sel == 1 ? b.y : sel == 2 ? b.z : b.w;
        int dx, dy;
        word_displacement(w, dx, dy);
        int sx = dx, sy = dy;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int ox = __shfl_up_sync(kFull, sx, off);
            const int oy = __shfl_up_sync(kFull, sy, off);
            if (lane >= off) {
                sx += ox;
                sy += oy;
            }
        }
        int x = px + sx - dx, y = py + sy - dy;
        int e = 0;
        if (abs(x) + abs(y) + 16 >= R) e = word_steps(w, R, x, y);
        const unsigned hit = __ballot_sync(kFull, e != 0);
        if (hit) {
            const int first = __ffs(hit) - 1;
            const int ef = __shfl_sync(kFull, e, first);
            result = m + 16LL * first + ef;
            break;
        }
        px += __shfl_sync(kFull, sx, 31);
        py += __shfl_sync(kFull, sy, 31);
        m += 512;
    }
    if (lane == 0) {
        if (result < 0 || result > job.max_steps) {
            job.tau[out] = -1;
            atomicExch(job.err, 1);
        } else {
            job.tau[out] = result;
        }
    }
}

// ceil(2^64 / n) for n >= 2, 0 for n = 1 (WalkJob::reps_magic).
unsigned long long reps_reciprocal(long long n) {
    if (n < 2) return 0ull;
    return static_cast<unsigned long long>(((static_cast<unsigned __int128>(1) << 64) + n - 1) / n);
}

}  // namespace

// Launch on device-resident (radius, dp) tables in processing order.
mrip_status walk_launch(const int32_t* d_radius_by_pos, const int32_t* d_dp_by_pos, int32_t n_dp,
                        int64_t rep0, int64_t n_reps, uint64_t seed, int64_t max_steps, int mapping,
                        int32_t warps_per_cta, int32_t ctas_per_sm, int32_t chunk, int64_t* d_tau,
                        unsigned long long* d_ticket, cudaStream_t st) {
    WalkJob job;
    job.radius = d_radius_by_pos;
    job.dp_of = d_dp_by_pos;
    job.n_reps = n_reps;
    job.rep0 = rep0;
    job.total = static_cast<long long>(n_dp) * n_reps;
    job.max_steps = max_steps;
    job.chunk = chunk > 0 ? chunk : 16;
    job.reps_magic = reps_reciprocal(n_reps);
    job.tau = d_tau;
    job.ticket = d_ticket;
    job.err = device_error_flags();
    if (!job.err) return fail(MRIP_ENOMEM, "walk: device error flag allocation failed");
    const RoundKeys rk = expand_key(seed);
    if (job.total == 0) return MRIP_OK;
    if (mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_PERSISTENT) {
        const int wpc = warps_per_cta > 0 ? warps_per_cta : 32;  // one CTA of 32 warps per SM
        const int cps = ctas_per_sm > 0 ? ctas_per_sm : 1;
        if (wpc > 32 || cps > 64) return fail(MRIP_EINVAL, "walk: warps_per_cta <= 32, ctas_per_sm <= 64");
        if (!d_ticket) return fail(MRIP_EINVAL, "walk: persistent mapping needs a ticket counter");
        cudaError_t e = cudaMemsetAsync(d_ticket, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return cuda_status(e, "walk: ticket reset");
        walk_persistent_kernel<<<sm_count() * cps, 32 * wpc, 0, st>>>(job, rk);
    } else if (mapping == MRIP_MAP_THREAD) {
        walk_serial_kernel<false><<<ceil_div_u(job.total, 128), 128, 0, st>>>(job, rk);
    } else if (mapping == MRIP_MAP_WARP_1LANE) {
        walk_serial_kernel<true><<<ceil_div_u(job.total * 32, 128), 128, 0, st>>>(job, rk);
    } else if (mapping == MRIP_MAP_WARP_COOP) {
        walk_warp_coop_kernel<<<ceil_div_u(job.total * 32, 128), 128, 0, st>>>(job, rk);
    } else {
        return fail(MRIP_EINVAL, "walk: unknown mapping");
    }
    return launch_status("walk");
}

// Host-side validation and processing order: largest radius first, so the
// longest replications start early and the tail is short.
mrip_status walk_tables(const double* radii, int32_t n_dp, std::vector<int32_t>& r_by_pos,
                        std::vector<int32_t>& dp_by_pos) {
    r_by_pos.resize(n_dp);
    dp_by_pos.resize(n_dp);
    std::vector<int32_t> order(n_dp);
    for (int32_t i = 0; i < n_dp; ++i) {
        const double r = radii[i];
        if (!(r >= 1.0 && r <= 65536.0) || r != static_cast<double>(static_cast<int32_t>(r)))
            return fail(MRIP_EINVAL, "walk: R must be an integer in 1..65536");
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return radii[a] > radii[b]; });
    for (int32_t k = 0; k < n_dp; ++k) {
        dp_by_pos[k] = order[k];
        r_by_pos[k] = static_cast<int32_t>(radii[order[k]]);
    }
    return MRIP_OK;
}

// ---------------------------------------------------------------------------
// Entry point for callers that cannot allocate device memory.
//
// Its scratch (work-stealing ticket, step-cap flag, radius and design-point
// tables) lives in one file-scope device array instead of library-allocated
// buffers.  Host code cannot pass the array's name to a kernel (in host code
// it is only a stand-in): every call looks the current device's address up
// with cudaGetSymbolAddress.  The tables travel to the GPU as a kernel
// argument (at most 8 KiB), and a one-CTA set-up kernel writes them and
// clears the ticket and the flag, so the call neither copies from host
// memory nor waits for the GPU.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxDp = 1024;
constexpr size_t kNoAllocHeader = 256;  // [0, 8) ticket, [8, 12) step-cap flag
constexpr size_t kNoAllocBytes = kNoAllocHeader + 2 * sizeof(int32_t) * kNoAllocMaxDp;

static __device__ __align__(256) unsigned char g_walk_noalloc_scratch[kNoAllocBytes];

namespace {
struct NoAllocTables {
    int32_t r_by_pos[kNoAllocMaxDp];
    int32_t dp_by_pos[kNoAllocMaxDp];
    int32_t n_dp;
};

__global__ void __launch_bounds__(256) walk_noalloc_setup(const __grid_constant__ NoAllocTables t,
                                                          unsigned char* base) {
    if (!MRIP_CHECK(t.n_dp >= 0 && t.n_dp <= kNoAllocMaxDp, 303, t.n_dp)) return;
    int32_t* d_r = reinterpret_cast<int32_t*>(base + kNoAllocHeader);
    int32_t* d_d = d_r + t.n_dp;
    for (int i = threadIdx.x; i < t.n_dp; i += blockDim.x) {
        d_r[i] = t.r_by_pos[i];
        d_d[i] = t.dp_by_pos[i];
    }
    if (threadIdx.x == 0) {
        *reinterpret_cast<unsigned long long*>(base) = 0ull;  // ticket
        *reinterpret_cast<int*>(base + 8) = 0;                 // step-cap flag
    }
}
}  // namespace

}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_walk_simulate_noalloc(const double* radii, int32_t n_dp, int64_t rep0,
                                                  int64_t n_reps, uint64_t seed, int64_t max_steps,
                                                  int mapping, int32_t warps_per_cta,
                                                  int32_t ctas_per_sm, int32_t chunk, int64_t* d_tau,
                                                  void* stream) {
    if (n_dp < 0 || n_reps < 0 || rep0 < 0)
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: negative size");
    if (n_dp > kNoAllocMaxDp)
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: n_dp " + std::to_string(n_dp) +
                                     " exceeds its fixed scratch limit of " +
                                     std::to_string(kNoAllocMaxDp) + " design points");
    if (rep0 + n_reps > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: replication indices < 2^32");
    if (max_steps < 1 || max_steps > (1LL << 38))
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: max_steps in 1..2^38");
    if (chunk < 0 || chunk > (1 << 20))
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: chunk in 0..2^20");
    if (static_cast<long long>(n_dp) * n_reps == 0) return MRIP_OK;
    if (!radii || !d_tau) return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: null pointer");
    // processing order: largest radius first (stable insertion sort)
    NoAllocTables t;
    t.n_dp = n_dp;
    for (int32_t i = 0; i < n_dp; ++i) {
        const double r = radii[i];
        if (!(r >= 1.0 && r <= 65536.0) || r != static_cast<double>(static_cast<int32_t>(r)))
            return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: R must be an integer in 1..65536");
        int32_t pos = i;
        while (pos > 0 && t.r_by_pos[pos - 1] < static_cast<int32_t>(r)) {
            t.r_by_pos[pos] = t.r_by_pos[pos - 1];
            t.dp_by_pos[pos] = t.dp_by_pos[pos - 1];
            --pos;
        }
        t.r_by_pos[pos] = static_cast<int32_t>(r);
        t.dp_by_pos[pos] = i;
    }
    if (mapping != MRIP_MAP_AUTO && mapping != MRIP_MAP_PERSISTENT && mapping != MRIP_MAP_THREAD &&
        mapping != MRIP_MAP_WARP_1LANE && mapping != MRIP_MAP_WARP_COOP)
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: unknown mapping");
    const int wpc = warps_per_cta > 0 ? warps_per_cta : 32;
    const int cps = ctas_per_sm > 0 ? ctas_per_sm : 1;
    if (wpc > 32 || cps > 64)
        return fail(MRIP_EINVAL, "mrip_walk_simulate_noalloc: warps_per_cta <= 32, ctas_per_sm <= 64");

    // this device's address of the array (looked up on every call: cheap, and
    // never stale)
    void* base_v = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base_v, g_walk_noalloc_scratch);
    if (e != cudaSuccess || !base_v)
        return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                           "mrip_walk_simulate_noalloc: cudaGetSymbolAddress");
    unsigned char* base = static_cast<unsigned char*>(base_v);
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) return cuda_status(e, "mrip_walk_simulate_noalloc: SM count");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    walk_noalloc_setup<<<1, 256, 0, st>>>(t, base);
    mrip_status s = launch_status("mrip_walk_simulate_noalloc: set-up");
    if (s != MRIP_OK) return s;

    WalkJob job;
    job.radius = reinterpret_cast<int32_t*>(base + kNoAllocHeader);
    job.dp_of = job.radius + n_dp;
    job.n_reps = n_reps;
    job.rep0 = rep0;
    job.total = static_cast<long long>(n_dp) * n_reps;
    job.max_steps = max_steps;
    job.chunk = chunk > 0 ? chunk : 16;
    job.reps_magic = reps_reciprocal(n_reps);
    job.tau = d_tau;
    job.ticket = reinterpret_cast<unsigned long long*>(base);
    job.err = reinterpret_cast<int*>(base + 8);
    const RoundKeys rk = expand_key(seed);
    if (mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_PERSISTENT) {
        walk_persistent_kernel<<<sms * cps, 32 * wpc, 0, st>>>(job, rk);
    } else if (mapping == MRIP_MAP_THREAD) {
        walk_serial_kernel<false><<<ceil_div_u(job.total, 128), 128, 0, st>>>(job, rk);
    } else if (mapping == MRIP_MAP_WARP_1LANE) {
        walk_serial_kernel<true><<<ceil_div_u(job.total * 32, 128), 128, 0, st>>>(job, rk);
    } else {
        walk_warp_coop_kernel<<<ceil_div_u(job.total * 32, 128), 128, 0, st>>>(job, rk);
    }
    return launch_status("mrip_walk_simulate_noalloc");
}

extern "C" mrip_status mrip_walk_simulate(const double* radii, int32_t n_dp, int64_t rep0, int64_t n_reps,
                                          uint64_t seed, int64_t max_steps, int mapping,
                                          int32_t warps_per_cta, int32_t ctas_per_sm,
                                          int32_t chunk, int64_t* d_tau, void* stream) {
    if (n_dp < 0 || n_reps < 0 || rep0 < 0) return fail(MRIP_EINVAL, "mrip_walk_simulate: negative size");
    if (n_dp >= (1 << 24) || rep0 + n_reps > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_walk_simulate: n_dp < 2^24 and replication indices < 2^32");
    if (max_steps < 1 || max_steps > (1LL << 38))
        return fail(MRIP_EINVAL, "mrip_walk_simulate: max_steps in 1..2^38");
    if (chunk < 0 || chunk > (1 << 20)) return fail(MRIP_EINVAL, "mrip_walk_simulate: chunk in 0..2^20");
    if (static_cast<long long>(n_dp) * n_reps == 0) return MRIP_OK;
    if (!radii || !d_tau) return fail(MRIP_EINVAL, "mrip_walk_simulate: null pointer");
    std::vector<int32_t> r_by_pos, dp_by_pos;
    mrip_status s = walk_tables(radii, n_dp, r_by_pos, dp_by_pos);
    if (s != MRIP_OK) return s;
    // tables and ticket in scratch slot 0: [ticket 256 B][radius][dp]
    const size_t tab = static_cast<size_t>(n_dp) * sizeof(int32_t);
    char* base = static_cast<char*>(scratch(256 + 2 * tab, 0));
    if (!base) return fail(MRIP_ENOMEM, "mrip_walk_simulate: scratch allocation failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t* d_r = reinterpret_cast<int32_t*>(base + 256);
    int32_t* d_d = reinterpret_cast<int32_t*>(base + 256 + tab);
    cudaError_t e = cudaMemcpyAsync(d_r, r_by_pos.data(), tab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_d, dp_by_pos.data(), tab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors die at return
    if (e != cudaSuccess) return cuda_status(e, "mrip_walk_simulate: table upload");
    return walk_launch(d_r, d_d, n_dp, rep0, n_reps, seed, max_steps, mapping, warps_per_cta, ctas_per_sm,
                       chunk, d_tau, reinterpret_cast<unsigned long long*>(base), st);
}

MRIP_DEBUG_UNIT(walk)
