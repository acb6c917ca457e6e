// Area walk: the paper's random-walk model (Section 5.1, third model) and
// the experiment it uses to compare one replication per warp (WLP) with one
// per thread (TLP) (Section 5.3).  A walker moves on a 60 x 50 periodic map
// split into 30 areas of 10 x 10 cells (area x/10 + 6 (y/10)), starting at
// (30, 25); move m reads field m mod 64 of Philox block (c0 = 0,
// c1 = m div 64) (0:+x 1:-x 2:+y 3:-y); after every move the visit count of
// the walker's area grows by one.  Outputs: final area and 30 visit counts.
//
// Mappings:
//   THREAD      one replication per thread; the CTA keeps one histogram per
//               thread in shared memory laid out [area][thread], so the
//               per-move scatter never conflicts on a bank;
//   WARP_1LANE  one replication per warp, lane 0 only (the paper's WLP);
//   WARP_COOP   one replication per warp: a round covers 512 moves, lane l
//               takes moves 16l .. 16l+15, a warp scan of the 16-move
//               displacements (popcounts) gives each lane's start, and the
//               lanes add their visits to one warp histogram.
#include "common.cuh"

namespace mrip {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kEven = 0x55555555u;
constexpr int kW = 60, kH = 50, kCell = 10, kAreas = 30, kThreads = 128;

__device__ __forceinline__ int area_of(int x, int y) { return x / kCell + (kW / kCell) * (y / kCell); }

__device__ __forceinline__ void move(uint32_t f, int& x, int& y) {
    if (f & 2u) {
        y += (f & 1u) ? kH - 1 : 1;
        if (y >= kH) y -= kH;
    } else {
        x += (f & 1u) ? kW - 1 : 1;
        if (x >= kW) x -= kW;
    }
}

// One replication on one thread; hist points at this walker's column.
__device__ void walk_serial(uint32_t rep, int n_steps, const RoundKeys& rk, uint32_t* hist,
                            int stride, int32_t* final_area) {
    int x = kW / 2, y = kH / 2;
    const uint32_t c3 = stream_word(0u, 0u);
    for (int m0 = 0; m0 < n_steps; m0 += 64) {
        const uint4 b = philox(0u, static_cast<uint32_t>(m0 >> 6), rep, c3, rk);
        const uint32_t words[4] = {b.x, b.y, b.z, b.w};
        const int n = min(64, n_steps - m0);
        for (int s = 0; s < n; ++s) {
            move((words[s >> 4] >> (2 * (s & 15))) & 3u, x, y);
            const int a = area_of(x, y);
            if (MRIP_CHECK(a >= 0 && a < kAreas, 601, a)) hist[a * stride] += 1u;
        }
    }
    *final_area = area_of(x, y);
}

template <bool kLane0Only>
__global__ void __launch_bounds__(kThreads) area_walk_serial_kernel(long long rep0, long long n_reps, int n_steps,
                                                                    const __grid_constant__ RoundKeys rk,
                                                                    int32_t* __restrict__ final_area,
                                                                    int32_t* __restrict__ visits) {
    __shared__ uint32_t hist[kAreas * kThreads];  // [area][slot]
    const int slot = kLane0Only ? (threadIdx.x >> 5) : threadIdx.x;
    const int stride = kLane0Only ? kThreads / 32 : kThreads;
    long long item;
    if (kLane0Only) {
        if ((threadIdx.x & 31) != 0) return;
        item = (blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x) >> 5;
    } else {
        item = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
    }
    if (item >= n_reps) return;
    for (int a = 0; a < kAreas; ++a) hist[a * stride + slot] = 0u;
    int32_t fa;
    walk_serial(static_cast<uint32_t>(rep0 + item), n_steps, rk, hist + slot, stride, &fa);
    final_area[item] = fa;
    if (visits)
        for (int a = 0; a < kAreas; ++a) visits[a * n_reps + item] = static_cast<int32_t>(hist[a * stride + slot]);
}

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

__global__ void __launch_bounds__(kThreads) area_walk_coop_kernel(long long rep0, long long n_reps, int n_steps,
                                                                  const __grid_constant__ RoundKeys rk,
                                                                  int32_t* __restrict__ final_area,
                                                                  int32_t* __restrict__ visits) {
    __shared__ uint32_t hist[kThreads / 32][kAreas];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long item = (blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x) >> 5;
    if (item >= n_reps) return;  // warp-uniform
    if (lane < kAreas) hist[warp][lane] = 0u;
    __syncwarp();
    const uint32_t rep = static_cast<uint32_t>(rep0 + item);
    const uint32_t c3 = stream_word(0u, 0u);
    int px = kW / 2, py = kH / 2;  // warp-uniform position before the round
    for (int m0 = 0; m0 < n_steps; m0 += 512) {
        const uint4 b = philox(0u, static_cast<uint32_t>((m0 >> 6) + (lane >> 2)), rep, c3, rk);
        const int sel = lane & 3;
        const uint32_t w = sel == 0 ? b.x : sel == 1 ? b.y : sel == 2 ? b.z : b.w;
        const int first = m0 + 16 * lane;
        const int cnt = max(0, min(16, n_steps - first));
        // displacement of this lane's moves (only the ones that exist)
        const uint32_t valid = cnt == 16 ? 0xFFFFFFFFu : ((1u << (2 * cnt)) - 1u);
        const uint32_t sgn = w & kEven & valid;
        const uint32_t axis = (w >> 1) & kEven & valid;
        const uint32_t used = kEven & valid;
        const int nx = __popc(~axis & used);
        const int dx = nx - 2 * __popc(~axis & sgn);
        const int dy = (cnt - nx) - 2 * __popc(axis & sgn);
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
        int x = wrap(px + sx - dx, kW), y = wrap(py + sy - dy, kH);
        for (int s = 0; s < cnt; ++s) {
            move((w >> (2 * s)) & 3u, x, y);
            const int a = area_of(x, y);
            if (MRIP_CHECK(a >= 0 && a < kAreas, 602, a)) atomicAdd(&hist[warp][a], 1u);
        }
        px = wrap(px + __shfl_sync(kFull, sx, 31), kW);
        py = wrap(py + __shfl_sync(kFull, sy, 31), kH);
    }
    __syncwarp();
    if (lane == 0) final_area[item] = area_of(px, py);
    if (visits && lane < kAreas) visits[lane * n_reps + item] = static_cast<int32_t>(hist[warp][lane]);
}

}  // namespace
}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_area_walk_simulate(int64_t rep0, int64_t n_reps, int32_t n_steps, uint64_t seed,
                                               int mapping, int32_t* d_final_area, int32_t* d_visits,
                                               void* stream) {
    if (rep0 < 0 || n_reps < 0 || n_steps < 0) return fail(MRIP_EINVAL, "mrip_area_walk_simulate: negative size");
    if (rep0 + n_reps > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_area_walk_simulate: replication indices < 2^32");
    if (n_steps > (1 << 30)) return fail(MRIP_EINVAL, "mrip_area_walk_simulate: n_steps <= 2^30");
    if (n_reps == 0) return MRIP_OK;
    if (!d_final_area) return fail(MRIP_EINVAL, "mrip_area_walk_simulate: null output");
    const RoundKeys rk = expand_key(seed);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_THREAD) {
        area_walk_serial_kernel<false><<<ceil_div_u(n_reps, kThreads), kThreads, 0, st>>>(rep0, n_reps, n_steps, rk,
                                                                                          d_final_area, d_visits);
    } else if (mapping == MRIP_MAP_WARP_1LANE) {
        area_walk_serial_kernel<true><<<ceil_div_u(n_reps * 32, kThreads), kThreads, 0, st>>>(
            rep0, n_reps, n_steps, rk, d_final_area, d_visits);
    } else if (mapping == MRIP_MAP_WARP_COOP) {
        area_walk_coop_kernel<<<ceil_div_u(n_reps * 32, kThreads), kThreads, 0, st>>>(rep0, n_reps, n_steps, rk,
                                                                                     d_final_area, d_visits);
    } else {
        return fail(MRIP_EINVAL, "mrip_area_walk_simulate: mapping must be THREAD, WARP_1LANE or WARP_COOP");
    }
    return launch_status("mrip_area_walk_simulate");
}

MRIP_DEBUG_UNIT(area_walk)
