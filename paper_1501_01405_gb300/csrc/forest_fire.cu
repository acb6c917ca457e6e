// Stochastic forest-fire cellular automaton (Drossel-Schwabl rules), one
// replication per CTA.
//
// Layout: the L x L lattice (L = 32 W) is two bit planes, "tree" and
// "burning", one 32-bit word per 32 cells of a row (bit m of word j of row y
// is cell x = 32 j + m).  Thread y owns row y in registers.  A cell's north
// and south neighbours come from the adjacent lanes by warp shuffle; the
// first and last row of each warp are exchanged through a double-buffered
// shared-memory halo, so one barrier per step suffices.  East and west
// neighbours are shifts within the row (periodic).  The random word of cell
// i = y L + x at step t is word (i mod 4) of Philox block (c0 = i div 4,
// c1 = t); a thread compares its 32 cells' words with the growth and
// lightning thresholds and packs the results into two words, then the new
// state of 32 cells is a handful of bitwise operations:
//   ignite = burning neighbour | lightning,
//   burning' = tree & ignite,
//   tree'    = (tree & ~ignite) | (empty & grow).
// The burning count of each step is a popcount, a warp reduction and a
// shared-memory atomic; counts are flushed to global memory every 64 steps
// (coalesced) from a double-buffered slot array.
#include "common.cuh"

namespace mrip {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int W>
__global__ void __launch_bounds__(32 * W) forest_fire_kernel(
    const double* __restrict__ dps, long long n_reps, int n_steps, uint32_t t_dens,
    const __grid_constant__ RoundKeys rk, const uint8_t* __restrict__ init,
    int32_t* __restrict__ counts, double* __restrict__ scalar, uint8_t* __restrict__ final_state) {
    constexpr int L = 32 * W;
    constexpr int NWARP = W;  // L rows, 32 rows per warp
    __shared__ uint32_t halo[2][2][NWARP][W];  // [state parity][first/last row][warp][word]
    __shared__ int cnt[2][64];
    __shared__ long long red[NWARP];

    const int y = threadIdx.x;
    const int lane = y & 31;
    const int warp = y >> 5;
    const long long item = blockIdx.x;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(item % n_reps);
    const uint32_t t_grow = threshold32(dps[2 * dp]);
    const uint32_t t_light = threshold32(dps[2 * dp + 1]);
    const uint32_t c3 = stream_word(0u, dp);
    const uint32_t row_c0 = static_cast<uint32_t>(y) * (L / 4);

    uint32_t T[W], B[W];
    if (init) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(
            init + item * static_cast<long long>(L) * L + static_cast<long long>(y) * L);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            uint32_t tw = 0, bw = 0;
            for (int r = 0; r < 8; ++r) {
                const uint32_t v = src[8 * j + r];
                for (int k = 0; k < 4; ++k) {
                    const uint32_t s = (v >> (8 * k)) & 0xFFu;
                    tw |= (s == 1u ? 1u : 0u) << (4 * r + k);
                    bw |= (s == 2u ? 1u : 0u) << (4 * r + k);
                }
            }
            T[j] = tw;
            B[j] = bw;
        }
    } else {
        const uint32_t c3i = stream_word(1u, dp);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            uint32_t tw = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 b = philox(row_c0 + 8 * j + q, 0u, rep, c3i, rk);
                tw |= (b.x < t_dens) ? (1u << (4 * q)) : 0u;
                tw |= (b.y < t_dens) ? (1u << (4 * q + 1)) : 0u;
                tw |= (b.z < t_dens) ? (1u << (4 * q + 2)) : 0u;
                tw |= (b.w < t_dens) ? (1u << (4 * q + 3)) : 0u;
            }
            T[j] = tw;
            B[j] = 0u;
        }
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) (&cnt[0][0])[i] = 0;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < W; ++j) halo[0][0][warp][j] = B[j];
    }
    if (lane == 31) {
#pragma unroll
        for (int j = 0; j < W; ++j) halo[0][1][warp][j] = B[j];
    }
    __syncthreads();

    const int wprev = (warp + NWARP - 1) % NWARP;
    const int wnext = (warp + 1) % NWARP;
    long long my_sum = 0;
    for (int t = 1; t <= n_steps; ++t) {
        const int rp = (t - 1) & 1;
        uint32_t TN[W], BN[W];
        int c = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            uint32_t up = __shfl_up_sync(kFull, B[j], 1);
            uint32_t dn = __shfl_down_sync(kFull, B[j], 1);
            if (lane == 0) up = halo[rp][1][wprev][j];
            if (lane == 31) dn = halo[rp][0][wnext][j];
            const uint32_t west = (B[j] << 1) | (B[(j + W - 1) % W] >> 31);
            const uint32_t east = (B[j] >> 1) | (B[(j + 1) % W] << 31);
            const uint32_t nb = up | dn | west | east;
            uint32_t g = 0, l = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 b = philox(row_c0 + 8 * j + q, static_cast<uint32_t>(t), rep, c3, rk);
                g |= (b.x < t_grow) ? (1u << (4 * q)) : 0u;
                g |= (b.y < t_grow) ? (1u << (4 * q + 1)) : 0u;
                g |= (b.z < t_grow) ? (1u << (4 * q + 2)) : 0u;
                g |= (b.w < t_grow) ? (1u << (4 * q + 3)) : 0u;
                l |= (b.x < t_light) ? (1u << (4 * q)) : 0u;
                l |= (b.y < t_light) ? (1u << (4 * q + 1)) : 0u;
                l |= (b.z < t_light) ? (1u << (4 * q + 2)) : 0u;
                l |= (b.w < t_light) ? (1u << (4 * q + 3)) : 0u;
            }
            const uint32_t ignite = nb | l;
            BN[j] = T[j] & ignite;
            TN[j] = (T[j] & ~ignite) | (~(T[j] | B[j]) & g);
            c += __popc(BN[j]);
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            T[j] = TN[j];
            B[j] = BN[j];
        }
        c = __reduce_add_sync(kFull, c);
        if (lane == 0) atomicAdd(&cnt[((t - 1) >> 6) & 1][(t - 1) & 63], c);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < W; ++j) halo[t & 1][0][warp][j] = B[j];
        }
        if (lane == 31) {
#pragma unroll
            for (int j = 0; j < W; ++j) halo[t & 1][1][warp][j] = B[j];
        }
        __syncthreads();
        if ((t & 63) == 0 || t == n_steps) {
            const int chunk = (t - 1) >> 6;
            const int n_slot = t - chunk * 64;
            for (int s = threadIdx.x; s < n_slot; s += blockDim.x) {
                const int v = cnt[chunk & 1][s];
                cnt[chunk & 1][s] = 0;
                my_sum += v;
                if (counts) counts[item * n_steps + chunk * 64 + s] = v;
            }
        }
    }

    if (scalar) {
        long long s = my_sum;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(kFull, s, off);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tot = 0;
            for (int w = 0; w < NWARP; ++w) tot += red[w];
            scalar[item] = static_cast<double>(tot) /
                           (static_cast<double>(n_steps) * static_cast<double>(L) * L);
        }
    }
    if (final_state) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(
            final_state + item * static_cast<long long>(L) * L + static_cast<long long>(y) * L);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            for (int r = 0; r < 8; ++r) {
                uint32_t v = 0;
                for (int k = 0; k < 4; ++k) {
                    const int m = 4 * r + k;
                    const uint32_t s = ((T[j] >> m) & 1u) ? 1u : (((B[j] >> m) & 1u) ? 2u : 0u);
                    v |= s << (8 * k);
                }
                dst[8 * j + r] = v;
            }
        }
    }
}

template <int W>
void launch_ff(const double* dps, long long n_items, long long n_reps, int n_steps, uint32_t t_dens,
               const RoundKeys& rk, const uint8_t* init, int32_t* counts, double* scalar,
               uint8_t* final_state, cudaStream_t st) {
    forest_fire_kernel<W><<<static_cast<unsigned>(n_items), 32 * W, 0, st>>>(
        dps, n_reps, n_steps, t_dens, rk, init, counts, scalar, final_state);
}

}  // namespace
}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_forest_fire_simulate(const double* d_dps, int32_t n_dp, int64_t n_reps,
                                                 int32_t L, int32_t n_steps, double density,
                                                 uint64_t seed, const uint8_t* d_init,
                                                 int32_t* d_counts, double* d_scalar,
                                                 uint8_t* d_final, void* stream) {
    if (n_dp < 0 || n_reps < 0 || n_steps < 0)
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: negative size");
    if (L < 32 || L > 512 || L % 32 != 0 || (L & (L - 1)) != 0)
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: L must be 32, 64, 128, 256 or 512");
    if (!(density >= 0.0 && density < 1.0))
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: density must be in [0, 1)");
    if (n_dp >= (1 << 24) || n_reps > 0xFFFFFFFFll)
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: n_dp < 2^24 and n_reps < 2^32");
    const long long n_items = static_cast<long long>(n_dp) * n_reps;
    if (n_items == 0) return MRIP_OK;
    if (n_items > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: too many replications");
    if (!d_dps) return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: null design points");
    if ((d_init && (reinterpret_cast<uintptr_t>(d_init) & 15u)) ||
        (d_final && (reinterpret_cast<uintptr_t>(d_final) & 15u)))
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: state buffers need 16-byte alignment");
    const RoundKeys rk = expand_key(seed);
    const uint32_t t_dens = threshold32(density);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (L) {
        case 32: launch_ff<1>(d_dps, n_items, n_reps, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 64: launch_ff<2>(d_dps, n_items, n_reps, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 128: launch_ff<4>(d_dps, n_items, n_reps, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 256: launch_ff<8>(d_dps, n_items, n_reps, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 512: launch_ff<16>(d_dps, n_items, n_reps, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
    }
    return launch_status("mrip_forest_fire_simulate");
}
