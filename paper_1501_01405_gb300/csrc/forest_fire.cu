// Stochastic forest-fire cellular automaton (Drossel-Schwabl rules), one
// replication per CTA, the lattice held in shared memory.
//
// Layout: the L x L lattice (L = 32 W) is two bit planes, "tree" and
// "burning", one 32-bit word per 32 cells of a row (bit m of word k =
// y W + j is cell x = 32 j + m of row y).  Both planes are double-buffered
// in shared memory (2 buffers x 2 planes x L W words = 16 L W bytes); a step reads buffer
// (t-1) mod 2 and writes buffer t mod 2, so one barrier per step suffices.
// Thread i of the CTA updates words i, i + blockDim, ...: the word's
// north/south neighbours are the words W above and below (periodic), its
// east/west neighbour bits are shifts with the carry bit from the adjacent
// word of the same row.  The random word of cell i = y L + x at step t is
// word (i mod 4) of Philox block (c0 = i div 4, c1 = t); for lattice word k
// that is blocks c0 = 8k .. 8k+7.  A thread compares its 32 cells' words
// with the growth and lightning thresholds and packs the results into two
// words.  The kernel is bound by Philox's 32x32->64 multiplies, which GB300
// retires at under one warp instruction per SM-clock, so everything else
// stays off that pipe and the multiplies are trimmed: all blocks of one step
// share (t, rep, dp), hence round 1's product of counter word 2 and round
// 2's product of counter word 0 are computed once per step (18 instead of
// 20 wide multiplies per block, same words).  Lightning is rare: its four
// compares run only for blocks whose smallest word is below its threshold.
// The new state of 32 cells is then a few bitwise operations:
//   ignite = burning neighbour | lightning,
//   burning' = tree & ignite,
//   tree'    = (tree & ~ignite) | (empty & grow).
// The burning count of each step is a popcount, a warp reduction and a
// shared-memory atomic; counts are flushed to global memory every 64 steps
// (coalesced) from a double-buffered slot array.
#include "common.cuh"
#include "model.cuh"

namespace mrip {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Philox4x32-10 of counter (c0, t, rep, c3) for one step: the parts that do
// not depend on c0 are precomputed once per step (StepKey).
struct StepKey {
    uint32_t x0, x1;      // words 0 and 1 after round 1 (independent of c0)
    uint32_t p_hi, p_lo;  // round 2's product 0xD2511F53 * x0
};

__device__ __forceinline__ StepKey step_key(uint32_t t, uint32_t rep, const RoundKeys& rk) {
    StepKey s;
    const uint32_t h1 = __umulhi(0xCD9E8D57u, rep);
    s.x0 = h1 ^ t ^ rk.k0[0];
    s.x1 = 0xCD9E8D57u * rep;
    s.p_hi = __umulhi(0xD2511F53u, s.x0);
    s.p_lo = 0xD2511F53u * s.x0;
    return s;
}

__device__ __forceinline__ uint4 philox_step(uint32_t c0, uint32_t c3, const StepKey& sk,
                                             const RoundKeys& rk) {
    // round 1: only the product with c0 varies
    const uint32_t a_hi = __umulhi(0xD2511F53u, c0);
    const uint32_t a_lo = 0xD2511F53u * c0;
    const uint32_t w2 = a_hi ^ c3 ^ rk.k1[0];
    // round 2: the product with word 0 is sk.p
    const uint32_t b_hi = __umulhi(0xCD9E8D57u, w2);
    const uint32_t b_lo = 0xCD9E8D57u * w2;
    uint32_t x0 = b_hi ^ sk.x1 ^ rk.k0[1];
    uint32_t x1 = b_lo;
    uint32_t x2 = sk.p_hi ^ a_lo ^ rk.k1[1];
    uint32_t x3 = sk.p_lo;
#pragma unroll
    for (int r = 2; r < 10; ++r) philox_round(x0, x1, x2, x3, rk.k0[r], rk.k1[r]);
    return make_uint4(x0, x1, x2, x3);
}

// Threads per CTA for a lattice of W words per row.
template <int W>
constexpr int ff_threads() {
    return W == 1 ? 32 : W == 2 ? 64 : W == 4 ? 128 : W == 8 ? 256 : 512;
}

template <int W>
__global__ void __launch_bounds__(ff_threads<W>()) forest_fire_kernel(
    const double* __restrict__ dps, long long n_reps, long long rep0, int n_steps, uint32_t t_dens,
    const __grid_constant__ RoundKeys rk, const uint8_t* __restrict__ init,
    int32_t* __restrict__ counts, double* __restrict__ scalar, uint8_t* __restrict__ final_state) {
    constexpr int L = 32 * W;
    constexpr int NWORD = L * W;  // words per plane
    constexpr int TPB = ff_threads<W>();
    constexpr int NWARP = TPB / 32;
    extern __shared__ uint32_t lattice[];  // [buffer][plane T, B][NWORD]
    __shared__ int cnt[2][64];
    __shared__ long long red[NWARP];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const long long item = blockIdx.x;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const uint32_t t_grow = threshold32(dps[2 * dp]);
    const uint32_t t_light = threshold32(dps[2 * dp + 1]);
    const uint32_t c3 = stream_word(0u, dp);

    if (init) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(init + item * static_cast<long long>(L) * L);
        for (int k = threadIdx.x; k < NWORD; k += TPB) {
            uint32_t tw = 0, bw = 0;
            for (int r = 0; r < 8; ++r) {
                const uint32_t v = src[8 * k + r];
                for (int q = 0; q < 4; ++q) {
                    const uint32_t s = (v >> (8 * q)) & 0xFFu;
                    tw |= (s == 1u ? 1u : 0u) << (4 * r + q);
                    bw |= (s == 2u ? 1u : 0u) << (4 * r + q);
                }
            }
            lattice[k] = tw;
            lattice[NWORD + k] = bw;
        }
    } else {
        const uint32_t c3i = stream_word(1u, dp);
        for (int k = threadIdx.x; k < NWORD; k += TPB) {
            uint32_t tw = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 b = philox(8u * k + q, 0u, rep, c3i, rk);
                tw |= (b.x < t_dens) ? (1u << (4 * q)) : 0u;
                tw |= (b.y < t_dens) ? (1u << (4 * q + 1)) : 0u;
                tw |= (b.z < t_dens) ? (1u << (4 * q + 2)) : 0u;
                tw |= (b.w < t_dens) ? (1u << (4 * q + 3)) : 0u;
            }
            lattice[k] = tw;
            lattice[NWORD + k] = 0u;
        }
    }
    for (int i = threadIdx.x; i < 128; i += TPB) (&cnt[0][0])[i] = 0;
    __syncthreads();

    long long my_sum = 0;
    for (int t = 1; t <= n_steps; ++t) {
        const uint32_t* cur_t = lattice + ((t - 1) & 1) * 2 * NWORD;
        const uint32_t* cur_b = cur_t + NWORD;
        uint32_t* nxt_t = lattice + (t & 1) * 2 * NWORD;
        uint32_t* nxt_b = nxt_t + NWORD;
        int c = 0;
        const StepKey sk = step_key(static_cast<uint32_t>(t), rep, rk);
        for (int k = threadIdx.x; k < NWORD; k += TPB) {
            const int y = k / W;
            const int j = k - y * W;
            const uint32_t tw = cur_t[k];
            const uint32_t bw = cur_b[k];
            const uint32_t up = cur_b[((y + L - 1) & (L - 1)) * W + j];
            const uint32_t dn = cur_b[((y + 1) & (L - 1)) * W + j];
            const uint32_t bwest = cur_b[y * W + ((j + W - 1) & (W - 1))];
            const uint32_t beast = cur_b[y * W + ((j + 1) & (W - 1))];
            const uint32_t nb = up | dn | (bw << 1) | (bwest >> 31) | (bw >> 1) | (beast << 31);
            uint32_t g = 0, l = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint4 b = philox_step(8u * k + q, c3, sk, rk);
                g |= (b.x < t_grow) ? (1u << (4 * q)) : 0u;
                g |= (b.y < t_grow) ? (1u << (4 * q + 1)) : 0u;
                g |= (b.z < t_grow) ? (1u << (4 * q + 2)) : 0u;
                g |= (b.w < t_grow) ? (1u << (4 * q + 3)) : 0u;
                const uint32_t lowest = min(min(b.x, b.y), min(b.z, b.w));
                if (__builtin_expect(lowest < t_light, 0)) {
                    l |= (b.x < t_light) ? (1u << (4 * q)) : 0u;
                    l |= (b.y < t_light) ? (1u << (4 * q + 1)) : 0u;
                    l |= (b.z < t_light) ? (1u << (4 * q + 2)) : 0u;
                    l |= (b.w < t_light) ? (1u << (4 * q + 3)) : 0u;
                }
            }
            const uint32_t ignite = nb | l;
            const uint32_t nbw = tw & ignite;
            nxt_b[k] = nbw;
            nxt_t[k] = (tw & ~ignite) | (~(tw | bw) & g);
            c += __popc(nbw);
        }
        c = __reduce_add_sync(kFull, c);
        if (lane == 0) atomicAdd(&cnt[((t - 1) >> 6) & 1][(t - 1) & 63], c);
        __syncthreads();
        if ((t & 63) == 0 || t == n_steps) {
            const int chunk = (t - 1) >> 6;
            const int n_slot = t - chunk * 64;
            for (int s = threadIdx.x; s < n_slot; s += TPB) {
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
        const uint32_t* fin_t = lattice + (n_steps & 1) * 2 * NWORD;
        const uint32_t* fin_b = fin_t + NWORD;
        uint32_t* dst = reinterpret_cast<uint32_t*>(final_state + item * static_cast<long long>(L) * L);
        for (int k = threadIdx.x; k < NWORD; k += TPB) {
            const uint32_t tw = fin_t[k], bw = fin_b[k];
            for (int r = 0; r < 8; ++r) {
                uint32_t v = 0;
                for (int q = 0; q < 4; ++q) {
                    const int m = 4 * r + q;
                    const uint32_t s = ((tw >> m) & 1u) ? 1u : (((bw >> m) & 1u) ? 2u : 0u);
                    v |= s << (8 * q);
                }
                dst[8 * k + r] = v;
            }
        }
    }
}

template <int W>
mrip_status launch_ff(const double* dps, long long n_items, long long n_reps, long long rep0, int n_steps,
                      uint32_t t_dens, const RoundKeys& rk, const uint8_t* init, int32_t* counts,
                      double* scalar, uint8_t* final_state, cudaStream_t st) {
    const size_t smem = 2 * 2 * static_cast<size_t>(32 * W) * W * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(forest_fire_kernel<W>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return cuda_status(e, "forest fire: shared memory attribute");
    }
    forest_fire_kernel<W><<<static_cast<unsigned>(n_items), ff_threads<W>(), smem, st>>>(
        dps, n_reps, rep0, n_steps, t_dens, rk, init, counts, scalar, final_state);
    return MRIP_OK;
}

}  // namespace
}  // namespace mrip

using namespace mrip;

namespace mrip {
mrip_status forest_fire_launch(const double* d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps, int32_t L,
                               int32_t n_steps, double density, uint64_t seed, const uint8_t* d_init,
                               int32_t* d_counts, double* d_scalar, uint8_t* d_final, cudaStream_t st) {
    if (n_dp < 0 || n_reps < 0 || n_steps < 0 || rep0 < 0)
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: negative size");
    if (L < 32 || L > 512 || L % 32 != 0 || (L & (L - 1)) != 0)
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: L must be 32, 64, 128, 256 or 512");
    if (!(density >= 0.0 && density < 1.0))
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: density must be in [0, 1)");
    if (n_dp >= (1 << 24) || rep0 + n_reps > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: n_dp < 2^24 and replication indices < 2^32");
    const long long n_items = static_cast<long long>(n_dp) * n_reps;
    if (n_items == 0) return MRIP_OK;
    if (n_items > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: too many replications");
    if (!d_dps) return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: null design points");
    if ((d_init && (reinterpret_cast<uintptr_t>(d_init) & 15u)) ||
        (d_final && (reinterpret_cast<uintptr_t>(d_final) & 15u)))
        return fail(MRIP_EINVAL, "mrip_forest_fire_simulate: state buffers need 16-byte alignment");
    const RoundKeys rk = expand_key(seed);
    const uint32_t t_dens = threshold32(density);
    mrip_status rc = MRIP_OK;
    switch (L) {
        case 32: rc = launch_ff<1>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 64: rc = launch_ff<2>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 128: rc = launch_ff<4>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 256: rc = launch_ff<8>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
        case 512: rc = launch_ff<16>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, d_init, d_counts, d_scalar, d_final, st); break;
    }
    if (rc != MRIP_OK) return rc;
    return launch_status("mrip_forest_fire_simulate");
}
}  // namespace mrip

extern "C" mrip_status mrip_forest_fire_simulate(const double* d_dps, int32_t n_dp, int64_t n_reps,
                                                 int32_t L, int32_t n_steps, double density,
                                                 uint64_t seed, const uint8_t* d_init,
                                                 int32_t* d_counts, double* d_scalar,
                                                 uint8_t* d_final, void* stream) {
    return forest_fire_launch(d_dps, n_dp, 0, n_reps, L, n_steps, density, seed, d_init, d_counts,
                              d_scalar, d_final, static_cast<cudaStream_t>(stream));
}
