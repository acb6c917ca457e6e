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
// (coalesced, 16-byte stores where aligned) from a double-buffered slot array.
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
    uint32_t h1;
    mul_wide_u32(0xCD9E8D57u, rep, h1, s.x1);
    s.x0 = h1 ^ t ^ rk.k0[0];
    mul_wide_u32(0xD2511F53u, s.x0, s.p_hi, s.p_lo);
    return s;
}

// prod = 0xD2511F53 * c0 as a 64-bit product (round 1's only varying product);
// the 8 blocks of one lattice word have c0 = 8k + q, so the caller forms it
// as 0xD2511F53 * 8k plus a constant: one 64-bit add instead of a wide
// multiply for 7 of every 8 blocks.
__device__ __forceinline__ uint4 philox_step(unsigned long long prod, uint32_t c3, const StepKey& sk,
                                             const RoundKeys& rk) {
    const uint32_t a_hi = static_cast<uint32_t>(prod >> 32);
    const uint32_t a_lo = static_cast<uint32_t>(prod);
    const uint32_t w2 = a_hi ^ c3 ^ rk.k1[0];
    // round 2: the product with word 0 is sk.p
    uint32_t b_hi, b_lo;
    mul_wide_u32(0xCD9E8D57u, w2, b_hi, b_lo);
    uint32_t x0 = b_hi ^ sk.x1 ^ rk.k0[1];
    uint32_t x1 = b_lo;
    uint32_t x2 = sk.p_hi ^ a_lo ^ rk.k1[1];
    uint32_t x3 = sk.p_lo;
#pragma unroll
    for (int r = 2; r < 10; ++r) philox_round(x0, x1, x2, x3, rk.k0[r], rk.k1[r]);
    return make_uint4(x0, x1, x2, x3);
}

// bits |= bit if w < t, as a compare and a predicated OR (integer ALU, not the
// multiply pipe that Philox saturates).
__device__ __forceinline__ void or_if_below(uint32_t& bits, uint32_t w, uint32_t t, uint32_t bit) {
    asm("{\n .reg .pred p;\n setp.lt.u32 p, %1, %2;\n @p or.b32 %0, %0, %3;\n}\n"
        : "+r"(bits)
        : "r"(w), "r"(t), "r"(bit));
}

// Flush the n_slot (<= 64) burning counts of one 64-step chunk from the
// shared slot array to dst (skipped when null) and add them to my_sum,
// clearing the slots when asked.  Where dst is 16-byte aligned and n_slot a
// multiple of 4 (every chunk when n_steps is), a thread moves four counts
// with one 16-byte store.
template <int TPB>
__device__ __forceinline__ void ff_flush(int* slot, int n_slot, int32_t* dst, bool clear, long long& my_sum) {
    if (dst && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 && (n_slot & 3) == 0) {
        for (int s4 = threadIdx.x; s4 < (n_slot >> 2); s4 += TPB) {
            int4* src = reinterpret_cast<int4*>(slot) + s4;
            const int4 v = *src;
            if (clear) *src = make_int4(0, 0, 0, 0);
            my_sum += static_cast<long long>(v.x) + v.y + v.z + v.w;
            reinterpret_cast<int4*>(dst)[s4] = v;
        }
    } else {
        for (int s = threadIdx.x; s < n_slot; s += TPB) {
            const int v = slot[s];
            if (clear) slot[s] = 0;
            my_sum += v;
            if (dst) dst[s] = v;
        }
    }
}

// Threads per CTA for a lattice of W words per row.
template <int W>
constexpr int ff_threads() {
    return W == 1 ? 32 : W == 2 ? 64 : W == 4 ? 128 : W == 8 ? 256 : 512;
}

// Initial state into buffer 0 (planes T, B): from `init` (one byte per cell,
// 0 empty, 1 tree, 2 burning) or from tag 1 (tree iff word < t_dens).
template <int W>
__device__ void ff_load_initial(uint32_t* lattice, const uint8_t* __restrict__ init, long long item,
                                uint32_t t_dens, uint32_t rep, uint32_t dp, const RoundKeys& rk) {
    constexpr int L = 32 * W;
    constexpr int NWORD = L * W;
    constexpr int TPB = ff_threads<W>();
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
}

// Planes (fin_t, fin_b) back to one byte per cell.
template <int W>
__device__ void ff_store_final(const uint32_t* fin_t, const uint32_t* fin_b, uint8_t* __restrict__ final_state,
                               long long item) {
    constexpr int L = 32 * W;
    constexpr int NWORD = L * W;
    constexpr int TPB = ff_threads<W>();
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

// Per-replication scalar: the mean burning fraction (block reduction of the
// threads' step sums).
template <int NWARP>
__device__ void ff_store_scalar(long long my_sum, long long* red, double* scalar, long long item, int n_steps,
                                int L) {
    long long s = my_sum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(kFull, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < NWARP; ++w) tot += red[w];
        scalar[item] = static_cast<double>(tot) / (static_cast<double>(n_steps) * static_cast<double>(L) * L);
    }
}

// Register budget: a word's eight Philox blocks are independent, and the
// more registers ptxas may use the more of them it interleaves.  256-thread
// CTAs (L = 256) are held to three per SM (78 registers: 4.2 % faster than
// five CTAs at 48); the other widths take the compiler's own maximum (L = 128:
// 110 registers, four CTAs per SM, 5 % faster than nine at 56).
template <int W>
constexpr int ff_min_blocks() {
    return W == 8 ? 3 : 1;
}

template <int W>
__global__ void __launch_bounds__(ff_threads<W>(), ff_min_blocks<W>()) forest_fire_kernel(
    const double* __restrict__ dps, long long n_reps, long long rep0, int n_steps, uint32_t t_dens,
    const __grid_constant__ RoundKeys rk, const uint8_t* __restrict__ init,
    int32_t* __restrict__ counts, double* __restrict__ scalar, uint8_t* __restrict__ final_state) {
    constexpr int L = 32 * W;
    constexpr int NWORD = L * W;  // words per plane
    constexpr int TPB = ff_threads<W>();
    constexpr int NWARP = TPB / 32;
    extern __shared__ uint32_t lattice[];  // [buffer][plane T, B][NWORD]
    __shared__ __align__(16) int cnt[2][64];
    __shared__ long long red[NWARP];

    const int lane = threadIdx.x & 31;
    const long long item = blockIdx.x;
    if (!MRIP_CHECK(4u * NWORD * sizeof(uint32_t) <= dynamic_smem_bytes(), 101, NWORD)) return;  // CTA-uniform
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const uint32_t t_grow = threshold32(dps[2 * dp]);
    const uint32_t t_light = threshold32(dps[2 * dp + 1]);
    const uint32_t c3 = stream_word(0u, dp);

    ff_load_initial<W>(lattice, init, item, t_dens, rep, dp, rk);
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
            uint32_t up, dn, bwest, beast;
            if constexpr (W >= 8) {  // the same words, indexed from k (rows are W words; L W a power of two)
                up = cur_b[(k + NWORD - W) & (NWORD - 1)];
                dn = cur_b[(k + W) & (NWORD - 1)];
                bwest = cur_b[(k & ~(W - 1)) | ((j + W - 1) & (W - 1))];
                beast = cur_b[(k & ~(W - 1)) | ((j + 1) & (W - 1))];
            } else {
                up = cur_b[((y + L - 1) & (L - 1)) * W + j];
                dn = cur_b[((y + 1) & (L - 1)) * W + j];
                bwest = cur_b[y * W + ((j + W - 1) & (W - 1))];
                beast = cur_b[y * W + ((j + 1) & (W - 1))];
            }
            const uint32_t nb = up | dn | (bw << 1) | (bwest >> 31) | (bw >> 1) | (beast << 31);
            uint32_t g = 0, l = 0;
            const unsigned long long base = 0xD2511F53ull * (8u * static_cast<uint32_t>(k));
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                unsigned long long pq = base + 0xD2511F53ull * q;
                if constexpr (W >= 8) {  // the same sum as an explicit carry chain of two 32-bit adds
                    const unsigned long long cq = 0xD2511F53ull * q;
                    uint32_t plo, phi;
                    asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, %5;"
                        : "=r"(plo), "=r"(phi)
                        : "r"(static_cast<uint32_t>(base)), "r"(static_cast<uint32_t>(base >> 32)),
                          "r"(static_cast<uint32_t>(cq)), "r"(static_cast<uint32_t>(cq >> 32)));
                    pq = (static_cast<unsigned long long>(phi) << 32) | plo;
                }
                const uint4 b = philox_step(pq, c3, sk, rk);
                or_if_below(g, b.x, t_grow, 1u << (4 * q));
                or_if_below(g, b.y, t_grow, 1u << (4 * q + 1));
                or_if_below(g, b.z, t_grow, 1u << (4 * q + 2));
                or_if_below(g, b.w, t_grow, 1u << (4 * q + 3));
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
            if (MRIP_CHECK(n_slot >= 1 && n_slot <= 64 && chunk * 64 + n_slot <= n_steps, 102, t))
                ff_flush<TPB>(cnt[chunk & 1], n_slot, counts ? counts + item * n_steps + chunk * 64 : nullptr,
                              true, my_sum);
        }
    }

    if (scalar) ff_store_scalar<NWARP>(my_sum, red, scalar, item, n_steps, L);
    if (final_state) {
        const uint32_t* fin_t = lattice + (n_steps & 1) * 2 * NWORD;
        ff_store_final<W>(fin_t, fin_t + NWORD, final_state, item);
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

// ---------------------------------------------------------------------------
// Skip-sampled variant: the same automaton, but each step's growth and
// lightning events are drawn as gaps between successes over the cells
// i = 0 .. L^2 - 1 (gap j: K_j = floor(E_j / mu), mu = -log1p(-p), E_j the
// exponential variate of words 2(j mod 2), 2(j mod 2)+1 of block
// (c0 = j div 2, c1 = t) under tag 5 (growth) or 6 (lightning)).  Work per
// step is p L^2 variates instead of L^2 words.
//
// A warp draws 64 gaps per round (lane l takes one block, i.e. two gaps), a
// warp scan of the lanes' (2 + K_2l + K_2l+1) places the events, and each
// event sets its bit in an event plane in shared memory (atomicOr).  All
// warps but the last share the growth set (a round's warp totals meet in
// shared memory), the last warp draws the lightning set (one warp draws
// both, in turn, when the CTA has one); then all threads update the lattice
// word-parallel:
//   ignite = burning neighbour | lightning event,
//   burning' = tree & ignite,
//   tree'    = (tree & ~ignite) | (empty & growth event),
// clearing the event words they read.  Event planes are double-buffered by
// step parity for L <= 256, so one barrier per step (between the draw and
// the update) suffices; L = 512 keeps one buffer and adds a second barrier.
// ---------------------------------------------------------------------------
// K = floor(E / mu) without the FP64 pipe: E = y57 2^-57 (the fixed-point
// log), 2^-57 / mu = dm 2^-shift with dm a 64-bit integer (dm = the double's
// significand scaled to [2^63, 2^64)), so K = (y57 dm) >> shift on the
// 128-bit product, saturated at n_cells.  It differs from floor of the FP64
// quotient only when that quotient is within a few ulps of an integer.
struct GapScale {
    unsigned long long dm;
    int shift;  // >= 0; >= 128 means every gap is 0 (p >= 1)
};

__device__ __forceinline__ GapScale gap_scale(double p) {
    GapScale g{0ull, 128};
    if (p >= 1.0) return g;
    const double d = 0x1p-57 / -log1p(-p);  // p in (0, 1)
    if (!(d < 0x1p64)) {                     // mu below 2^-121: every positive E saturates
        g.dm = ~0ull;
        g.shift = 0;
        return g;
    }
    int ex;
    const double mant = frexp(d, &ex);  // d = mant 2^ex, mant in [0.5, 1), ex <= 64
    g.dm = static_cast<unsigned long long>(ldexp(mant, 64));
    g.shift = 64 - ex;  // >= 128: d < 2^-64, so y57 d < 1 and every gap is 0
    return g;
}

__device__ __forceinline__ int gap_cells(unsigned long long y57, const GapScale& g, int n_cells) {
    if (g.shift >= 128) return 0;
    const unsigned long long hi = __umul64hi(y57, g.dm);
    unsigned long long k;
    if (g.shift >= 64) {
        k = hi >> (g.shift - 64);
    } else {
        const unsigned long long lo = y57 * g.dm;
        if (g.shift == 0)
            k = hi ? ~0ull : lo;
        else
            k = (hi >> g.shift) ? ~0ull : ((hi << (64 - g.shift)) | (lo >> g.shift));
    }
    return k >= static_cast<unsigned long long>(n_cells) ? n_cells : static_cast<int>(k);
}

// Smallest 53-bit u (as an integer) for which the first gap of a set of
// probability p passes n cells: u >= 1 - (1 - p)^n, i.e. -log(1 - u) >= n mu.
// At least 1 (u = 0 gives the gap 0) and at most 2^53 (never, for p >= 1).
// At the boundary this and the gap's own floor can disagree only where
// E / mu is within a few ulps of n, which the oracle reports as a near tie.
__device__ __forceinline__ unsigned long long first_gap_none(double p, int n) {
    if (p >= 1.0) return 1ull << 53;
    const double q = -expm1(static_cast<double>(n) * log1p(-p));  // 1 - (1 - p)^n
    const double t = ceil(q * 0x1p53);
    if (!(t >= 1.0)) return 1ull;
    return t >= 0x1p53 ? (1ull << 53) : static_cast<unsigned long long>(t);
}

__device__ __forceinline__ unsigned long long expo_q57(uint32_t lo, uint32_t hi, const LogTable& tab) {
    const unsigned long long bits = (static_cast<unsigned long long>(hi) << 32) | lo;
    return neg_log_q57((1ULL << 53) - (bits >> 11), tab);
}

// Call only for p > 0.
__device__ void draw_events(uint32_t* __restrict__ ev, int n_cells, const GapScale& gs, uint32_t t, uint32_t rep,
                            uint32_t c3, const RoundKeys& rk, const LogTable& tab) {
    const int lane = threadIdx.x & 31;
    int pos = -1;  // last event so far (warp-uniform)
    for (uint32_t r = 0; pos + 1 < n_cells; ++r) {
        const uint4 b = philox(32u * r + static_cast<uint32_t>(lane), t, rep, c3, rk);
        const int k0 = gap_cells(expo_q57(b.x, b.y, tab), gs, n_cells);
        const int k1 = gap_cells(expo_q57(b.z, b.w, tab), gs, n_cells);
        const int span = 2 + k0 + k1;
        int incl = span;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += v;
        }
        const int p0 = pos + (incl - span) + 1 + k0;
        const int p1 = p0 + 1 + k1;
        if (p0 < n_cells && MRIP_CHECK(p0 >= 0, 103, p0)) atomicOr(ev + (p0 >> 5), 1u << (p0 & 31));
        if (p1 < n_cells && MRIP_CHECK(p1 > p0, 104, p1)) atomicOr(ev + (p1 >> 5), 1u << (p1 & 31));
        pos += __shfl_sync(kFull, incl, 31);
    }
}

// All warps draw: warps 0 .. NG-1 share the growth gaps (round r, warp w
// takes blocks (r NG + w) 32 + lane), warp NG the lightning gaps (blocks
// 32 r + lane) while its set is unfinished.  Each warp scans its 64 gaps; the
// warp totals meet in shared memory (double-buffered by round parity, one
// barrier per round) and give every warp its offset and every thread the new
// last position, so all threads agree on when each set ends.
template <int NWARP>
__device__ void draw_step_events(uint32_t* __restrict__ ev_g, uint32_t* __restrict__ ev_h, int n_cells,
                                 bool grow_on, bool light_on, const GapScale& gsg, const GapScale& gsh,
                                 unsigned long long light_none, uint32_t t, uint32_t rep, uint32_t c3g,
                                 uint32_t c3h, const RoundKeys& rk, const LogTable& tab, int (*tot)[NWARP]) {
    static_assert(NWARP >= 2, "one-warp CTAs draw with draw_events");
    constexpr int NG = NWARP - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int pos_g = -1, pos_h = -1;
    for (int r = 0; grow_on || light_on; ++r) {
        int* tt = tot[r & 1];
        const bool mine = (warp < NG) ? grow_on : light_on;
        int k0 = 0, k1 = 0, span = 0, incl = 0;
        if (mine) {
            const bool g = warp < NG;
            const uint32_t c0 = static_cast<uint32_t>(g ? (r * NG + warp) * 32 + lane : r * 32 + lane);
            const uint4 b = philox(c0, t, rep, g ? c3g : c3h, rk);
            // The lightning set's first gap passes the lattice (no event this
            // step) iff u >= 1 - (1 - p)^(L^2): one compare of gap 0's 53 bits
            // instead of the logs and the scan, most steps.
            bool none = false;
            if (!g && r == 0) {
                const unsigned long long bits = ((static_cast<unsigned long long>(b.y) << 32) | b.x) >> 11;
                none = __shfl_sync(kFull, bits >= light_none ? 1 : 0, 0) != 0;
            }
            if (none) {
                k0 = n_cells;
                k1 = n_cells;
                incl = n_cells + 1;  // the set ends; no event bits
                if (lane == 31) tt[warp] = incl;
            } else {
                const GapScale& gs = g ? gsg : gsh;
                k0 = gap_cells(expo_q57(b.x, b.y, tab), gs, n_cells);
                k1 = gap_cells(expo_q57(b.z, b.w, tab), gs, n_cells);
                span = 2 + k0 + k1;
                incl = span;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int v = __shfl_up_sync(kFull, incl, off);
                    if (lane >= off) incl += v;
                }
                if (lane == 31) tt[warp] = incl;
            }
        }
        __syncthreads();
        int before = 0, total_g = 0;
        if (grow_on) {
            for (int w = 0; w < NG; ++w) {
                const int v = tt[w];
                before += (w < warp) ? v : 0;
                total_g += v;
            }
        }
        if (mine) {
            const bool g = warp < NG;
            const int p0 = (g ? pos_g + before : pos_h) + (incl - span) + 1 + k0;
            const int p1 = p0 + 1 + k1;
            uint32_t* ev = g ? ev_g : ev_h;
            if (p0 < n_cells && MRIP_CHECK(p0 >= 0, 105, p0)) atomicOr(ev + (p0 >> 5), 1u << (p0 & 31));
            if (p1 < n_cells && MRIP_CHECK(p1 > p0, 106, p1)) atomicOr(ev + (p1 >> 5), 1u << (p1 & 31));
        }
        if (grow_on) {
            pos_g += total_g;
            grow_on = pos_g + 1 < n_cells;
        }
        if (light_on) {
            pos_h += tt[NG];
            light_on = pos_h + 1 < n_cells;
        }
    }
}

template <int W>
constexpr int ev_buffers() {
    return W <= 8 ? 2 : 1;
}

template <int W>
__global__ void __launch_bounds__(ff_threads<W>()) forest_fire_skip_kernel(
    const double* __restrict__ dps, long long n_reps, long long rep0, int n_steps, uint32_t t_dens,
    const __grid_constant__ RoundKeys rk, LogTable tab, const uint8_t* __restrict__ init,
    int32_t* __restrict__ counts, double* __restrict__ scalar, uint8_t* __restrict__ final_state) {
    constexpr int L = 32 * W;
    constexpr int NWORD = L * W;
    constexpr int TPB = ff_threads<W>();
    constexpr int NWARP = TPB / 32;
    constexpr int NEV = ev_buffers<W>();
    extern __shared__ uint32_t lattice[];  // [buffer][plane T, B][NWORD], then events [NEV][G, H][NWORD]
    uint32_t* events = lattice + 4 * NWORD;
    __shared__ __align__(16) int cnt[2][64];
    __shared__ long long red[NWARP];
    __shared__ int tot[2][NWARP];

    const int lane = threadIdx.x & 31;
    const long long item = blockIdx.x;
    if (!MRIP_CHECK((4u + 2u * NEV) * NWORD * sizeof(uint32_t) <= dynamic_smem_bytes(), 107, NWORD)) return;
    const uint32_t dp = static_cast<uint32_t>(item / n_reps);
    const uint32_t rep = static_cast<uint32_t>(rep0 + item % n_reps);
    const double p_grow = dps[2 * dp], p_light = dps[2 * dp + 1];
    const bool any_grow = p_grow > 0.0, any_light = p_light > 0.0;
    const GapScale gs_grow = any_grow ? gap_scale(p_grow) : GapScale{0ull, 128};
    const GapScale gs_light = any_light ? gap_scale(p_light) : GapScale{0ull, 128};
    const unsigned long long light_none = any_light ? first_gap_none(p_light, L * L) : (1ull << 53);
    const uint32_t c3_grow = stream_word(5u, dp), c3_light = stream_word(6u, dp);

    ff_load_initial<W>(lattice, init, item, t_dens, rep, dp, rk);
    for (int k = threadIdx.x; k < NEV * 2 * NWORD; k += TPB) events[k] = 0u;
    for (int i = threadIdx.x; i < 128; i += TPB) (&cnt[0][0])[i] = 0;
    __syncthreads();

    long long my_sum = 0;
    for (int t = 1; t <= n_steps; ++t) {
        uint32_t* ev_g = events + ((NEV == 2) ? (t & 1) : 0) * 2 * NWORD;
        uint32_t* ev_h = ev_g + NWORD;
        if constexpr (NWARP == 1) {
            if (any_grow) draw_events(ev_g, L * L, gs_grow, t, rep, c3_grow, rk, tab);
            if (any_light) draw_events(ev_h, L * L, gs_light, t, rep, c3_light, rk, tab);
        } else {
            draw_step_events<NWARP>(ev_g, ev_h, L * L, any_grow, any_light, gs_grow, gs_light, light_none, t, rep,
                                    c3_grow, c3_light, rk, tab, tot);
        }
        __syncthreads();
        // counts of the steps before t are complete: flush a finished chunk
        if (t > 1 && ((t - 1) & 63) == 0) {
            const int chunk = (t - 2) >> 6;
            if (MRIP_CHECK(chunk * 64 + 64 <= n_steps, 108, t))
                ff_flush<TPB>(cnt[chunk & 1], 64, counts ? counts + item * n_steps + chunk * 64 : nullptr, true,
                              my_sum);
        }
        const uint32_t* cur_t = lattice + ((t - 1) & 1) * 2 * NWORD;
        const uint32_t* cur_b = cur_t + NWORD;
        uint32_t* nxt_t = lattice + (t & 1) * 2 * NWORD;
        uint32_t* nxt_b = nxt_t + NWORD;
        int c = 0;
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
            const uint32_t g = ev_g[k];
            const uint32_t h = ev_h[k];
            ev_g[k] = 0u;
            ev_h[k] = 0u;
            const uint32_t ignite = nb | h;
            const uint32_t nbw = tw & ignite;
            nxt_b[k] = nbw;
            nxt_t[k] = (tw & ~ignite) | (~(tw | bw) & g);
            c += __popc(nbw);
        }
        c = __reduce_add_sync(kFull, c);
        if (lane == 0) atomicAdd(&cnt[((t - 1) >> 6) & 1][(t - 1) & 63], c);
        if (NEV == 1) __syncthreads();
    }
    __syncthreads();
    if (n_steps > 0) {
        const int chunk = (n_steps - 1) >> 6;
        const int n_slot = n_steps - chunk * 64;
        ff_flush<TPB>(cnt[chunk & 1], n_slot, counts ? counts + item * n_steps + chunk * 64 : nullptr, false,
                      my_sum);
    }
    if (scalar) ff_store_scalar<NWARP>(my_sum, red, scalar, item, n_steps, L);
    if (final_state) {
        const uint32_t* fin_t = lattice + (n_steps & 1) * 2 * NWORD;
        ff_store_final<W>(fin_t, fin_t + NWORD, final_state, item);
    }
}

template <int W>
mrip_status launch_ff_skip(const double* dps, long long n_items, long long n_reps, long long rep0, int n_steps,
                           uint32_t t_dens, const RoundKeys& rk, const LogTable& tab, const uint8_t* init,
                           int32_t* counts, double* scalar, uint8_t* final_state, cudaStream_t st) {
    const size_t nword = static_cast<size_t>(32 * W) * W;
    const size_t smem = (4 + 2 * ev_buffers<W>()) * nword * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(forest_fire_skip_kernel<W>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return cuda_status(e, "forest fire (skip): shared memory attribute");
    }
    forest_fire_skip_kernel<W><<<static_cast<unsigned>(n_items), ff_threads<W>(), smem, st>>>(
        dps, n_reps, rep0, n_steps, t_dens, rk, tab, init, counts, scalar, final_state);
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

extern "C" mrip_status mrip_forest_fire_skip_simulate(const double* d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                                                      int32_t L, int32_t n_steps, double density,
                                                      uint64_t seed, const uint8_t* d_init,
                                                      int32_t* d_counts, double* d_scalar,
                                                      uint8_t* d_final, void* stream) {
    if (n_dp < 0 || n_reps < 0 || n_steps < 0 || rep0 < 0)
        return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: negative size");
    if (L < 32 || L > 512 || L % 32 != 0 || (L & (L - 1)) != 0)
        return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: L must be 32, 64, 128, 256 or 512");
    if (!(density >= 0.0 && density < 1.0))
        return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: density must be in [0, 1)");
    if (n_dp >= (1 << 24) || rep0 + n_reps > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: n_dp < 2^24 and replication indices < 2^32");
    const long long n_items = static_cast<long long>(n_dp) * n_reps;
    if (n_items == 0) return MRIP_OK;
    if (n_items > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: too many replications");
    if (!d_dps) return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: null design points");
    if ((d_init && (reinterpret_cast<uintptr_t>(d_init) & 15u)) ||
        (d_final && (reinterpret_cast<uintptr_t>(d_final) & 15u)))
        return fail(MRIP_EINVAL, "mrip_forest_fire_skip_simulate: state buffers need 16-byte alignment");
    LogTable tab;
    mrip_status rc = log_table(&tab);
    if (rc != MRIP_OK) return rc;
    const RoundKeys rk = expand_key(seed);
    const uint32_t t_dens = threshold32(density);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (L) {
        case 32: rc = launch_ff_skip<1>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, tab, d_init, d_counts, d_scalar, d_final, st); break;
        case 64: rc = launch_ff_skip<2>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, tab, d_init, d_counts, d_scalar, d_final, st); break;
        case 128: rc = launch_ff_skip<4>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, tab, d_init, d_counts, d_scalar, d_final, st); break;
        case 256: rc = launch_ff_skip<8>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, tab, d_init, d_counts, d_scalar, d_final, st); break;
        case 512: rc = launch_ff_skip<16>(d_dps, n_items, n_reps, rep0, n_steps, t_dens, rk, tab, d_init, d_counts, d_scalar, d_final, st); break;
    }
    if (rc != MRIP_OK) return rc;
    return launch_status("mrip_forest_fire_skip_simulate");
}

extern "C" mrip_status mrip_forest_fire_simulate(const double* d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                                                 int32_t L, int32_t n_steps, double density,
                                                 uint64_t seed, const uint8_t* d_init,
                                                 int32_t* d_counts, double* d_scalar,
                                                 uint8_t* d_final, void* stream) {
    return forest_fire_launch(d_dps, n_dp, rep0, n_reps, L, n_steps, density, seed, d_init, d_counts,
                              d_scalar, d_final, static_cast<cudaStream_t>(stream));
}

MRIP_DEBUG_UNIT(forest_fire)
