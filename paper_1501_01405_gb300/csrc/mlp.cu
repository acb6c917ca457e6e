// Learned control variate, network stages: a d_in -> 64 -> 64 -> 1 ReLU
// network (d_in = 8 for the tandem queue, 6 for the forest fire) trained on
// replications the engine generates, used as a control variate.  The paper
// has no learned component; its estimator (the replication mean, Section 1)
// stays the fallback and the yardstick the control variate is checked against.
//
// Arithmetic: parameters are FP32 masters; every matmul takes BF16 operands
// (round to nearest even from FP32) and accumulates in FP32:
//   forward  z1 = x~ W1~^T + b1, h1 = relu(z1); z2 = h1~ W2~^T + b2, h2 = relu(z2);
//            yhat = h2~ . W3~ + b3
//   backward dyhat = 2 (yhat - y) / B; dW3 = sum dyhat h2~; dz2 = dyhat W3~ [z2 > 0];
//            dW2 = dz2~^T h1~; dz1 = (dz2~ W2~) [z1 > 0]; dW1 = dz1~^T x~;
//            bias gradients are FP32 sums of the unrounded dz.
// The matrices are 64 wide, so the passes are latency- not throughput-bound:
// a CTA takes a tile of 32 samples with the BF16-rounded weights staged in
// shared memory (both orientations of W2, so every inner product reads
// consecutive words), and writes its per-parameter partial sums; a second
// kernel adds the partials of all CTAs in a fixed order (deterministic) and,
// during training, applies Adam in the same pass.  These serve the stage
// entry points; the control-variate driver trains in one launch on the
// tensor cores (mlp_train_tc_kernel).
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "model.cuh"
#include "tc.cuh"

namespace mrip {

namespace {

constexpr int H = 64;
constexpr int kTile = 32;        // samples per CTA
constexpr int kGradThreads = 256;
constexpr int kMaxIn = 8;

__host__ __device__ constexpr long long off_b1(int d) { return static_cast<long long>(H) * d; }
__host__ __device__ constexpr long long off_w2(int d) { return off_b1(d) + H; }
__host__ __device__ constexpr long long off_b2(int d) { return off_w2(d) + H * H; }
__host__ __device__ constexpr long long off_w3(int d) { return off_b2(d) + H; }
__host__ __device__ constexpr long long off_b3(int d) { return off_w3(d) + H; }
__host__ __device__ constexpr long long n_params(int d) { return off_b3(d) + 1; }

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// W1 element (unit u, input k); W1 is stored row-major [u][k].
__device__ __forceinline__ float theta_w1(const float* theta, int d_in, int u, int k) { return theta[u * d_in + k]; }

// He-uniform weights from stream tag 3: element e of (W1, W2, W3) reads words
// 2(e mod 2), 2(e mod 2)+1 of block (c0 = e div 2, c1 = 0, rep 0, dp 0).
__global__ void mlp_init_kernel(int d_in, const __grid_constant__ RoundKeys rk, float* theta) {
    const long long n_w = static_cast<long long>(H) * d_in + H * H + H;
    const long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (e < n_w) {
        const uint4 b = philox(static_cast<uint32_t>(e >> 1), 0u, 0u, stream_word(3u, 0u), rk);
        const double u = (e & 1) ? u53(b.z, b.w) : u53(b.x, b.y);
        long long dst;
        double fan;
        if (e < static_cast<long long>(H) * d_in) {
            dst = e;
            fan = d_in;
        } else if (e < static_cast<long long>(H) * d_in + H * H) {
            dst = off_w2(d_in) + (e - static_cast<long long>(H) * d_in);
            fan = H;
        } else {
            dst = off_w3(d_in) + (e - static_cast<long long>(H) * d_in - H * H);
            fan = H;
        }
        theta[dst] = static_cast<float>((2.0 * u - 1.0) * sqrt(6.0 / fan));
    }
    // biases
    if (e < H) {
        theta[off_b1(d_in) + e] = 0.0f;
        theta[off_b2(d_in) + e] = 0.0f;
    }
    if (e == 0) theta[off_b3(d_in)] = 0.0f;
}

// Which sample sits at batch position i.
struct SampleMap {
    const int64_t* idx;   // explicit indices, or null
    unsigned long long a, b, n;  // affine permutation (a i + b) mod n when n > 0
    long long off;        // batch offset within the epoch
};

__device__ __forceinline__ long long sample_of(const SampleMap& m, long long i) {
    if (m.idx) return m.idx[i];
    const unsigned long long k = static_cast<unsigned long long>(m.off + i);
    if (m.n > 0) return static_cast<long long>((m.a * k + m.b) % m.n);
    return static_cast<long long>(k);
}

constexpr int HP = H + 4;

struct GradSmem {
    alignas(16) float w1t[kMaxIn][H];  // [k][u]
    alignas(16) float w2t[H][H];       // [u][v]
    alignas(16) float w2[H][H];        // [v][u]
    float w3[H], b1[H], b2[H];
    float b3;
    float xt[kTile][kMaxIn];
    // per-sample rows padded to HP words: samples 4 apart in a warp sit in
    // different banks, and rows stay 16-byte aligned for float4 loads
    alignas(16) float h1[kTile][HP];
    alignas(16) float h1t[kTile][HP];
    alignas(16) float h2[kTile][HP];
    alignas(16) float h2t[kTile][HP];
    alignas(16) float dz2[kTile][HP];
    alignas(16) float dz2t[kTile][HP];
    alignas(16) float dz1[kTile][HP];
    float dy[kTile];
    float ys[kTile];
};

// Stage the BF16-rounded weights (and FP32 biases) of theta (global or
// shared) into S.
__device__ void stage_weights(GradSmem& S, const float* theta, int d_in) {
    const int t = threadIdx.x;
    for (int i = t; i < H * d_in; i += kGradThreads) {
        const int u = i / d_in, k = i - u * d_in;
        S.w1t[k][u] = bf(theta[i]);
    }
    for (int i = t; i < H * H; i += kGradThreads) {
        const int v = i / H, u = i - v * H;
        const float w = bf(theta[off_w2(d_in) + i]);
        S.w2[v][u] = w;
        S.w2t[u][v] = w;
    }
    for (int i = t; i < H; i += kGradThreads) {
        S.w3[i] = bf(theta[off_w3(d_in) + i]);
        S.b1[i] = theta[off_b1(d_in) + i];
        S.b2[i] = theta[off_b2(d_in) + i];
    }
    if (t == 0) S.b3 = theta[off_b3(d_in)];
}

// Stage samples at batch positions pos0 .. pos0 + n_valid - 1 (n_valid <= kTile;
// the rest of the tile is zero and contributes nothing).
__device__ void stage_tile(GradSmem& S, int d_in, const float* __restrict__ X, long long n_total,
                           const float* __restrict__ Y, const SampleMap& map, long long pos0, int n_valid) {
    const int t = threadIdx.x;
    for (int i = t; i < kTile * kMaxIn; i += kGradThreads) {
        const int s = i / kMaxIn, k = i - s * kMaxIn;
        float v = 0.0f;
        if (s < n_valid && k < d_in) {
            const long long smp = sample_of(map, pos0 + s);
            if (MRIP_CHECK(smp >= 0 && smp < n_total, 403, smp)) v = bf(X[k * n_total + smp]);
        }
        S.xt[s][k] = v;
    }
    if (t < kTile) {
        float y = 0.0f;
        if (t < n_valid) {
            const long long smp = sample_of(map, pos0 + t);
            if (MRIP_CHECK(smp >= 0 && smp < n_total, 404, smp)) y = Y[smp];
        }
        S.ys[t] = y;
    }
}

// Forward and backward passes of the staged tile (batch size B_scale for the
// loss gradient 2 r / B).  Leaves h1, h2, dz1, dz2, dy and the squared
// residuals (in ys) in S.
__device__ void tile_passes(GradSmem& S, int d_in, int n_valid, float B_scale) {
    const int t = threadIdx.x;
    const int s = t >> 3;  // sample of this thread for the per-sample passes
    const int g = t & 7;   // its slice of units: g, g + 8, ..., g + 56
    // layer 1
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int u = g + 8 * i;
        float acc = 0.0f;
        for (int k = 0; k < d_in; ++k) acc = fmaf(S.xt[s][k], S.w1t[k][u], acc);
        const float h = fmaxf(acc + S.b1[u], 0.0f);
        S.h1[s][u] = h;
        S.h1t[s][u] = bf(h);
    }
    __syncthreads();
    // layer 2: thread = 2 samples x 4 units, operands read once per 8 FMAs
    {
        const int v0 = 4 * (t & 15), s0 = 2 * (t >> 4);
        float acc[2][4] = {};
#pragma unroll 8
        for (int u = 0; u < H; ++u) {
            const float a0 = S.h1t[s0][u], a1 = S.h1t[s0 + 1][u];
            const float4 w = *reinterpret_cast<const float4*>(&S.w2t[u][v0]);
            acc[0][0] = fmaf(a0, w.x, acc[0][0]);
            acc[0][1] = fmaf(a0, w.y, acc[0][1]);
            acc[0][2] = fmaf(a0, w.z, acc[0][2]);
            acc[0][3] = fmaf(a0, w.w, acc[0][3]);
            acc[1][0] = fmaf(a1, w.x, acc[1][0]);
            acc[1][1] = fmaf(a1, w.y, acc[1][1]);
            acc[1][2] = fmaf(a1, w.z, acc[1][2]);
            acc[1][3] = fmaf(a1, w.w, acc[1][3]);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float h = fmaxf(acc[j][i] + S.b2[v0 + i], 0.0f);
                S.h2[s0 + j][v0 + i] = h;
                S.h2t[s0 + j][v0 + i] = bf(h);
            }
    }
    __syncthreads();
    // output and residual (8 threads per sample, lanes 8s'..8s'+7 of a warp)
    {
        float part = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) part = fmaf(S.h2t[s][g + 8 * i], S.w3[g + 8 * i], part);
        part += __shfl_xor_sync(0xFFFFFFFFu, part, 1);
        part += __shfl_xor_sync(0xFFFFFFFFu, part, 2);
        part += __shfl_xor_sync(0xFFFFFFFFu, part, 4);
        if (g == 0) {
            const bool valid = s < n_valid;
            const float r = valid ? (part + S.b3) - S.ys[s] : 0.0f;
            S.dy[s] = valid ? 2.0f * r / B_scale : 0.0f;
            S.ys[s] = r * r;  // reuse: squared residual
        }
    }
    __syncthreads();
    // dz2 = dyhat W3~ [z2 > 0]
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int v = g + 8 * i;
        const float d = S.h2[s][v] > 0.0f ? S.dy[s] * S.w3[v] : 0.0f;
        S.dz2[s][v] = d;
        S.dz2t[s][v] = bf(d);
    }
    __syncthreads();
    // dz1 = (dz2~ W2~) [z1 > 0], same blocking
    {
        const int u0 = 4 * (t & 15), s0 = 2 * (t >> 4);
        float acc[2][4] = {};
#pragma unroll 8
        for (int v = 0; v < H; ++v) {
            const float a0 = S.dz2t[s0][v], a1 = S.dz2t[s0 + 1][v];
            const float4 w = *reinterpret_cast<const float4*>(&S.w2[v][u0]);
            acc[0][0] = fmaf(a0, w.x, acc[0][0]);
            acc[0][1] = fmaf(a0, w.y, acc[0][1]);
            acc[0][2] = fmaf(a0, w.z, acc[0][2]);
            acc[0][3] = fmaf(a0, w.w, acc[0][3]);
            acc[1][0] = fmaf(a1, w.x, acc[1][0]);
            acc[1][1] = fmaf(a1, w.y, acc[1][1]);
            acc[1][2] = fmaf(a1, w.z, acc[1][2]);
            acc[1][3] = fmaf(a1, w.w, acc[1][3]);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                S.dz1[s0 + j][u0 + i] = S.h1[s0 + j][u0 + i] > 0.0f ? acc[j][i] : 0.0f;
    }
    __syncthreads();
}

// The tile's gradient into out[0 .. P) and its squared-residual sum into
// *loss (every parameter has one owner thread).
__device__ void tile_write(const GradSmem& S, int d_in, float* out, float* loss) {
    const int t = threadIdx.x;
    {  // dW2: thread = 4 x 4 block, two float4 loads per 16 FMAs
        const int v0 = 4 * (t >> 4), u0 = 4 * (t & 15);
        float acc[4][4] = {};
#pragma unroll 4
        for (int q = 0; q < kTile; ++q) {
            const float4 a = *reinterpret_cast<const float4*>(&S.dz2t[q][v0]);
            const float4 b = *reinterpret_cast<const float4*>(&S.h1t[q][u0]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                out[off_w2(d_in) + (v0 + i) * H + u0 + j] = acc[i][j];
            }
    }
    for (int i = t; i < H * d_in; i += kGradThreads) {
        const int u = i / d_in, k = i - u * d_in;
        float acc = 0.0f;
        for (int q = 0; q < kTile; ++q) acc = fmaf(bf(S.dz1[q][u]), S.xt[q][k], acc);
        out[i] = acc;
    }
    if (t < H) {
        float a3 = 0.0f, a2 = 0.0f, a1 = 0.0f;
        for (int q = 0; q < kTile; ++q) {
            a3 = fmaf(S.dy[q], S.h2t[q][t], a3);
            a2 += S.dz2[q][t];
            a1 += S.dz1[q][t];
        }
        out[off_w3(d_in) + t] = a3;
        out[off_b2(d_in) + t] = a2;
        out[off_b1(d_in) + t] = a1;
    }
    if (t == H) {
        float a = 0.0f, l = 0.0f;
        for (int q = 0; q < kTile; ++q) {
            a += S.dy[q];
            l += S.ys[q];
        }
        out[off_b3(d_in)] = a;
        *loss = l;
    }
}

// Forward + backward of one tile of kTile samples; partial[blockIdx][p] gets
// the tile's gradient, partial_loss[blockIdx] its sum of squared residuals.
__global__ void __launch_bounds__(kGradThreads) mlp_grad_kernel(
    const float* __restrict__ theta, int d_in, const float* __restrict__ X, long long n_total,
    const float* __restrict__ Y, SampleMap map, long long B, float* __restrict__ partial,
    float* __restrict__ partial_loss) {
    extern __shared__ unsigned char smem_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
    const long long base = static_cast<long long>(blockIdx.x) * kTile;
    const int n_valid = static_cast<int>(min(static_cast<long long>(kTile), B - base));
    stage_weights(S, theta, d_in);
    stage_tile(S, d_in, X, n_total, Y, map, base, n_valid);
    __syncthreads();
    tile_passes(S, d_in, n_valid, static_cast<float>(B));
    tile_write(S, d_in, partial + static_cast<long long>(blockIdx.x) * n_params(d_in),
                      partial_loss + blockIdx.x);
}

// grad[p] = sum over CTAs of partial[c][p] (fixed order); optionally Adam.
template <bool kAdam>
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, const float* __restrict__ partial_loss,
                                  int n_cta, long long P, long long B, float* __restrict__ grad,
                                  float* __restrict__ loss, float* __restrict__ theta, float* __restrict__ m,
                                  float* __restrict__ v, float lr, float beta1, float beta2, float eps,
                                  float bc1, float bc2) {
    const long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (p < P) {
        float acc = 0.0f;
        for (int c = 0; c < n_cta; ++c) acc += partial[static_cast<long long>(c) * P + p];
        if (grad) grad[p] = acc;
        if (kAdam) {
            const float mi = beta1 * m[p] + (1.0f - beta1) * acc;
            const float vi = beta2 * v[p] + (1.0f - beta2) * acc * acc;
            m[p] = mi;
            v[p] = vi;
            const float mhat = mi / bc1;
            const float vhat = vi / bc2;
            theta[p] = theta[p] - lr * mhat / (sqrtf(vhat) + eps);
        }
    }
    if (p == 0 && loss) {
        float l = 0.0f;
        for (int c = 0; c < n_cta; ++c) l += partial_loss[c];
        *loss = l / static_cast<float>(B);
    }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float beta1, float beta2,
                            float eps, float bc1, float bc2) {
    const long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (p >= n) return;
    const float gi = g[p];
    const float mi = beta1 * m[p] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[p] + (1.0f - beta2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    theta[p] = theta[p] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ---------------------------------------------------------------------------
// Whole training run in one launch (mlp_train_tc_kernel below): a cluster of
// CTAs keeps the network in shared memory for all epochs.
// ---------------------------------------------------------------------------
struct TrainArgs {
    const float* X;  // standardised features, d_in planes of n_tr
    const float* Y;
    long long n_tr, B, steps_per_epoch;
    int epochs, d_in;
    const unsigned long long* ab;  // per epoch: the affine order (a, b)
    const float* bc;               // per step: the bias corrections (1 - beta1^t, 1 - beta2^t)
    float lr, beta1, beta2, eps;
    float* theta;   // in: initial parameters; out: trained (the best epoch's with validation)
    float* losses;  // per step: mean squared residual of the minibatch (may be null)
    long long max_steps;  // > 0: stop after this many steps
    float* grad;    // may be null: the gradient of the last step
    float* m_out;   // may be null: Adam's first moment after the last step
    float* v_out;   // may be null: Adam's second moment after the last step
    const float* Xv;  // validation features, d_in planes of n_val (n_val = 0: none)
    const float* Yv;
    long long n_val;
    int patience;       // > 0: stop after this many epochs without a lower validation loss
    float* val_losses;  // per epoch (may be null)
    int* info;          // may be null: epochs run, epoch kept, steps run
    const float* m_in;  // may be null (zero): Adam's moments to resume from
    const float* v_in;
    float best0;        // validation loss to beat (+inf: none yet)
    int bad0;           // epochs without a lower validation loss so far
    const float* theta_in;  // may be null (= theta): the parameters to start from
    float* theta_last;      // may be null: the parameters after the last step run
};

// ---------------------------------------------------------------------------
// Training with the four 64-wide contractions on the tensor cores (tcgen05,
// FP32 accumulators in tensor memory).  A cluster of kTcCluster CTAs of 512
// threads holds the FP32 parameters in every CTA's shared memory; per step
// each CTA takes 1/kTcCluster of the minibatch in tiles of 128 samples
// (sample m = TMEM lane m, its 64 columns split over 4 threads):
//   Z1  = X~ W1~^T        (M 128, N 64, K 16: the d_in features, zero-padded)
//   Z2  = H1~ W2~^T       (K 64)
//   dH1 = dZ2~ W2~        (K 64, B = W2~ transposed)
//   dW2 = dZ2~^T H1~      (M 128 with rows 64..127 zero, K = the 128 samples)
//   dW1 = dZ1~^T X~       (M 128 with rows 64..127 zero, N 16, K = the 128 samples)
// Each thread turns its 16 columns of a row of Z1 / Z2 / dH1 into
// activations, residual and deltas (FP32, rounded to BF16 where the next
// contraction reads them) and writes them in the operands' core-matrix
// layouts (16-byte stores where a row's 8 columns are contiguous); the bias
// and W3 gradients are FP32 column sums over the tile in a fixed order
// (chunks of 16 samples, then the chunks in order).  After a cluster barrier CTA r owns the r-th slice of the
// parameters: it adds that slice of every CTA's gradient in rank order over
// distributed shared memory, applies Adam and writes the new values into
// every CTA's copy; a second barrier ends the step.  Same arithmetic as
// mlp_step (BF16 operands, FP32 sums; only the order of the sums differs).
// Every MMA completion is awaited with an
// iteration limit; on a timeout the CTA stops issuing MMAs, runs on to the
// same barriers (so no peer waits forever) and reports it in *err.
// ---------------------------------------------------------------------------
constexpr int kTcCluster = 8;
constexpr int kTcThreads = 512;  // 4 threads per sample row, 16 columns each
constexpr int kTcRows = 128;
constexpr int kTcChunks = kTcThreads / H;  // row chunks of the column sums
constexpr int kTcWait = 1 << 22;

struct TcSmem {
    alignas(1024) unsigned char a1[kTcRows * 16 * 2];      // X~ tile, K = 16
    alignas(1024) unsigned char w1b[H * 16 * 2];           // W1~ as B, K = 16
    alignas(1024) unsigned char a2[kTcRows * H * 2];       // H1~ rows, K = 64
    alignas(1024) unsigned char w2b[H * H * 2];            // W2~ [v][u] as B
    alignas(1024) unsigned char w2tb[H * H * 2];           // W2~ [u][v] as B
    alignas(1024) unsigned char h1tt[H * kTcRows * 2];     // H1~ transposed [u][m], K = 128
    alignas(1024) unsigned char a3[kTcRows * H * 2];       // dZ2~ rows, K = 64
    alignas(1024) unsigned char dz2tt[kTcRows * kTcRows * 2];  // dZ2~, then dZ1~, transposed [v][m]; rows 64.. zero
    alignas(1024) unsigned char xtt[16 * kTcRows * 2];     // X~ transposed [k][m], K = 128; rows d_in.. zero
    float f32[kTcRows][H + 1];                             // dZ2, then dZ1 (FP32)
    __nv_bfloat16 h2t[kTcRows][H + 2];                     // H2~ rows (for dW3)
    float ypart[4][kTcRows];                               // output partials per column block
    float colpart[3][kTcChunks][H];                        // column sums per row chunk
    float dy[kTcRows], r2[kTcRows];
    float w3[H], b1[H], b2[H];
    float b3;
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ void put_bf16(unsigned char* tile, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(tile + off) = __float2bfloat16_rn(v);
}

// Eight FP32 values rounded to BF16 (nearest even), the first at the lowest
// address: one core-matrix row of 16 bytes.
__device__ __forceinline__ uint4 pack_bf16x8(const float* w) {
    uint32_t r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(w[2 * q], w[2 * q + 1]);
        r[q] = *reinterpret_cast<const uint32_t*>(&p);
    }
    return make_uint4(r[0], r[1], r[2], r[3]);
}

__global__ void __cluster_dims__(kTcCluster, 1, 1) __launch_bounds__(kTcThreads, 1)
    mlp_train_tc_kernel(TrainArgs ta, int* err) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw);
    const int d_in = ta.d_in;
    const int P = static_cast<int>(n_params(d_in));
    const int P4 = (P + 1 + 3) & ~3;
    float* th = reinterpret_cast<float*>(tc_raw + sizeof(TcSmem));
    float* part = th + P4;
    const int slice = (P + kTcCluster - 1) / kTcCluster;
    float* mom = part + P4;
    float* vel = mom + slice;
    const int rank = static_cast<int>(cluster.block_rank());
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int quarter = warp & 3, cb = warp >> 2;  // TMEM lane quarter, column block
    const int m = 32 * quarter + lane;              // this thread's sample row / TMEM lane
    const int c0 = 16 * cb;                         // its 16 columns
    const int p_lo = rank * slice, p_hi = min(P, p_lo + slice);
    constexpr uint32_t kIdesc = tc::idesc_bf16(kTcRows, H);
    constexpr uint32_t kIdescW1 = tc::idesc_bf16(kTcRows, 16);
    // (debug build: the layout must fit the launch's shared memory; every CTA
    // of the cluster computes the same sizes, so all leave together, before
    // any cluster barrier or tensor-memory allocation)
    if (!MRIP_CHECK(sizeof(TcSmem) + (2ull * P4 + 2ull * slice) * sizeof(float) <= dynamic_smem_bytes(), 402, P)) {
        if (t == 0 && rank == 0) atomicExch(err, 1);
        return;
    }

    if (warp == 0) tc::tmem_alloc(&S.tmem, 256);
    if (t == 0) tc::mbar_init(&S.bar);
    const float* th_src = ta.theta_in ? ta.theta_in : ta.theta;
    for (int i = t; i < P; i += kTcThreads) th[i] = th_src[i];
    for (int i = t; i < slice; i += kTcThreads) {
        const int p = p_lo + i;
        mom[i] = (ta.m_in && p < P) ? ta.m_in[p] : 0.0f;
        vel[i] = (ta.v_in && p < P) ? ta.v_in[p] : 0.0f;
    }
    for (int i = t; i < kTcRows * kTcRows * 2 / 16; i += kTcThreads)
        reinterpret_cast<uint4*>(S.dz2tt)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = t; i < kTcRows * 16 * 2 / 16; i += kTcThreads) {
        reinterpret_cast<uint4*>(S.a1)[i] = make_uint4(0u, 0u, 0u, 0u);
        reinterpret_cast<uint4*>(S.xtt)[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_before_sync();
    cluster.sync();
    tc::fence_after_sync();
    const uint32_t tm = S.tmem;
    const uint32_t lane_base = static_cast<uint32_t>(32 * quarter) << 16;
    uint32_t phase = 0;
    bool ok = true;

    // one MMA group's completion: every thread polls; ok stays CTA-uniform
    auto wait_mma = [&]() {
        bool mine = ok ? tc::mbar_wait(&S.bar, phase, kTcWait) : false;
        phase ^= 1u;
        tc::fence_before_sync();
        const bool all = __syncthreads_and(mine) != 0;
        tc::fence_after_sync();
        if (ok && !all) {
            ok = false;
            if (t == 0) atomicExch(err, 1);
        }
    };
    auto sync_for_mma = [&]() {
        tc::fence_smem_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    // BF16 operands (and FP32 biases) of the current parameters th; every
    // thread packs 8 consecutive K elements of one operand row into one
    // 16-byte store (a core-matrix row)
    auto stage_weights = [&]() {
        if (t < 2 * H) {  // W1~ as B: row u, K = the 16 (zero-padded) inputs
            const int u = t >> 1, k0 = 8 * (t & 1);
            float w[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] = k0 + q < d_in ? theta_w1(th, d_in, u, k0 + q) : 0.0f;
            *reinterpret_cast<uint4*>(S.w1b + tc::core_offset(u, k0, 16)) = pack_bf16x8(w);
        }
        {   // W2~ [v][u] as B of Z2 (K = u): row v, columns 8j .. 8j + 7
            const int v = t >> 3, j = t & 7;
            const float4* src = reinterpret_cast<const float4*>(th + off_w2(d_in) + v * H + 8 * j);
            const float4 a = src[0], b = src[1];
            const float w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            *reinterpret_cast<uint4*>(S.w2b + tc::core_offset(v, 8 * j, H)) = pack_bf16x8(w);
        }
        {   // W2~ transposed [u][v] as B of dH1 (K = v): row u, columns 8j .. 8j + 7
            const int u = t & (H - 1), j = t >> 6;
            float w[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] = th[off_w2(d_in) + (8 * j + q) * H + u];
            *reinterpret_cast<uint4*>(S.w2tb + tc::core_offset(u, 8 * j, H)) = pack_bf16x8(w);
        }
        for (int i = t; i < H; i += kTcThreads) {
            S.w3[i] = bf(th[off_w3(d_in) + i]);
            S.b1[i] = th[off_b1(d_in) + i];
            S.b2[i] = th[off_b2(d_in) + i];
        }
        if (t == 0) S.b3 = th[off_b3(d_in)];
    };
    // Forward pass of one tile: row m is sample smp of the planes Xs (n_total
    // samples each) when valid, else zero.  Leaves H1~ (rows and transposed),
    // H2~ rows and X~ in shared memory and the ReLU masks of this thread's 16
    // columns in mask1 / mask2; returns the output of row m without b3.
    auto forward_tile = [&](const float* Xs, long long n_total, long long smp, bool valid, uint32_t& mask1,
                            uint32_t& mask2) -> float {
        for (int k = 2 * cb; k < 2 * cb + 2 && k < d_in; ++k) {  // features 2cb, 2cb + 1 of row m
            const float x = valid ? bf(Xs[k * n_total + smp]) : 0.0f;
            put_bf16(S.a1, tc::core_offset(m, k, 16), x);
            put_bf16(S.xtt, tc::core_offset(k, m, kTcRows), x);
        }
        sync_for_mma();
        if (t == 0 && ok) {
            tc::mma_bf16(tm, tc::smem_desc(tc::smem_addr(S.a1), 128, 256),
                         tc::smem_desc(tc::smem_addr(S.w1b), 128, 256), kIdesc, false);
            tc::mma_commit(&S.bar);
        }
        wait_mma();
        // layer 1 epilogue: h1 = relu(z1 + b1) on columns c0 .. c0 + 15
        mask1 = 0u;
        {
            float z[16];
            tc::tmem_ld16(tm + lane_base + c0, z);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int u = c0 + j;
                const float h = fmaxf(z[j] + S.b1[u], 0.0f);
                if (h > 0.0f) mask1 |= 1u << j;
                z[j] = bf(h);
                put_bf16(S.h1tt, tc::core_offset(u, m, kTcRows), z[j]);
            }
            *reinterpret_cast<uint4*>(S.a2 + tc::core_offset(m, c0, H)) = pack_bf16x8(z);
            *reinterpret_cast<uint4*>(S.a2 + tc::core_offset(m, c0 + 8, H)) = pack_bf16x8(z + 8);
        }
        sync_for_mma();
        if (t == 0 && ok) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                tc::mma_bf16(tm + 64, tc::smem_desc(tc::smem_addr(S.a2) + 256 * ks, 128, 1024),
                             tc::smem_desc(tc::smem_addr(S.w2b) + 256 * ks, 128, 1024), kIdesc, ks > 0);
            tc::mma_commit(&S.bar);
        }
        wait_mma();
        // layer 2 epilogue: h2 and this block's share of the output
        mask2 = 0u;
        {
            float z[16], yp = 0.0f;
            tc::tmem_ld16(tm + lane_base + 64 + c0, z);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int v = c0 + j;
                const float h = fmaxf(z[j] + S.b2[v], 0.0f);
                if (h > 0.0f) mask2 |= 1u << j;
                const float hb = bf(h);
                S.h2t[m][v] = __float2bfloat16_rn(hb);
                yp = fmaf(hb, S.w3[v], yp);
            }
            S.ypart[cb][m] = yp;
        }
        __syncthreads();
        return ((S.ypart[0][m] + S.ypart[1][m]) + S.ypart[2][m]) + S.ypart[3][m];
    };

    long long step = 0;
    bool stop = false;
    float best = ta.best0;
    int bad = ta.bad0, best_epoch = 0, epochs_run = 0;
    for (int ep = 0; ep < ta.epochs && !stop; ++ep) {
        const SampleMap map{nullptr, ta.ab[2 * ep], ta.ab[2 * ep + 1], static_cast<unsigned long long>(ta.n_tr), 0};
        for (long long off = 0; off < ta.n_tr; off += ta.B, ++step) {
            if (ta.max_steps > 0 && step >= ta.max_steps) {  // uniform across the cluster
                stop = true;
                break;
            }
            const long long nb = (off + ta.B <= ta.n_tr) ? ta.B : ta.n_tr - off;
            const long long chunk = (nb + kTcCluster - 1) / kTcCluster;
            const long long lo = min(nb, rank * chunk), hi = min(nb, lo + chunk);
            SampleMap smap = map;
            smap.off = off;
            stage_weights();
            for (int i = t; i <= P; i += kTcThreads) part[i] = 0.0f;

            for (long long p0 = lo; p0 < hi; p0 += kTcRows) {
                const int n_valid = static_cast<int>(min(static_cast<long long>(kTcRows), hi - p0));
                const bool valid = m < n_valid;
                long long smp = valid ? sample_of(smap, p0 + m) : 0;
                if (valid && !MRIP_CHECK(smp >= 0 && smp < ta.n_tr, 401, smp)) smp = 0;
                const float y = valid ? ta.Y[smp] : 0.0f;
                uint32_t mask1, mask2;
                const float yhat = forward_tile(ta.X, ta.n_tr, smp, valid, mask1, mask2);
                const float r = valid ? (yhat + S.b3) - y : 0.0f;
                const float dyv = valid ? 2.0f * r / static_cast<float>(nb) : 0.0f;
                if (cb == 0) {
                    S.dy[m] = dyv;
                    S.r2[m] = r * r;
                }
                {
                    float db[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int v = c0 + j;
                        const float d = ((mask2 >> j) & 1u) ? dyv * S.w3[v] : 0.0f;
                        S.f32[m][v] = d;
                        db[j] = bf(d);
                        put_bf16(S.dz2tt, tc::core_offset(v, m, kTcRows), db[j]);
                    }
                    *reinterpret_cast<uint4*>(S.a3 + tc::core_offset(m, c0, H)) = pack_bf16x8(db);
                    *reinterpret_cast<uint4*>(S.a3 + tc::core_offset(m, c0 + 8, H)) = pack_bf16x8(db + 8);
                }
                sync_for_mma();
                if (t == 0 && ok) {
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)  // dH1 = dZ2~ W2~
                        tc::mma_bf16(tm, tc::smem_desc(tc::smem_addr(S.a3) + 256 * ks, 128, 1024),
                                     tc::smem_desc(tc::smem_addr(S.w2tb) + 256 * ks, 128, 1024), kIdesc, ks > 0);
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks)  // dW2 = dZ2~^T H1~
                        tc::mma_bf16(tm + 128, tc::smem_desc(tc::smem_addr(S.dz2tt) + 256 * ks, 128, 2048),
                                     tc::smem_desc(tc::smem_addr(S.h1tt) + 256 * ks, 128, 2048), kIdesc, ks > 0);
                    tc::mma_commit(&S.bar);
                }
                // meanwhile: column sums of dZ2 (b2) and dy h2~ (W3) per chunk of 16 rows
                {
                    const int v = t & (H - 1), ch = t / H;
                    float a2 = 0.0f, a3 = 0.0f;
                    for (int q = 16 * ch; q < 16 * ch + 16; ++q) {
                        a2 += S.f32[q][v];
                        a3 = fmaf(S.dy[q], __bfloat162float(S.h2t[q][v]), a3);
                    }
                    S.colpart[0][ch][v] = a2;
                    S.colpart[1][ch][v] = a3;
                }
                wait_mma();  // includes the barrier that frees S.f32
                if (t < H) {
                    float a2 = 0.0f, a3 = 0.0f;
                    for (int ch = 0; ch < kTcChunks; ++ch) {
                        a2 += S.colpart[0][ch][t];
                        a3 += S.colpart[1][ch][t];
                    }
                    part[off_b2(d_in) + t] += a2;
                    part[off_w3(d_in) + t] += a3;
                } else if (t == H) {
                    float a = 0.0f, l = 0.0f;
                    for (int q = 0; q < kTcRows; ++q) {
                        a += S.dy[q];
                        l += S.r2[q];
                    }
                    part[off_b3(d_in)] += a;
                    part[P] += l;
                }
                // dZ1 = dH1 [z1 > 0] (FP32 for b1; BF16 transposed into the
                // freed dZ2~ buffer for dW1); dW2 rows 0..63 (TMEM lanes 0..63)
                // into the gradient
                {
                    float z[16];
                    tc::tmem_ld16(tm + lane_base + c0, z);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float d = ((mask1 >> j) & 1u) ? z[j] : 0.0f;
                        S.f32[m][c0 + j] = d;
                        put_bf16(S.dz2tt, tc::core_offset(c0 + j, m, kTcRows), d);
                    }
                }
                if (quarter < 2) {
                    float z[16];
                    tc::tmem_ld16(tm + lane_base + 128 + c0, z);
#pragma unroll
                    for (int j = 0; j < 16; ++j) part[off_w2(d_in) + m * H + c0 + j] += z[j];
                }
                sync_for_mma();
                if (t == 0 && ok) {
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks)  // dW1 = dZ1~^T X~
                        tc::mma_bf16(tm + 192, tc::smem_desc(tc::smem_addr(S.dz2tt) + 256 * ks, 128, 2048),
                                     tc::smem_desc(tc::smem_addr(S.xtt) + 256 * ks, 128, 2048), kIdescW1, ks > 0);
                    tc::mma_commit(&S.bar);
                }
                // meanwhile: column sums of dZ1 (b1) per chunk
                {
                    const int u = t & (H - 1), ch = t / H;
                    float a1 = 0.0f;
                    for (int q = 16 * ch; q < 16 * ch + 16; ++q) a1 += S.f32[q][u];
                    S.colpart[2][ch][u] = a1;
                }
                wait_mma();
                if (t < H) {
                    float a1 = 0.0f;
                    for (int ch = 0; ch < kTcChunks; ++ch) a1 += S.colpart[2][ch][t];
                    part[off_b1(d_in) + t] += a1;
                }
                if (quarter < 2 && cb == 0) {  // dW1 rows u = m < 64 (TMEM lanes 0..63), columns = inputs
                    float z[16];
                    tc::tmem_ld16(tm + lane_base + 192, z);
                    for (int k = 0; k < d_in; ++k) part[m * d_in + k] += z[k];
                }
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
            }
            cluster.sync();  // every CTA's gradient is complete
            const float bc1 = ta.bc[2 * step], bc2 = ta.bc[2 * step + 1];
            for (int p = p_lo + t; p < p_hi; p += kTcThreads) {
                float g = 0.0f;
                for (int rr = 0; rr < kTcCluster; ++rr) g += cluster.map_shared_rank(part, rr)[p];
                if (ta.grad) ta.grad[p] = g;
                const int q = p - p_lo;
                const float mi = ta.beta1 * mom[q] + (1.0f - ta.beta1) * g;
                const float vi = ta.beta2 * vel[q] + (1.0f - ta.beta2) * g * g;
                mom[q] = mi;
                vel[q] = vi;
                const float nv = th[p] - ta.lr * (mi / bc1) / (sqrtf(vi / bc2) + ta.eps);
                for (int rr = 0; rr < kTcCluster; ++rr) cluster.map_shared_rank(th, rr)[p] = nv;
            }
            if (rank == 0 && t == 0) {
                float l = 0.0f;
                for (int rr = 0; rr < kTcCluster; ++rr) l += cluster.map_shared_rank(part, rr)[P];
                if (ta.losses) ta.losses[step] = l / static_cast<float>(nb);
            }
            cluster.sync();
        }
        if (stop) break;
        ++epochs_run;
        if (ta.n_val > 0) {
            // validation loss of this epoch's parameters (each CTA a slice of
            // the validation samples, in order; the CTAs' sums added in rank
            // order, so every CTA computes the same value and takes the same
            // early-stopping decision)
            stage_weights();
            if (t == 0) part[P] = 0.0f;
            __syncthreads();
            const long long vchunk = (ta.n_val + kTcCluster - 1) / kTcCluster;
            const long long vlo = min(ta.n_val, rank * vchunk), vhi = min(ta.n_val, vlo + vchunk);
            for (long long p0 = vlo; p0 < vhi; p0 += kTcRows) {
                const int n_valid = static_cast<int>(min(static_cast<long long>(kTcRows), vhi - p0));
                const bool valid = m < n_valid;
                const long long smp = valid ? p0 + m : 0;
                uint32_t mask1, mask2;
                const float yhat = forward_tile(ta.Xv, ta.n_val, smp, valid, mask1, mask2);
                const float r = valid ? (yhat + S.b3) - ta.Yv[smp] : 0.0f;
                if (cb == 0) S.r2[m] = r * r;
                __syncthreads();
                if (t == H) {
                    float l = 0.0f;
                    for (int q = 0; q < kTcRows; ++q) l += S.r2[q];
                    part[P] += l;
                }
                __syncthreads();
            }
            cluster.sync();
            float vl = 0.0f;
            for (int rr = 0; rr < kTcCluster; ++rr) vl += cluster.map_shared_rank(part, rr)[P];
            vl /= static_cast<float>(ta.n_val);
            cluster.sync();  // every CTA has read the sums before part[] is cleared again
            if (rank == 0 && t == 0 && ta.val_losses) ta.val_losses[ep] = vl;
            if (vl < best) {
                best = vl;
                best_epoch = ep + 1;
                bad = 0;
                for (int p = p_lo + t; p < p_hi; p += kTcThreads) ta.theta[p] = th[p];
            } else if (ta.patience > 0 && ++bad >= ta.patience) {
                stop = true;
            }
        }
    }
    if (ta.n_val == 0)
        for (int p = p_lo + t; p < p_hi; p += kTcThreads) ta.theta[p] = th[p];
    if (ta.theta_last)
        for (int p = p_lo + t; p < p_hi; p += kTcThreads) ta.theta_last[p] = th[p];
    if (ta.m_out)
        for (int p = p_lo + t; p < p_hi; p += kTcThreads) ta.m_out[p] = mom[p - p_lo];
    if (ta.v_out)
        for (int p = p_lo + t; p < p_hi; p += kTcThreads) ta.v_out[p] = vel[p - p_lo];
    if (rank == 0 && t == 0 && ta.info) {
        ta.info[0] = epochs_run;
        ta.info[1] = ta.n_val > 0 ? best_epoch : epochs_run;
        ta.info[2] = static_cast<int>(step);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tm, 256);
}

size_t mlp_train_tc_smem(int d_in) {
    const int P = static_cast<int>(n_params(d_in));
    const int P4 = (P + 1 + 3) & ~3;
    const int slice = (P + kTcCluster - 1) / kTcCluster;
    return sizeof(TcSmem) + (2 * static_cast<size_t>(P4) + 2 * slice) * sizeof(float);
}

// Inference, one sample per thread, weights (BF16-rounded) in shared memory.
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ theta, int d_in,
                                                         const float* __restrict__ X, long long n,
                                                         float* __restrict__ yhat) {
    __shared__ float w1[H][kMaxIn];
    __shared__ __align__(16) float w2[H][H];  // [v][u]
    __shared__ float w3[H], b1[H], b2[H];
    __shared__ float b3;
    for (int i = threadIdx.x; i < H * kMaxIn; i += blockDim.x) {
        const int u = i / kMaxIn, k = i - u * kMaxIn;
        w1[u][k] = k < d_in ? bf(theta[u * d_in + k]) : 0.0f;
    }
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) w2[i / H][i % H] = bf(theta[off_w2(d_in) + i]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        w3[i] = bf(theta[off_w3(d_in) + i]);
        b1[i] = theta[off_b1(d_in) + i];
        b2[i] = theta[off_b2(d_in) + i];
    }
    if (threadIdx.x == 0) b3 = theta[off_b3(d_in)];
    __syncthreads();
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    float x[kMaxIn];
#pragma unroll
    for (int k = 0; k < kMaxIn; ++k) x[k] = k < d_in ? bf(X[k * n + i]) : 0.0f;
    float h1[H];
#pragma unroll
    for (int u = 0; u < H; ++u) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < kMaxIn; ++k) acc = fmaf(x[k], w1[u][k], acc);
        h1[u] = bf(fmaxf(acc + b1[u], 0.0f));
    }
    float out = 0.0f;
    for (int v = 0; v < H; ++v) {
        float acc = 0.0f;
        const float4* row = reinterpret_cast<const float4*>(&w2[v][0]);
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
            const float4 w = row[q];
            acc = fmaf(h1[4 * q], w.x, acc);
            acc = fmaf(h1[4 * q + 1], w.y, acc);
            acc = fmaf(h1[4 * q + 2], w.z, acc);
            acc = fmaf(h1[4 * q + 3], w.w, acc);
        }
        out = fmaf(bf(fmaxf(acc + b2[v], 0.0f)), w3[v], out);
    }
    yhat[i] = out + b3;
}

// Control-variate reduction of one design point per CTA (FP64, two passes,
// fixed-order tree sums).
constexpr int kCvThreads = 256;

__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int stride = kCvThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) sh[threadIdx.x] += sh[threadIdx.x + stride];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kCvThreads) cv_reduce_kernel(const double* __restrict__ y,
                                                               const double* __restrict__ g, long long n,
                                                               const double* __restrict__ gc, long long m,
                                                               double* __restrict__ out) {
    __shared__ double sh[kCvThreads];
    const long long dp = blockIdx.x;
    const double* yr = y + dp * n;
    const double* gr = g + dp * n;
    const double* cr = gc + dp * m;
    double sy = 0.0, sg = 0.0, sc = 0.0;
    for (long long i = threadIdx.x; i < n; i += kCvThreads) {
        sy += yr[i];
        sg += gr[i];
    }
    for (long long i = threadIdx.x; i < m; i += kCvThreads) sc += cr[i];
    const double ybar = block_sum(sy, sh) / static_cast<double>(n);
    const double gbar = block_sum(sg, sh) / static_cast<double>(n);
    const double cbar = block_sum(sc, sh) / static_cast<double>(m);
    double sxy = 0.0, sgg = 0.0, scc = 0.0;
    for (long long i = threadIdx.x; i < n; i += kCvThreads) {
        const double dy = yr[i] - ybar, dg = gr[i] - gbar;
        sxy += dy * dg;
        sgg += dg * dg;
    }
    for (long long i = threadIdx.x; i < m; i += kCvThreads) {
        const double dc = cr[i] - cbar;
        scc += dc * dc;
    }
    const double cov = block_sum(sxy, sh) / static_cast<double>(n - 1);
    const double var_g = block_sum(sgg, sh) / static_cast<double>(n - 1);
    const double var_c = block_sum(scc, sh) / static_cast<double>(m - 1);
    const double beta = var_g > 0.0 ? cov / var_g : 0.0;
    double sr = 0.0;
    for (long long i = threadIdx.x; i < n; i += kCvThreads) sr += yr[i] - beta * gr[i];
    const double rbar = block_sum(sr, sh) / static_cast<double>(n);
    double srr = 0.0;
    for (long long i = threadIdx.x; i < n; i += kCvThreads) {
        const double d = (yr[i] - beta * gr[i]) - rbar;
        srr += d * d;
    }
    const double s_r2 = block_sum(srr, sh) / static_cast<double>(n - 2);
    if (threadIdx.x == 0) {
        out[5 * dp] = beta;
        out[5 * dp + 1] = ybar - beta * (gbar - cbar);
        out[5 * dp + 2] = s_r2 / static_cast<double>(n) + beta * beta * var_c / static_cast<double>(m);
        out[5 * dp + 3] = ybar;
        out[5 * dp + 4] = gbar - cbar;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// internal launchers used by the control-variate driver
// ---------------------------------------------------------------------------
long long mlp_params(int d_in) { return n_params(d_in); }

mrip_status mlp_init(int d_in, uint64_t seed, float* theta, cudaStream_t st) {
    const long long n_w = static_cast<long long>(H) * d_in + H * H + H;
    mlp_init_kernel<<<ceil_div_u(n_w, 256), 256, 0, st>>>(d_in, expand_key(seed), theta);
    return launch_status("mlp init");
}

size_t mlp_grad_partial_floats(int d_in, long long B) {
    return static_cast<size_t>((B + kTile - 1) / kTile) * static_cast<size_t>(n_params(d_in) + 1);
}

// One gradient (and optionally Adam) step over batch positions [0, B) of map.
mrip_status mlp_step(const float* theta_in, int d_in, const float* X, long long n_total, const float* Y,
                     const int64_t* idx, unsigned long long a, unsigned long long b, unsigned long long n_perm,
                     long long off, long long B, float* partial, float* grad, float* loss, float* theta,
                     float* m, float* v, const float* adam /* lr, b1, b2, eps, bc1, bc2 */, cudaStream_t st) {
    const int n_cta = static_cast<int>((B + kTile - 1) / kTile);
    const long long P = n_params(d_in);
    float* part_loss = partial + static_cast<long long>(n_cta) * P;
    SampleMap map{idx, a, b, n_perm, off};
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sizeof(GradSmem)));
    if (e != cudaSuccess) return cuda_status(e, "mlp: shared memory attribute");
    mlp_grad_kernel<<<n_cta, kGradThreads, sizeof(GradSmem), st>>>(theta_in, d_in, X, n_total, Y, map, B,
                                                                   partial, part_loss);
    mrip_status s = launch_status("mlp grad");
    if (s != MRIP_OK) return s;
    if (adam) {
        mlp_reduce_kernel<true><<<ceil_div_u(P, 256), 256, 0, st>>>(
            partial, part_loss, n_cta, P, B, grad, loss, theta, m, v, adam[0], adam[1], adam[2], adam[3],
            adam[4], adam[5]);
    } else {
        mlp_reduce_kernel<false><<<ceil_div_u(P, 256), 256, 0, st>>>(
            partial, part_loss, n_cta, P, B, grad, loss, nullptr, nullptr, nullptr, 0, 0, 0, 0, 1, 1);
    }
    return launch_status("mlp reduce");
}

// Epoch order (a, b) of n samples: block (0, epoch) of tag 4, rep 0, dp 0;
// a = 1 + w0 mod (n - 1) stepped up to the first value coprime with n,
// b = w1 mod n.
void epoch_affine(uint64_t seed, int epoch, unsigned long long n, unsigned long long& a, unsigned long long& b) {
    if (n <= 1) {
        a = 1;
        b = 0;
        return;
    }
    const uint4 w = philox(0u, static_cast<uint32_t>(epoch), 0u, stream_word(4u, 0u), expand_key(seed));
    a = 1 + static_cast<unsigned long long>(w.x) % (n - 1);
    while (std::gcd(a, n) != 1) {
        ++a;
        if (a >= n) a = 1;
    }
    b = static_cast<unsigned long long>(w.y) % n;
}

// Adam training in one cluster launch with the contractions on the tensor
// cores (mlp_train_tc_kernel).  The host computes the schedule -- per epoch
// the affine order, per step Adam's bias corrections in double rounded to
// float -- and uploads it to library scratch.  Synchronous: reads back
// whether an MMA completion wait ran out, and the run's counts.
mrip_status mlp_train(const TrainSpec& sp, TrainInfo* info, cudaStream_t st) {
    NvtxRange range("mlp_train");
    TrainInfo none{0, 0, 0};
    if (info) *info = none;
    if (sp.n == 0 || sp.epochs == 0) return MRIP_OK;
    const long long spe = (sp.n + sp.B - 1) / sp.B;
    long long n_steps = spe * sp.epochs;
    if (sp.max_steps > 0 && sp.max_steps < n_steps) n_steps = sp.max_steps;
    // resuming at epoch epoch0: its order and Adam's step count continue
    const long long step0 = static_cast<long long>(sp.epoch0) * spe;
    std::vector<unsigned long long> ab(2 * static_cast<size_t>(sp.epochs));
    for (int ep = 0; ep < sp.epochs; ++ep)
        epoch_affine(sp.order_seed, sp.epoch0 + ep, static_cast<unsigned long long>(sp.n), ab[2 * ep],
                     ab[2 * ep + 1]);
    std::vector<float> bc(2 * static_cast<size_t>(n_steps));
    for (long long k = 1; k <= n_steps; ++k) {
        const double kk = static_cast<double>(step0 + k);
        bc[2 * (k - 1)] = static_cast<float>(1.0 - std::pow(static_cast<double>(sp.beta1), kk));
        bc[2 * (k - 1) + 1] = static_cast<float>(1.0 - std::pow(static_cast<double>(sp.beta2), kk));
    }
    // scratch: [info 16 B, timeout flag 16 B][ab][bc]
    const size_t ab_bytes = ab.size() * sizeof(unsigned long long);
    const size_t bytes = 32 + ab_bytes + bc.size() * sizeof(float);
    char* base = static_cast<char*>(scratch(bytes, 4));
    if (!base) return fail(MRIP_ENOMEM, "mlp train: scratch allocation failed");
    int* d_info = reinterpret_cast<int*>(base);
    int* flag = reinterpret_cast<int*>(base + 16);
    unsigned long long* d_ab = reinterpret_cast<unsigned long long*>(base + 32);
    float* d_bc = reinterpret_cast<float*>(base + 32 + ab_bytes);
    cudaError_t e = cudaMemsetAsync(base, 0, 32, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ab, ab.data(), ab_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_bc, bc.data(), bc.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "mlp train: schedule upload");
    const size_t smem = mlp_train_tc_smem(sp.d_in);
    e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return cuda_status(e, "mlp train: shared memory attribute");
    TrainArgs ta{sp.X, sp.Y, sp.n, sp.B, spe, sp.epochs, sp.d_in, d_ab, d_bc, sp.lr, sp.beta1, sp.beta2, sp.eps,
                 sp.theta, sp.losses, sp.max_steps, sp.grad, sp.m_out, sp.v_out, sp.Xv, sp.Yv,
                 sp.Xv ? sp.n_val : 0, sp.patience, sp.val_losses, d_info, sp.m_in, sp.v_in,
                 sp.best0, sp.bad0, sp.theta_in, sp.theta_last};
    mlp_train_tc_kernel<<<kTcCluster, kTcThreads, smem, st>>>(ta, flag);
    mrip_status s = launch_status("mlp train (tensor cores)");
    if (s != MRIP_OK) return s;
    int h[8] = {0};
    e = cudaMemcpyAsync(h, base, 32, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // also: the host schedule dies at return
    if (e != cudaSuccess) return cuda_status(e, "mlp train (tensor cores)");
    if (h[4]) return fail(MRIP_ECUDA, "mlp train: a tensor-core MMA did not complete in time");
    if (info) {
        info->epochs_run = h[0];
        info->best_epoch = h[1];
        info->steps = h[2];
    }
    return MRIP_OK;
}

mrip_status mlp_forward(const float* theta, int d_in, const float* X, long long n, float* yhat, cudaStream_t st) {
    if (n == 0) return MRIP_OK;
    mlp_forward_kernel<<<ceil_div_u(n, 128), 128, 0, st>>>(theta, d_in, X, n, yhat);
    return launch_status("mlp forward");
}

mrip_status cv_reduce(const double* y, const double* g, long long n, const double* gc, long long m, int n_dp,
                      double* out, cudaStream_t st) {
    if (n_dp == 0) return MRIP_OK;
    cv_reduce_kernel<<<n_dp, kCvThreads, 0, st>>>(y, g, n, gc, m, out);
    return launch_status("cv reduce");
}

}  // namespace mrip

using namespace mrip;

extern "C" int64_t mrip_mlp_param_count(int32_t d_in) { return d_in >= 1 && d_in <= 8 ? n_params(d_in) : -1; }

extern "C" mrip_status mrip_mlp_init(int32_t d_in, uint64_t seed, float* d_theta, void* stream) {
    if (d_in < 1 || d_in > kMaxIn) return fail(MRIP_EINVAL, "mrip_mlp_init: d_in in 1..8");
    if (!d_theta) return fail(MRIP_EINVAL, "mrip_mlp_init: null theta");
    return mlp_init(d_in, seed, d_theta, static_cast<cudaStream_t>(stream));
}

extern "C" mrip_status mrip_mlp_forward(const float* d_theta, int32_t d_in, const float* d_x, int64_t n,
                                        float* d_yhat, void* stream) {
    if (d_in < 1 || d_in > kMaxIn || n < 0) return fail(MRIP_EINVAL, "mrip_mlp_forward: d_in in 1..8, n >= 0");
    if (n > 0 && (!d_theta || !d_x || !d_yhat)) return fail(MRIP_EINVAL, "mrip_mlp_forward: null pointer");
    return mlp_forward(d_theta, d_in, d_x, n, d_yhat, static_cast<cudaStream_t>(stream));
}

extern "C" mrip_status mrip_mlp_loss_grad(const float* d_theta, int32_t d_in, const float* d_x, const float* d_y,
                                          int64_t n, const int64_t* d_idx, int64_t B, float* d_grad,
                                          float* d_loss, void* stream) {
    if (d_in < 1 || d_in > kMaxIn || n < 1 || B < 1 || (!d_idx && B > n))
        return fail(MRIP_EINVAL, "mrip_mlp_loss_grad: d_in in 1..8, 1 <= B (<= n without idx)");
    if (!d_theta || !d_x || !d_y || !d_grad) return fail(MRIP_EINVAL, "mrip_mlp_loss_grad: null pointer");
    const size_t need = mlp_grad_partial_floats(d_in, B) * sizeof(float);
    float* partial = static_cast<float*>(scratch(need, 2));
    if (!partial) return fail(MRIP_ENOMEM, "mrip_mlp_loss_grad: scratch allocation failed");
    return mlp_step(d_theta, d_in, d_x, n, d_y, d_idx, 0, 0, 0, 0, B, partial, d_grad, d_loss, nullptr,
                    nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

extern "C" mrip_status mrip_adam_step(float* d_theta, float* d_m, float* d_v, const float* d_grad, int64_t n,
                                      int64_t t, float lr, float beta1, float beta2, float eps, void* stream) {
    if (n < 0 || t < 1) return fail(MRIP_EINVAL, "mrip_adam_step: n >= 0, t >= 1");
    if (n == 0) return MRIP_OK;
    if (!d_theta || !d_m || !d_v || !d_grad) return fail(MRIP_EINVAL, "mrip_adam_step: null pointer");
    const float bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(t)));
    const float bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(t)));
    adam_kernel<<<ceil_div_u(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_theta, d_m, d_v, d_grad, n,
                                                                                  lr, beta1, beta2, eps, bc1, bc2);
    return launch_status("mrip_adam_step");
}

extern "C" mrip_status mrip_mlp_train(int32_t d_in, const float* d_x, const float* d_y, int64_t n,
                                      const float* d_xv, const float* d_yv, int64_t n_val,
                                      const mrip_train_params* prm, float* d_theta, const float* d_m_in,
                                      const float* d_v_in, float* d_losses, float* d_grad, float* d_m,
                                      float* d_v, float* d_val_losses, int32_t* info_out, void* stream) {
    if (d_in < 1 || d_in > kMaxIn || n < 1 || n_val < 0 || !prm)
        return fail(MRIP_EINVAL, "mrip_mlp_train: d_in in 1..8, n >= 1, n_val >= 0, params");
    if (prm->batch < 1 || prm->epochs < 1 || prm->epoch0 < 0 || prm->patience < 0 || prm->max_steps < 0 ||
        !(prm->lr > 0.0f) ||
        !(prm->beta1 >= 0.0f && prm->beta1 < 1.0f) || !(prm->beta2 >= 0.0f && prm->beta2 < 1.0f) ||
        !(prm->eps > 0.0f))
        return fail(MRIP_EINVAL, "mrip_mlp_train: batch, epochs >= 1, patience, max_steps >= 0, lr, eps > 0, "
                                 "beta1, beta2 in [0, 1)");
    if (n > 0x7FFFFFFFll || n_val > 0x7FFFFFFFll) return fail(MRIP_EINVAL, "mrip_mlp_train: n, n_val < 2^31");
    if (!d_x || !d_y || !d_theta || (n_val > 0 && (!d_xv || !d_yv)))
        return fail(MRIP_EINVAL, "mrip_mlp_train: null pointer");
    TrainSpec sp{};
    sp.d_in = d_in;
    sp.X = d_x;
    sp.Y = d_y;
    sp.n = n;
    sp.Xv = n_val > 0 ? d_xv : nullptr;
    sp.Yv = n_val > 0 ? d_yv : nullptr;
    sp.n_val = n_val;
    sp.B = prm->batch;
    sp.epochs = prm->epochs;
    sp.epoch0 = prm->epoch0;
    sp.m_in = d_m_in;
    sp.v_in = d_v_in;
    sp.max_steps = prm->max_steps;
    sp.patience = prm->patience;
    sp.order_seed = prm->order_seed;
    sp.lr = prm->lr;
    sp.beta1 = prm->beta1;
    sp.beta2 = prm->beta2;
    sp.eps = prm->eps;
    sp.theta = d_theta;
    sp.losses = d_losses;
    sp.grad = d_grad;
    sp.m_out = d_m;
    sp.v_out = d_v;
    sp.val_losses = d_val_losses;
    TrainInfo info{};
    mrip_status s = mlp_train(sp, &info, static_cast<cudaStream_t>(stream));
    if (s == MRIP_OK && info_out) {
        info_out[0] = info.epochs_run;
        info_out[1] = info.best_epoch;
        info_out[2] = info.steps;
    }
    return s;
}

extern "C" mrip_status mrip_cv_reduce(const double* d_y, const double* d_g, int64_t n, const double* d_gc,
                                      int64_t m, int32_t n_dp, double* d_out, void* stream) {
    if (n < 3 || m < 2 || n_dp < 0) return fail(MRIP_EINVAL, "mrip_cv_reduce: n >= 3, m >= 2, n_dp >= 0");
    if (n_dp > 0 && (!d_y || !d_g || !d_gc || !d_out)) return fail(MRIP_EINVAL, "mrip_cv_reduce: null pointer");
    return cv_reduce(d_y, d_g, n, d_gc, m, n_dp, d_out, static_cast<cudaStream_t>(stream));
}

MRIP_DEBUG_UNIT(mlp)
