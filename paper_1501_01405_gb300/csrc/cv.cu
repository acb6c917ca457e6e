// Learned control variate driver (mrip_run_cv).  The paper's estimator is
// the replication mean with a Student-t interval (Section 1); this driver
// runs it unchanged as the plain estimator and, beside it:
//   1. gathers each replication's early-window features (tandem: lambda,
//      mu1..3 and the means of the first `window` gaps and services; forest
//      fire: log10 p_grow, log10 p_lightning and the mean burning fraction of
//      the four quarters of the first `window` steps) and its output Y;
//   2. trains the network on the first ceil(train_frac n) replications of
//      every design point with the engine's kernels (inputs and target
//      standardised by the training set's FP64 mean and population std;
//      Adam; epoch order pi(i) = (a i + b) mod n from stream tag 4);
//   3. predicts g for the held-out replications and for m_ctrl control runs
//      per design point -- replications n .. n + m_ctrl - 1 of the same
//      streams, simulated only for the early window;
//   4. reduces per design point: beta = Cov(Y, g)/Var(g),
//      Y_cv = mean(Y) - beta (mean(g) - mean(g_ctrl)),
//      Var = s_r^2 / n + beta^2 Var(g_ctrl) / m, t on n - 2 degrees of freedom.
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "model.cuh"

namespace mrip {
namespace {

constexpr int kT = 256;

// dst[k][dp n_sel + r] = src[k][dp n_reps + r0 + r]
__global__ void gather_planes(const double* __restrict__ src, long long src_plane, int d, long long n_reps,
                              long long r0, long long n_sel, long long n_out, double* __restrict__ dst) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n_out) return;
    const long long dp = i / n_sel, r = i - dp * n_sel;
    const long long j = dp * n_reps + r0 + r;
    for (int k = 0; k < d; ++k) dst[k * n_out + i] = src[k * src_plane + j];
}

// Forest-fire features of n_items replications (6 planes).
__global__ void ff_features(const int32_t* __restrict__ counts, int n_steps, int window,
                            const double* __restrict__ dps, long long n_reps, long long n_items,
                            double cells, double* __restrict__ feat) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n_items) return;
    const long long dp = i / n_reps;
    feat[i] = log10(fmax(dps[2 * dp], 1e-30));
    feat[n_items + i] = log10(fmax(dps[2 * dp + 1], 1e-30));
    const int32_t* c = counts + i * n_steps;
    for (int q = 0; q < 4; ++q) {
        const int a = (q * window) / 4, b = ((q + 1) * window) / 4;
        long long s = 0;
        for (int t = a; t < b; ++t) s += c[t];
        feat[(2 + q) * n_items + i] =
            b > a ? static_cast<double>(s) / (static_cast<double>(b - a) * cells) : 0.0;
    }
}

// out[k][i] = fp32((x[k][i] - mean_k) / std_k)
__global__ void standardize(const double* __restrict__ x, long long n, int d, const double* __restrict__ ms,
                            float* __restrict__ out) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < d; ++k) out[k * n + i] = static_cast<float>((x[k * n + i] - ms[2 * k]) / ms[2 * k + 1]);
}

__global__ void to_double(const float* __restrict__ a, long long n, double* __restrict__ b) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i < n) b[i] = static_cast<double>(a[i]);
}

unsigned blocks(long long n) { return ceil_div_u(n, kT); }

// Epoch order (a, b) for n samples: block (0, epoch) of tag 4, rep 0, dp 0.
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

// Per-plane FP64 mean and population std (zero std -> 1) of d planes of n.
mrip_status plane_moments(const double* x, int d, long long n, DevBuf& tmp, double* host_ms, double* dev_ms,
                          cudaStream_t st) {
    const size_t head = static_cast<size_t>(d) * 3 * sizeof(double);
    if (!tmp.ensure(head + stats_scratch_bytes(d, n))) return fail(MRIP_ENOMEM, "cv: moments");
    mrip_status s = stats_reduce_double(x, d, n, tmp.as<double>(), st, tmp.as<double>() + 3 * d);
    if (s != MRIP_OK) return s;
    std::vector<double> h(3 * d);
    cudaError_t e = cudaMemcpyAsync(h.data(), tmp.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "cv: moments");
    for (int k = 0; k < d; ++k) {
        const double mean = h[3 * k + 1];
        double sd = std::sqrt(h[3 * k + 2] / h[3 * k]);
        if (!(sd > 0.0)) sd = 1.0;
        host_ms[2 * k] = mean;
        host_ms[2 * k + 1] = sd;
    }
    if (dev_ms) {
        e = cudaMemcpyAsync(dev_ms, host_ms, 2 * d * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e, "cv: moments upload");
    }
    return MRIP_OK;
}

}  // namespace

mrip_status run_cv_impl(mrip_model* m, const double* dps, int32_t n_dp, int64_t n_reps, uint64_t seed,
                        const mrip_cv_params* p, mrip_stat* plain_out, mrip_cv_stat* cv_out, float* loss_out) {
    if (m->kind != MRIP_TANDEM3 && m->kind != MRIP_FOREST_FIRE)
        return fail(MRIP_EUNSUPPORTED, "mrip_run_cv: control variates exist for TANDEM3 and FOREST_FIRE");
    if (!(p->train_frac > 0.0 && p->train_frac < 1.0) || p->epochs < 1 || p->batch < 1 || p->m_ctrl < 2 ||
        !(p->conf > 0.0 && p->conf < 1.0) || !(p->lr > 0.0f))
        return fail(MRIP_EINVAL, "mrip_run_cv: train_frac in (0,1), epochs, batch >= 1, m_ctrl >= 2, conf in (0,1)");
    const long long n_train = static_cast<long long>(std::ceil(p->train_frac * static_cast<double>(n_reps)));
    const long long n_held = n_reps - n_train;
    if (n_train < 1 || n_held < 3) return fail(MRIP_EINVAL, "mrip_run_cv: need >= 1 training and >= 3 held-out replications");
    if (n_reps + p->m_ctrl > 0x100000000ll) return fail(MRIP_EINVAL, "mrip_run_cv: replication indices < 2^32");
    const bool tandem = m->kind == MRIP_TANDEM3;
    const int d_in = tandem ? 8 : 6;
    const long long window = tandem ? m->tandem.window : m->ff.window;
    if (!tandem && window < 4) return fail(MRIP_EINVAL, "mrip_run_cv: forest-fire window must be >= 4 steps");

    // 1. plain run (the reference estimate and fallback) and its intervals
    mrip_status s = mrip_run(m, dps, n_dp, n_reps, seed);
    if (s != MRIP_OK) return s;
    s = mrip_stats(m, p->conf, plain_out);
    if (s != MRIP_OK) return s;
    cudaStream_t st = m->stream;
    const long long items = static_cast<long long>(n_dp) * n_reps;
    const double cells = tandem ? 0.0 : static_cast<double>(m->ff.L) * m->ff.L;

    DevBuf feat_all, y_all_ff, x_tr, y_tr, x_ho, y_ho, ms_dev, tmp, xs_tr, ys_tr, xs_ho, g_ho, g_hod, theta, sched,
        losses, c_y, c_feat, c_counts, xs_c, g_c, g_cd, out5;
    const double* feat_src;  // d_in planes of `items`
    const double* y_src;     // items
    if (tandem) {
        feat_src = m->out1.as<double>();
        y_src = m->out0.as<double>();
    } else {
        if (!feat_all.ensure(static_cast<size_t>(d_in) * items * sizeof(double)))
            return fail(MRIP_ENOMEM, "cv: features");
        ff_features<<<blocks(items), kT, 0, st>>>(m->out0.as<int32_t>(), m->ff.n_steps, static_cast<int>(window),
                                                  m->dps.as<double>(), n_reps, items, cells, feat_all.as<double>());
        s = launch_status("cv: forest-fire features");
        if (s != MRIP_OK) return s;
        feat_src = feat_all.as<double>();
        y_src = m->out1.as<double>();
    }

    // 2. training and held-out sets
    const long long n_tr = static_cast<long long>(n_dp) * n_train;
    const long long n_ho = static_cast<long long>(n_dp) * n_held;
    if (!x_tr.ensure(d_in * n_tr * sizeof(double)) || !y_tr.ensure(n_tr * sizeof(double)) ||
        !x_ho.ensure(d_in * n_ho * sizeof(double)) || !y_ho.ensure(n_ho * sizeof(double)) ||
        !xs_tr.ensure(d_in * n_tr * sizeof(float)) || !ys_tr.ensure(n_tr * sizeof(float)) ||
        !xs_ho.ensure(d_in * n_ho * sizeof(float)) || !g_ho.ensure(n_ho * sizeof(float)) ||
        !g_hod.ensure(n_ho * sizeof(double)) || !ms_dev.ensure(2 * (d_in + 1) * sizeof(double)))
        return fail(MRIP_ENOMEM, "cv: training buffers");
    gather_planes<<<blocks(n_tr), kT, 0, st>>>(feat_src, items, d_in, n_reps, 0, n_train, n_tr, x_tr.as<double>());
    gather_planes<<<blocks(n_tr), kT, 0, st>>>(y_src, items, 1, n_reps, 0, n_train, n_tr, y_tr.as<double>());
    gather_planes<<<blocks(n_ho), kT, 0, st>>>(feat_src, items, d_in, n_reps, n_train, n_held, n_ho, x_ho.as<double>());
    gather_planes<<<blocks(n_ho), kT, 0, st>>>(y_src, items, 1, n_reps, n_train, n_held, n_ho, y_ho.as<double>());
    s = launch_status("cv: gather");
    if (s != MRIP_OK) return s;
    std::vector<double> ms(2 * (d_in + 1));
    s = plane_moments(x_tr.as<double>(), d_in, n_tr, tmp, ms.data(), ms_dev.as<double>(), st);
    if (s != MRIP_OK) return s;
    s = plane_moments(y_tr.as<double>(), 1, n_tr, tmp, ms.data() + 2 * d_in, ms_dev.as<double>() + 2 * d_in, st);
    if (s != MRIP_OK) return s;
    standardize<<<blocks(n_tr), kT, 0, st>>>(x_tr.as<double>(), n_tr, d_in, ms_dev.as<double>(), xs_tr.as<float>());
    standardize<<<blocks(n_tr), kT, 0, st>>>(y_tr.as<double>(), n_tr, 1, ms_dev.as<double>() + 2 * d_in,
                                             ys_tr.as<float>());
    standardize<<<blocks(n_ho), kT, 0, st>>>(x_ho.as<double>(), n_ho, d_in, ms_dev.as<double>(), xs_ho.as<float>());
    s = launch_status("cv: standardise");
    if (s != MRIP_OK) return s;

    // 3. training
    const long long P = mlp_params(d_in);
    const long long B = p->batch;
    const long long steps_per_epoch = (n_tr + B - 1) / B;
    const long long n_steps = steps_per_epoch * p->epochs;
    // per epoch the affine order (a, b), per step Adam's bias corrections,
    // computed here in double and rounded to float as the stage entry points
    // take them; then all epochs in one cluster launch
    std::vector<unsigned long long> ab(2 * static_cast<size_t>(p->epochs));
    for (int ep = 0; ep < p->epochs; ++ep)
        epoch_affine(p->net_seed, ep, static_cast<unsigned long long>(n_tr), ab[2 * ep], ab[2 * ep + 1]);
    std::vector<float> bc(2 * static_cast<size_t>(n_steps));
    for (long long k = 1; k <= n_steps; ++k) {
        bc[2 * (k - 1)] = static_cast<float>(1.0 - std::pow(static_cast<double>(p->beta1), static_cast<double>(k)));
        bc[2 * (k - 1) + 1] =
            static_cast<float>(1.0 - std::pow(static_cast<double>(p->beta2), static_cast<double>(k)));
    }
    const size_t ab_bytes = ab.size() * sizeof(unsigned long long);
    if (!theta.ensure(P * sizeof(float)) || !losses.ensure(n_steps * sizeof(float)) ||
        !sched.ensure(ab_bytes + bc.size() * sizeof(float)))
        return fail(MRIP_ENOMEM, "cv: network buffers");
    cudaError_t e = cudaMemcpyAsync(sched.p, ab.data(), ab_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char*>(sched.p) + ab_bytes, bc.data(), bc.size() * sizeof(float),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    if (e != cudaSuccess) return cuda_status(e, "cv: training schedule");
    s = mlp_init(d_in, p->net_seed, theta.as<float>(), st);
    if (s != MRIP_OK) return s;
    s = mlp_train_tc(d_in, xs_tr.as<float>(), ys_tr.as<float>(), n_tr, B, p->epochs, sched.as<unsigned long long>(),
                  reinterpret_cast<const float*>(static_cast<char*>(sched.p) + ab_bytes), p->lr, p->beta1,
                  p->beta2, p->eps, theta.as<float>(), losses.as<float>(), st);
    if (s != MRIP_OK) return s;
    if (loss_out) {
        std::vector<float> hl(steps_per_epoch);
        e = cudaMemcpyAsync(hl.data(), losses.as<float>() + (n_steps - steps_per_epoch),
                            steps_per_epoch * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e, "cv: loss read");
        double acc = 0.0, wsum = 0.0;
        for (long long k = 0; k < steps_per_epoch; ++k) {
            const double w = static_cast<double>((k + 1) * B <= n_tr ? B : n_tr - k * B);
            acc += w * hl[k];
            wsum += w;
        }
        *loss_out = static_cast<float>(acc / wsum);
    }

    // 4. held-out predictions
    s = mlp_forward(theta.as<float>(), d_in, xs_ho.as<float>(), n_ho, g_ho.as<float>(), st);
    if (s != MRIP_OK) return s;
    to_double<<<blocks(n_ho), kT, 0, st>>>(g_ho.as<float>(), n_ho, g_hod.as<double>());

    // 5. control runs: replications n_reps .. n_reps + m_ctrl - 1, early window only
    const long long M = p->m_ctrl;
    const long long n_c = static_cast<long long>(n_dp) * M;
    if (!c_feat.ensure(d_in * n_c * sizeof(double)) || !c_y.ensure(n_c * sizeof(double)) ||
        !xs_c.ensure(d_in * n_c * sizeof(float)) || !g_c.ensure(n_c * sizeof(float)) ||
        !g_cd.ensure(n_c * sizeof(double)) || !out5.ensure(5 * static_cast<size_t>(n_dp) * sizeof(double)))
        return fail(MRIP_ENOMEM, "cv: control-run buffers");
    if (tandem) {
        s = mrip_tandem3_simulate(m->dps.as<double>(), n_dp, n_reps, M, window, window, seed, 0, MRIP_MAP_THREAD,
                                  c_y.as<double>(), c_feat.as<double>(), st);
    } else {
        if (!c_counts.ensure(static_cast<size_t>(n_c) * window * sizeof(int32_t)))
            return fail(MRIP_ENOMEM, "cv: control-run counts");
        s = forest_fire_launch(m->dps.as<double>(), n_dp, n_reps, M, m->ff.L, static_cast<int32_t>(window),
                               m->ff.density, seed, nullptr, c_counts.as<int32_t>(), nullptr, nullptr, st);
        if (s == MRIP_OK) {
            ff_features<<<blocks(n_c), kT, 0, st>>>(c_counts.as<int32_t>(), static_cast<int>(window),
                                                   static_cast<int>(window), m->dps.as<double>(), M, n_c, cells,
                                                   c_feat.as<double>());
            s = launch_status("cv: control features");
        }
    }
    if (s != MRIP_OK) return s;
    standardize<<<blocks(n_c), kT, 0, st>>>(c_feat.as<double>(), n_c, d_in, ms_dev.as<double>(), xs_c.as<float>());
    s = mlp_forward(theta.as<float>(), d_in, xs_c.as<float>(), n_c, g_c.as<float>(), st);
    if (s != MRIP_OK) return s;
    to_double<<<blocks(n_c), kT, 0, st>>>(g_c.as<float>(), n_c, g_cd.as<double>());

    // 6. per-design-point estimator
    s = cv_reduce(y_ho.as<double>(), g_hod.as<double>(), n_held, g_cd.as<double>(), M, n_dp, out5.as<double>(), st);
    if (s != MRIP_OK) return s;
    std::vector<double> h(5 * static_cast<size_t>(n_dp));
    e = cudaMemcpyAsync(h.data(), out5.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "cv: result read");
    const double tc = t_critical(p->conf, n_held - 2);
    for (int32_t d = 0; d < n_dp; ++d) {
        mrip_cv_stat& o = cv_out[d];
        o.n = n_held;
        o.m = M;
        o.beta = h[5 * d];
        o.mean = h[5 * d + 1];
        o.var = h[5 * d + 2];
        o.t_crit = tc;
        o.half_width = tc * std::sqrt(o.var);
    }
    return MRIP_OK;
}

}  // namespace mrip
