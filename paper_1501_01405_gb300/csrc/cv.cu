// Learned control variate driver (mrip_run_cv).  The paper's estimator is
// the replication mean with a Student-t interval (Section 1); this driver
// runs it unchanged as the plain estimator and, beside it:
//   1. gathers each replication's early-window features (tandem: lambda,
//      mu1..3 and the means of the first `window` gaps and services; forest
//      fire: log10 p_grow, log10 p_lightning and the mean burning fraction of
//      the four quarters of the first `window` steps) and its output Y;
//   2. trains the network on the first n_fit of the n_train = ceil(train_frac
//      n) training replications of every design point with the tensor-core
//      kernel (inputs and target standardised by the fit set's FP64 mean and
//      population std; Adam; epoch order pi(i) = (a i + b) mod n from stream
//      tag 4), the other n_val = ceil(val_frac n_train) being the validation
//      set of the early stop;
//   3. estimates rho^2, the pooled within-design-point squared correlation
//      of Y and the prediction g on the validation replications (each design
//      point's deviations scaled by its fit-set standard deviations, so all
//      design points weigh the same), sizes the
//      control runs from it (the control mean may add a tenth to the
//      residual variance) and, with the gate on, declines the control
//      variate when its predicted variance at this n is not below the plain
//      estimator's;
//   4. predicts g for the held-out replications and for M control runs per
//      design point -- replications n .. n + M - 1 of the same streams,
//      simulated only for the early window;
//   5. reduces per design point: beta = Cov(Y, g)/Var(g),
//      Y_cv = mean(Y) - beta (mean(g) - mean(g_ctrl)),
//      Var = s_r^2 / n + beta^2 Var(g_ctrl) / M, t on n - 2 degrees of freedom.
#include <algorithm>
#include <cmath>
#include <limits>
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
    if (!MRIP_CHECK(r0 + r < n_reps && j < src_plane, 501, i)) return;
    for (int k = 0; k < d; ++k) dst[k * n_out + i] = src[k * src_plane + j];
}

// Forest-fire features of n_items replications (6 planes).
__global__ void ff_features(const int32_t* __restrict__ counts, int n_steps, int window,
                            const double* __restrict__ dps, long long n_reps, long long n_items,
                            double cells, double* __restrict__ feat) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n_items) return;
    if (!MRIP_CHECK(window >= 0 && window <= n_steps, 502, window)) return;
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

// Per design point (one thread each): the within-design-point sums S_yg,
// S_yy, S_gg of its n validation pairs (y, g) about their means, each
// deviation divided by the design point's population standard deviation of
// y (or g) over its n_fit fit replications, so that every design point
// weighs the same whatever its variance; a design point whose fit y or g is
// constant contributes nothing (FP64, two passes each).
__global__ void within_dp_sums(const double* __restrict__ y, const double* __restrict__ g, long long n,
                               const double* __restrict__ yf, const double* __restrict__ gf, long long n_fit,
                               int n_dp, double* __restrict__ out) {
    const int dp = blockIdx.x * blockDim.x + threadIdx.x;
    if (dp >= n_dp) return;
    auto mean = [](const double* a, long long k) {
        double s = 0.0;
        for (long long i = 0; i < k; ++i) s += a[i];
        return s / static_cast<double>(k);
    };
    auto pstd = [](const double* a, long long k, double m) {
        double s = 0.0;
        for (long long i = 0; i < k; ++i) s += (a[i] - m) * (a[i] - m);
        return sqrt(s / static_cast<double>(k));
    };
    const double* yfr = yf + dp * n_fit;
    const double* gfr = gf + dp * n_fit;
    const double sy = pstd(yfr, n_fit, mean(yfr, n_fit)), sg = pstd(gfr, n_fit, mean(gfr, n_fit));
    double syg = 0.0, syy = 0.0, sgg = 0.0;
    if (sy > 0.0 && sg > 0.0) {
        const double* yr = y + dp * n;
        const double* gr = g + dp * n;
        const double ym = mean(yr, n), gm = mean(gr, n);
        for (long long i = 0; i < n; ++i) {
            const double dy = (yr[i] - ym) / sy, dg = (gr[i] - gm) / sg;
            syg += dy * dg;
            syy += dy * dy;
            sgg += dg * dg;
        }
    }
    out[3 * dp] = syg;
    out[3 * dp + 1] = syy;
    out[3 * dp + 2] = sgg;
}

unsigned blocks(long long n) { return ceil_div_u(n, kT); }

// Control runs per design point for a pooled validation rho^2: the control
// mean's term beta^2 Var(g_ctrl) / M ~ rho^2 sigma^2 / M at most a tenth of
// the residual term (1 - rho^2) sigma^2 / n_held; [2, 100 n_held].
long long control_runs(double rho2, long long n_held) {
    if (!(rho2 >= 0.0)) return 10 * n_held;  // no validation: the fixed default
    const double r = rho2 > 0.999999 ? 0.999999 : rho2;
    double m = std::ceil(static_cast<double>(n_held) * r / (0.1 * (1.0 - r)));
    const double cap = 100.0 * static_cast<double>(n_held);
    if (m > cap) m = cap;
    return m < 2.0 ? 2 : static_cast<long long>(m);
}

struct PhaseTimer {
    cudaEvent_t ev[6] = {nullptr};
    int n = 0;
    cudaStream_t st;
    explicit PhaseTimer(cudaStream_t s) : st(s) {
        for (auto& e : ev) cudaEventCreate(&e);
    }
    ~PhaseTimer() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
    void mark() {
        if (n < 6) cudaEventRecord(ev[n++], st);
    }
    double ms(int a, int b) const {
        if (b >= n) return 0.0;
        float t = 0.0f;
        cudaEventSynchronize(ev[b]);
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
};

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
                        const mrip_cv_params* p, mrip_stat* plain_out, mrip_cv_stat* cv_out, mrip_cv_report* rep) {
    if (m->kind != MRIP_TANDEM3 && m->kind != MRIP_FOREST_FIRE)
        return fail(MRIP_EUNSUPPORTED, "mrip_run_cv: control variates exist for TANDEM3 and FOREST_FIRE");
    if (!(p->train_frac > 0.0 && p->train_frac < 1.0) || !(p->val_frac >= 0.0 && p->val_frac < 1.0) ||
        p->epochs < 1 || p->batch < 1 || p->patience < 0 || (p->m_ctrl != 0 && p->m_ctrl < 2) ||
        !(p->conf > 0.0 && p->conf < 1.0) || !(p->lr > 0.0f))
        return fail(MRIP_EINVAL, "mrip_run_cv: train_frac in (0,1), val_frac in [0,1), epochs, batch >= 1, "
                                 "patience >= 0, m_ctrl 0 or >= 2, conf in (0,1)");
    const long long n_train = static_cast<long long>(std::ceil(p->train_frac * static_cast<double>(n_reps)));
    const long long n_held = n_reps - n_train;
    const long long n_val =
        p->val_frac > 0.0 ? static_cast<long long>(std::ceil(p->val_frac * static_cast<double>(n_train))) : 0;
    const long long n_fit = n_train - n_val;
    if (n_fit < 1 || n_held < 3)
        return fail(MRIP_EINVAL, "mrip_run_cv: need >= 1 fit and >= 3 held-out replications");
    const long long m_cap = 100 * n_held;  // the most control runs the sizing asks for
    if (n_reps + std::max<long long>(p->m_ctrl, m_cap) > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_run_cv: replication indices < 2^32");
    const bool tandem = m->kind == MRIP_TANDEM3;
    const int d_in = tandem ? 8 : 6;
    const long long window = tandem ? m->tandem.window : m->ff.window;
    if (!tandem && window < 4) return fail(MRIP_EINVAL, "mrip_run_cv: forest-fire window must be >= 4 steps");
    cudaStream_t st = m->stream;
    PhaseTimer timer(st);
    mrip_cv_report R{};
    R.val_loss = std::nanf("");
    R.val_rho2 = std::nan("");
    R.var_ratio = std::nan("");
    R.n_val = static_cast<int32_t>(n_val);

    // 1. plain run (the reference estimate and fallback) and its intervals
    timer.mark();
    mrip_status s = mrip_run(m, dps, n_dp, n_reps, seed);
    if (s != MRIP_OK) return s;
    s = mrip_stats(m, p->conf, plain_out);
    if (s != MRIP_OK) return s;
    timer.mark();
    const long long items = static_cast<long long>(n_dp) * n_reps;
    const double cells = tandem ? 0.0 : static_cast<double>(m->ff.L) * m->ff.L;

    auto& B_ = m->cvb;  // the handle's buffers: grown on demand, kept between calls
    DevBuf &feat_all = B_.feat_all, &x_fit = B_.x_fit, &y_fit = B_.y_fit, &x_val = B_.x_val, &y_val = B_.y_val,
           &x_ho = B_.x_ho, &y_ho = B_.y_ho, &ms_dev = B_.ms_dev, &tmp = B_.tmp, &xs_fit = B_.xs_fit,
           &ys_fit = B_.ys_fit, &xs_val = B_.xs_val, &ys_val = B_.ys_val, &xs_ho = B_.xs_ho, &g_val = B_.g_val,
           &g_vald = B_.g_vald, &g_fit = B_.g_fit, &g_fitd = B_.g_fitd, &g_ho = B_.g_ho, &g_hod = B_.g_hod,
           &losses = B_.losses, &val_losses = B_.val_losses, &wsums = B_.wsums, &adam = B_.adam, &c_y = B_.c_y,
           &c_feat = B_.c_feat, &c_counts = B_.c_counts, &xs_c = B_.xs_c, &g_c = B_.g_c, &g_cd = B_.g_cd,
           &out5 = B_.out5;
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

    // 2. fit, validation and held-out sets (replications [0, n_fit), [n_fit,
    //    n_train), [n_train, n_reps) of every design point)
    const long long n_f = static_cast<long long>(n_dp) * n_fit;
    const long long n_v = static_cast<long long>(n_dp) * n_val;
    const long long n_ho = static_cast<long long>(n_dp) * n_held;
    if (!x_fit.ensure(d_in * n_f * sizeof(double)) || !y_fit.ensure(n_f * sizeof(double)) ||
        !xs_fit.ensure(d_in * n_f * sizeof(float)) || !ys_fit.ensure(n_f * sizeof(float)) ||
        !x_ho.ensure(d_in * n_ho * sizeof(double)) || !y_ho.ensure(n_ho * sizeof(double)) ||
        !xs_ho.ensure(d_in * n_ho * sizeof(float)) || !g_ho.ensure(n_ho * sizeof(float)) ||
        !g_hod.ensure(n_ho * sizeof(double)) || !ms_dev.ensure(2 * (d_in + 1) * sizeof(double)))
        return fail(MRIP_ENOMEM, "cv: training buffers");
    if (n_v > 0 && (!x_val.ensure(d_in * n_v * sizeof(double)) || !y_val.ensure(n_v * sizeof(double)) ||
                    !xs_val.ensure(d_in * n_v * sizeof(float)) || !ys_val.ensure(n_v * sizeof(float)) ||
                    !g_val.ensure(n_v * sizeof(float)) || !g_vald.ensure(n_v * sizeof(double)) ||
                    !wsums.ensure(3 * static_cast<size_t>(n_dp) * sizeof(double))))
        return fail(MRIP_ENOMEM, "cv: validation buffers");
    gather_planes<<<blocks(n_f), kT, 0, st>>>(feat_src, items, d_in, n_reps, 0, n_fit, n_f, x_fit.as<double>());
    gather_planes<<<blocks(n_f), kT, 0, st>>>(y_src, items, 1, n_reps, 0, n_fit, n_f, y_fit.as<double>());
    gather_planes<<<blocks(n_ho), kT, 0, st>>>(feat_src, items, d_in, n_reps, n_train, n_held, n_ho, x_ho.as<double>());
    gather_planes<<<blocks(n_ho), kT, 0, st>>>(y_src, items, 1, n_reps, n_train, n_held, n_ho, y_ho.as<double>());
    if (n_v > 0) {
        gather_planes<<<blocks(n_v), kT, 0, st>>>(feat_src, items, d_in, n_reps, n_fit, n_val, n_v,
                                                  x_val.as<double>());
        gather_planes<<<blocks(n_v), kT, 0, st>>>(y_src, items, 1, n_reps, n_fit, n_val, n_v, y_val.as<double>());
    }
    s = launch_status("cv: gather");
    if (s != MRIP_OK) return s;
    std::vector<double> ms(2 * (d_in + 1));
    s = plane_moments(x_fit.as<double>(), d_in, n_f, tmp, ms.data(), ms_dev.as<double>(), st);
    if (s != MRIP_OK) return s;
    s = plane_moments(y_fit.as<double>(), 1, n_f, tmp, ms.data() + 2 * d_in, ms_dev.as<double>() + 2 * d_in, st);
    if (s != MRIP_OK) return s;
    const double* d_ms = ms_dev.as<double>();
    standardize<<<blocks(n_f), kT, 0, st>>>(x_fit.as<double>(), n_f, d_in, d_ms, xs_fit.as<float>());
    standardize<<<blocks(n_f), kT, 0, st>>>(y_fit.as<double>(), n_f, 1, d_ms + 2 * d_in, ys_fit.as<float>());
    standardize<<<blocks(n_ho), kT, 0, st>>>(x_ho.as<double>(), n_ho, d_in, d_ms, xs_ho.as<float>());
    if (n_v > 0) {
        standardize<<<blocks(n_v), kT, 0, st>>>(x_val.as<double>(), n_v, d_in, d_ms, xs_val.as<float>());
        standardize<<<blocks(n_v), kT, 0, st>>>(y_val.as<double>(), n_v, 1, d_ms + 2 * d_in, ys_val.as<float>());
    }
    s = launch_status("cv: standardise");
    if (s != MRIP_OK) return s;

    // 3. training (early stop on the validation set), validation rho^2.
    //    With the gate on, the first ceil(64 / steps per epoch) epochs run
    //    alone (at least 64 Adam steps); a validation rho^2 below a quarter
    //    of the break-even value (with M sized as below, the control variate
    //    needs rho^2 > 1 - n_held / (1.1 n_reps)) then declines at once;
    //    otherwise training resumes from that point (parameters, Adam state,
    //    best validation loss and epochs since) exactly as one run would go on.
    const long long P = mlp_params(d_in);
    const long long B = p->batch;
    const long long spe = (n_f + B - 1) / B;
    const long long n_steps = spe * p->epochs;
    if (!m->cv_theta.ensure(P * sizeof(float)) || !losses.ensure(n_steps * sizeof(float)) ||
        !val_losses.ensure(static_cast<size_t>(p->epochs) * sizeof(float)) ||
        !adam.ensure(5 * P * sizeof(float)))
        return fail(MRIP_ENOMEM, "cv: network buffers");
    float* theta = m->cv_theta.as<float>();
    m->cv_d_in = 0;  // valid again once training succeeded
    s = mlp_init(d_in, p->net_seed, theta, st);
    if (s != MRIP_OK) return s;
    TrainSpec sp{};
    sp.d_in = d_in;
    sp.X = xs_fit.as<float>();
    sp.Y = ys_fit.as<float>();
    sp.n = n_f;
    sp.Xv = n_v > 0 ? xs_val.as<float>() : nullptr;
    sp.Yv = n_v > 0 ? ys_val.as<float>() : nullptr;
    sp.n_val = n_v;
    sp.B = B;
    const int screen_epochs = static_cast<int>(std::min<long long>(p->epochs, (64 + spe - 1) / spe));
    const bool screen_first = p->gate && n_v > 0 && n_val >= 2 && screen_epochs < p->epochs;
    sp.epochs = screen_first ? screen_epochs : p->epochs;
    sp.patience = p->patience;
    sp.order_seed = p->net_seed;
    sp.lr = p->lr;
    sp.beta1 = p->beta1;
    sp.beta2 = p->beta2;
    sp.eps = p->eps;
    sp.theta = theta;
    sp.losses = losses.as<float>();
    sp.val_losses = n_v > 0 ? val_losses.as<float>() : nullptr;
    sp.m_out = adam.as<float>();
    sp.v_out = adam.as<float>() + P;
    sp.theta_last = adam.as<float>() + 4 * P;
    TrainInfo info{};
    s = mlp_train(sp, &info, st);
    if (s != MRIP_OK) return s;
    m->cv_d_in = d_in;
    m->cv_norm = ms;
    int epochs_run = info.epochs_run, best_epoch = info.best_epoch;
    float v_best = std::numeric_limits<float>::infinity();
    if (n_v > 0 && best_epoch > 0) {
        cudaError_t e = cudaMemcpyAsync(&v_best, val_losses.as<float>() + (best_epoch - 1), sizeof(float),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e, "cv: validation loss read");
    }
    // the pooled within-design-point rho^2 of the current network on the
    // validation replications (each design point scaled by its fit set)
    auto validation_rho2 = [&](double& out) -> mrip_status {
        out = std::nan("");
        if (!(n_v > 0 && n_val >= 2)) return MRIP_OK;
        if (!g_fit.ensure(n_f * sizeof(float)) || !g_fitd.ensure(n_f * sizeof(double)))
            return fail(MRIP_ENOMEM, "cv: fit predictions");
        mrip_status r = mlp_forward(theta, d_in, xs_val.as<float>(), n_v, g_val.as<float>(), st);
        if (r == MRIP_OK) r = mlp_forward(theta, d_in, xs_fit.as<float>(), n_f, g_fit.as<float>(), st);
        if (r != MRIP_OK) return r;
        to_double<<<blocks(n_v), kT, 0, st>>>(g_val.as<float>(), n_v, g_vald.as<double>());
        to_double<<<blocks(n_f), kT, 0, st>>>(g_fit.as<float>(), n_f, g_fitd.as<double>());
        within_dp_sums<<<ceil_div_u(n_dp, 128), 128, 0, st>>>(y_val.as<double>(), g_vald.as<double>(), n_val,
                                                             y_fit.as<double>(), g_fitd.as<double>(), n_fit,
                                                             n_dp, wsums.as<double>());
        r = launch_status("cv: validation correlation");
        if (r != MRIP_OK) return r;
        std::vector<double> h(3 * static_cast<size_t>(n_dp));
        cudaError_t e = cudaMemcpyAsync(h.data(), wsums.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e, "cv: validation correlation");
        double syg = 0.0, syy = 0.0, sgg = 0.0;
        for (int32_t d = 0; d < n_dp; ++d) {  // design points in order
            syg += h[3 * d];
            syy += h[3 * d + 1];
            sgg += h[3 * d + 2];
        }
        out = (syy > 0.0 && sgg > 0.0) ? (syg * syg) / (syy * sgg) : 0.0;
        return MRIP_OK;
    };
    double rho2 = std::nan("");
    const double rho2_be = 1.0 - static_cast<double>(n_held) / (1.1 * static_cast<double>(n_reps));
    bool screened = false;
    // a first part that ran to its end (no early stop inside) is screened
    if (screen_first && epochs_run == screen_epochs) {
        s = validation_rho2(rho2);
        if (s != MRIP_OK) return s;
        screened = rho2 >= 0.0 && rho2 < 0.25 * rho2_be;
        if (!screened) {
            const int e0 = epochs_run;
            TrainSpec rest = sp;
            rest.epochs = p->epochs - e0;
            rest.epoch0 = e0;
            rest.theta_in = adam.as<float>() + 4 * P;  // the trajectory, not the kept epoch
            rest.theta_last = nullptr;
            rest.m_in = adam.as<float>();
            rest.v_in = adam.as<float>() + P;
            rest.m_out = adam.as<float>() + 2 * P;
            rest.v_out = adam.as<float>() + 3 * P;
            rest.losses = losses.as<float>() + e0 * spe;
            rest.val_losses = val_losses.as<float>() + e0;
            rest.best0 = v_best;
            rest.bad0 = e0 - best_epoch;
            TrainInfo more{};
            s = mlp_train(rest, &more, st);
            if (s != MRIP_OK) return s;
            epochs_run = e0 + more.epochs_run;
            if (more.best_epoch > 0) best_epoch = e0 + more.best_epoch;
            rho2 = std::nan("");
        }
    }
    if (!screened) {
        s = validation_rho2(rho2);  // of the kept network
        if (s != MRIP_OK) return s;
    }
    long long last0 = 0;  // first step of the last epoch run, in `losses`
    last0 = static_cast<long long>(epochs_run > 0 ? epochs_run - 1 : 0) * spe;
    R.epochs_run = epochs_run;
    R.best_epoch = best_epoch;
    {   // mean minibatch loss of the last epoch run, and the kept epoch's validation loss
        std::vector<float> hl(spe);
        cudaError_t e = cudaMemcpyAsync(hl.data(), losses.as<float>() + last0, spe * sizeof(float),
                                        cudaMemcpyDeviceToHost, st);
        float vl = std::nanf("");
        if (e == cudaSuccess && n_v > 0 && best_epoch > 0)
            e = cudaMemcpyAsync(&vl, val_losses.as<float>() + (best_epoch - 1), sizeof(float),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e, "cv: loss read");
        double acc = 0.0, wsum = 0.0;
        for (long long k = 0; k < spe; ++k) {
            const double w = static_cast<double>((k + 1) * B <= n_f ? B : n_f - k * B);
            acc += w * hl[k];
            wsum += w;
        }
        R.train_loss = static_cast<float>(acc / wsum);
        R.val_loss = vl;
    }
    R.val_rho2 = rho2;
    const long long M = p->m_ctrl > 0 ? p->m_ctrl : control_runs(rho2, n_held);
    if (rho2 >= 0.0)
        R.var_ratio = static_cast<double>(n_reps) *
                      ((1.0 - rho2) / static_cast<double>(n_held) + rho2 / static_cast<double>(M));
    timer.mark();

    if (p->gate && (screened || R.var_ratio >= 1.0)) {  // the plain estimator stays
        R.declined = screened ? 2 : 1;
        R.m_ctrl = 0;
        for (int32_t d = 0; d < n_dp; ++d) {
            mrip_cv_stat& o = cv_out[d];
            o.n = plain_out[d].n;
            o.m = 0;
            o.beta = 0.0;
            o.mean = plain_out[d].mean;
            o.var = plain_out[d].var / static_cast<double>(plain_out[d].n);
            o.half_width = plain_out[d].half_width;
            o.t_crit = plain_out[d].t_crit;
        }
        R.ms_simulate = timer.ms(0, 1);
        R.ms_train = timer.ms(1, 2);
        if (rep) *rep = R;
        return MRIP_OK;
    }
    R.m_ctrl = M;

    // 4. control runs: replications n_reps .. n_reps + M - 1, early window only
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
    standardize<<<blocks(n_c), kT, 0, st>>>(c_feat.as<double>(), n_c, d_in, d_ms, xs_c.as<float>());
    s = launch_status("cv: control standardise");
    if (s != MRIP_OK) return s;
    timer.mark();

    // predictions of the held-out replications and the control runs
    s = mlp_forward(theta, d_in, xs_ho.as<float>(), n_ho, g_ho.as<float>(), st);
    if (s != MRIP_OK) return s;
    s = mlp_forward(theta, d_in, xs_c.as<float>(), n_c, g_c.as<float>(), st);
    if (s != MRIP_OK) return s;
    to_double<<<blocks(n_ho), kT, 0, st>>>(g_ho.as<float>(), n_ho, g_hod.as<double>());
    to_double<<<blocks(n_c), kT, 0, st>>>(g_c.as<float>(), n_c, g_cd.as<double>());
    s = launch_status("cv: predictions");
    if (s != MRIP_OK) return s;
    timer.mark();

    // 5. per-design-point estimator
    s = cv_reduce(y_ho.as<double>(), g_hod.as<double>(), n_held, g_cd.as<double>(), M, n_dp, out5.as<double>(), st);
    if (s != MRIP_OK) return s;
    std::vector<double> h(5 * static_cast<size_t>(n_dp));
    cudaError_t e = cudaMemcpyAsync(h.data(), out5.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
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
    timer.mark();
    R.ms_simulate = timer.ms(0, 1);
    R.ms_train = timer.ms(1, 2);
    R.ms_control = timer.ms(2, 3);
    R.ms_infer = timer.ms(3, 4);
    R.ms_estimate = timer.ms(4, 5);
    if (rep) *rep = R;
    return MRIP_OK;
}

}  // namespace mrip

MRIP_DEBUG_UNIT(cv)
