// Private declarations shared by the engine's translation units: the model
// handle, its device buffers and the internal launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <limits>
#include <vector>

#include "../../include/mrip.h"

struct Plan {
    int mapping = MRIP_MAP_AUTO;
    int warps_per_cta = 0;
    int ctas_per_sm = 0;
    int chunk = 0;
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool ensure(size_t bytes) {
        if (bytes <= cap && p) return true;
        if (p) {
            cudaFree(p);
            p = nullptr;
            cap = 0;
        }
        if (cudaMalloc(&p, bytes < 256 ? 256 : bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        cap = bytes < 256 ? 256 : bytes;
        return true;
    }
    template <typename T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

struct mrip_model {
    int kind = 0;
    mrip_mm1_params mm1{};
    mrip_tandem3_params tandem{};
    mrip_forest_fire_params ff{};
    mrip_walk_params walk{};
    cudaStream_t stream = nullptr;
    Plan plan;
    DevBuf dps, out0, out1, nmm2, walk_tab, ticket, spart;
    std::vector<double> host_dps;
    int32_t n_dp = 0;
    int64_t n_reps = 0;
    int64_t rep0 = 0;  // replication index of output column 0 (mrip_run_range)
    bool has_run = false;
    // the control variate's working buffers (kept between mrip_run_cv calls)
    // and the network of the last one
    struct {
        DevBuf feat_all, x_fit, y_fit, x_val, y_val, x_ho, y_ho, ms_dev, tmp, xs_fit, ys_fit, xs_val, ys_val, xs_ho,
            g_val, g_vald, g_fit, g_fitd, g_ho, g_hod, losses, val_losses, wsums, adam, c_y, c_feat, c_counts, xs_c,
            g_c, g_cd, out5;
    } cvb;
    DevBuf cv_theta;
    std::vector<double> cv_norm;
    int cv_d_in = 0;
    // graph cache
    cudaGraphExec_t exec = nullptr;
    int32_t g_n_dp = -1;
    int64_t g_n_reps = -1;
    int64_t g_rep0 = -1;
    uint64_t g_seed = 0;
    Plan g_plan;
    ~mrip_model() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

namespace mrip {
int dp_dim(int kind);
mrip_status check_dps(int kind, const double* dps, int32_t n_dp);
mrip_status walk_launch(const int32_t* d_radius_by_pos, const int32_t* d_dp_by_pos, int32_t n_dp,
                        int64_t rep0, int64_t n_reps, uint64_t seed, int64_t max_steps, int mapping,
                        int32_t warps_per_cta, int32_t ctas_per_sm, int32_t chunk, int64_t* d_tau,
                        unsigned long long* d_ticket, cudaStream_t st);
mrip_status walk_tables(const double* radii, int32_t n_dp, std::vector<int32_t>& r_by_pos,
                        std::vector<int32_t>& dp_by_pos);
mrip_status stats_reduce_double(const double* d_x, int32_t n_dp, int64_t n_reps, double* d_out,
                                cudaStream_t st, double* d_part);
mrip_status stats_reduce_int64(const int64_t* d_x, int32_t n_dp, int64_t n_reps, double* d_out,
                               cudaStream_t st, double* d_part);
// Bytes of the slice-partials buffer stats_reduce_* needs (0: none).
size_t stats_scratch_bytes(int32_t n_dp, int64_t n_reps);
double t_critical(double conf, long long df);
mrip_status forest_fire_launch(const double* d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                               int32_t L, int32_t n_steps, double density, uint64_t seed,
                               const uint8_t* d_init, int32_t* d_counts, double* d_scalar,
                               uint8_t* d_final, cudaStream_t st);
mrip_status run_cv_impl(mrip_model* m, const double* dps, int32_t n_dp, int64_t n_reps,
                        uint64_t seed, const mrip_cv_params* p, mrip_stat* plain_out,
                        mrip_cv_stat* cv_out, mrip_cv_report* report);
// network stages (mlp.cu)
long long mlp_params(int d_in);
mrip_status mlp_init(int d_in, uint64_t seed, float* theta, cudaStream_t st);
size_t mlp_grad_partial_floats(int d_in, long long B);
mrip_status mlp_step(const float* theta_in, int d_in, const float* X, long long n_total, const float* Y,
                     const int64_t* idx, unsigned long long a, unsigned long long b, unsigned long long n_perm,
                     long long off, long long B, float* partial, float* grad, float* loss, float* theta,
                     float* m, float* v, const float* adam, cudaStream_t st);
// One training run on the tensor cores (mlp.cu): inputs and outputs as
// mrip_mlp_train.
struct TrainSpec {
    int d_in;
    const float* X;   // d_in planes of n (standardised)
    const float* Y;
    long long n;
    const float* Xv;  // validation, d_in planes of n_val (null: none)
    const float* Yv;
    long long n_val;
    long long B;
    int epochs;
    long long max_steps;  // > 0: stop after this many steps
    int patience;         // > 0: early stop on the validation loss
    uint64_t order_seed;
    float lr, beta1, beta2, eps;
    float* theta;  // in: initial; out: trained (the kept epoch's)
    float* losses;
    float* grad;
    float* m_out;
    float* v_out;
    float* val_losses;
    int epoch0 = 0;               // resume at this epoch (order and step count continue)
    const float* m_in = nullptr;  // Adam's moments to resume from (null: zero)
    const float* v_in = nullptr;
    float best0 = std::numeric_limits<float>::infinity();  // validation loss to beat
    int bad0 = 0;                       // epochs without a lower validation loss so far
    const float* theta_in = nullptr;    // start from these (null: theta)
    float* theta_last = nullptr;        // the parameters after the last step (may be null)
};
struct TrainInfo {
    int epochs_run, best_epoch, steps;
};
mrip_status mlp_train(const TrainSpec& spec, TrainInfo* info, cudaStream_t st);
mrip_status mlp_forward(const float* theta, int d_in, const float* X, long long n, float* yhat,
                        cudaStream_t st);
mrip_status cv_reduce(const double* y, const double* g, long long n, const double* gc, long long m,
                      int n_dp, double* out, cudaStream_t st);
}  // namespace mrip
