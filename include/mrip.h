/*
 * mrip.h -- C ABI of the GB300 engine for Multiple Replications In Parallel
 * (MRIP) of stochastic simulations.
 *
 * Method (Passerat-Palmbach, Caux, Siregar, Mazel, Hill, "Warp-Level
 * Parallelism: Enabling Multiple Replications In Parallel on GPU", ESM 2011):
 *   - Section 1: a stochastic model is run many times with independent random
 *     sources; the replication mean, by the Central Limit Theorem, gives a
 *     confidence interval; an experimental plan runs a set of replications
 *     for each combination of factor levels (a "design point").
 *   - Section 3: each replication is mapped to its own warp (WLP) rather than
 *     to one thread (TLP).  Here the mapping is chosen per model (thread,
 *     cooperative warp, CTA) and WLP is kept as a measurable baseline.
 *   - Section 5.1: the models (M/M/1 queue, random walk).  This engine adds
 *     a 3-station tandem queue, a forest-fire cellular automaton and an
 *     L1-exit walk as workloads of the same method.
 *
 * Random streams.  Every replication draws from Philox4x32-10 (Salmon et al.,
 * SC'11) with key = (seed low 32 bits, seed high 32 bits) and counter
 *   c0 = sub-block index within a step, c1 = step index,
 *   c2 = replication index,             c3 = (tag << 24) | design point,
 * tags 0 simulation (the control variate's control runs are further
 * replications of tag 0), 1 lattice initial state, 3 network
 * initialisation, 4 minibatch order, 5 and 6 the skip-sampled forest fire's
 * growth and lightning events (2 is unused).  (The paper split one
 * Tausworthe stream by random spacing, Section 5; a counter-based generator
 * lets any replication be recomputed alone.)  Hence design points < 2^24 and
 * replication indices < 2^32.
 *
 * Conventions for every entry point:
 *   - Return value: MRIP_OK or an error code; mrip_last_error() returns a
 *     thread-local, library-owned message for the last failure on the
 *     calling thread.  No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device, owned by the caller (for instance allocated by PyTorch); "host"
 *     pointers are ordinary host memory owned by the caller.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that take a stream only enqueue work on it and return without waiting,
 *     unless the description says "synchronous".
 *   - Per-replication outputs are laid out design-point-major:
 *     element (dp, rep) sits at index dp * n_reps + rep.  Multi-valued
 *     outputs are structure-of-arrays planes: value k of item i sits at
 *     k * n_items + i.
 *   - Scratch memory (work-stealing tickets, partial sums, device error
 *     flags) is allocated by the library once per device and grown on
 *     demand; it is freed at process exit.
 *   - Invalid arguments return MRIP_EINVAL before anything is enqueued.
 *   - A CUDA error returns MRIP_ECUDA with the runtime's message.
 */
#ifndef MRIP_H
#define MRIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MRIP_OK = 0,
    MRIP_EINVAL = 1,        /* invalid argument                                  */
    MRIP_ENOMEM = 2,        /* device or host allocation failed                  */
    MRIP_ECUDA = 3,         /* CUDA runtime or launch error                      */
    MRIP_ESTEPCAP = 4,      /* a replication hit its step cap (output set to -1) */
    MRIP_ESTATE = 5,        /* call out of order (e.g. stats before run)         */
    MRIP_EUNSUPPORTED = 6   /* valid request this library does not implement     */
} mrip_status;

typedef enum {
    MRIP_MM1 = 1,
    MRIP_TANDEM3 = 2,
    MRIP_FOREST_FIRE = 3,
    MRIP_WALK_L1_EXIT = 4
} mrip_kind;

/* Replication-to-hardware mappings (paper, Section 3, and its TLP baseline). */
typedef enum {
    MRIP_MAP_AUTO = 0,        /* use the model's plan (autotuned or default)      */
    MRIP_MAP_THREAD = 1,      /* one replication per thread (TLP)                 */
    MRIP_MAP_WARP_1LANE = 2,  /* one replication per warp, lane 0 only (WLP)      */
    MRIP_MAP_WARP_COOP = 3,   /* one replication per warp, all lanes cooperate    */
    MRIP_MAP_CTA = 4,         /* one replication per CTA (lattice models)         */
    MRIP_MAP_PERSISTENT = 5   /* persistent work-stealing warps, lanes refilled   */
} mrip_mapping;

/* Per-design-point interval (paper, Section 1). */
typedef struct {
    int64_t n;          /* replications used                                    */
    double mean;        /* replication mean                                     */
    double var;         /* unbiased sample variance (NaN if n < 2)              */
    double half_width;  /* t_{(1+conf)/2, df} * sqrt(var / n)  (NaN if n < 2)   */
    double t_crit;      /* the Student-t critical value used                    */
} mrip_stat;

/* Control-variate result of one design point (df = n - 2). */
typedef struct {
    int64_t n;          /* held-out replications                                */
    int64_t m;          /* control-mean runs                                    */
    double beta;        /* Cov(Y, g) / Var(g) over the held-out replications    */
    double mean;        /* mean(Y) - beta (mean(g) - mean(g_ctrl))              */
    double var;         /* s_r^2 / n + beta^2 Var(g_ctrl) / m                    */
    double half_width;  /* t_{(1+conf)/2, n-2} sqrt(var)                         */
    double t_crit;
} mrip_cv_stat;

/* ------------------------------------------------------------------------ */
/* Model handles (the high-level API)                                        */
/* ------------------------------------------------------------------------ */

/* Fixed parameters per model kind, passed to mrip_create_model. */
typedef struct { int64_t n_clients; } mrip_mm1_params;
typedef struct { int64_t n_clients; int64_t window; } mrip_tandem3_params;
typedef struct {
    int32_t L;          /* lattice side, multiple of 32, 32..512                 */
    int32_t n_steps;    /* synchronous steps T >= 1                              */
    double density;     /* initial tree probability in [0, 1)                    */
    int32_t window;     /* early-window length for the network features (<= T)  */
} mrip_forest_fire_params;
typedef struct { int64_t max_steps; } mrip_walk_params;  /* <= 2^38 */

typedef struct mrip_model mrip_model;   /* opaque, library-owned */

/* Create a model of `kind` from its fixed-parameter struct (one of the above;
 * params_bytes must equal its size).  The handle owns the device buffers of
 * its runs.  Not thread-safe per handle; separate handles are independent.
 * Errors: MRIP_EINVAL (unknown kind, wrong size, parameter out of range). */
mrip_status mrip_create_model(int kind, const void *params, size_t params_bytes,
                              mrip_model **out);

/* Run all later work of this handle on `cuda_stream` (a cudaStream_t). */
mrip_status mrip_set_stream(mrip_model *model, void *cuda_stream);

/* Run n_reps replications of every design point (paper, Section 1: MRIP over
 * an experimental plan) and reduce them to per-design-point (n, mean, M2) on
 * the device.  design_points: host array, n_dp x dp_dim, row-major, with
 * dp_dim and meaning per kind: MM1 (lambda, mu); TANDEM3 (lambda, mu1, mu2,
 * mu3); FOREST_FIRE (p_grow, p_lightning) each in [0, 1); WALK_L1_EXIT (R),
 * an integer 1..65536.  Rates must be finite and > 0.  The design points are
 * copied to the device on the handle's stream; the call returns once the
 * work is enqueued (the replay of a CUDA graph captured on first use for this
 * shape).  Per-replication outputs stay on the device (mrip_outputs).
 * The scalar per replication is: MM1 mean wait; TANDEM3 mean sojourn;
 * FOREST_FIRE mean burning fraction sum_t burning_t / (T L^2); WALK tau. */
mrip_status mrip_run(mrip_model *model, const double *design_points, int32_t n_dp,
                     int64_t n_reps, uint64_t seed);

/* Replications rep_lo .. rep_hi - 1 of every design point: the shard of one
 * experiment that one GPU (or one process) runs when the replications of
 * an experimental plan are split (paper, Section 1: replications are
 * independent).  Every replication is a function of (seed, design point,
 * replication index) alone, so the shards of any partition of 0 .. n - 1
 * give exactly the per-replication outputs of one mrip_run of n; their
 * (n, mean, M2) triples (mrip_moments) merge with mrip_stats_merge.
 * Outputs have rep_hi - rep_lo columns per design point; otherwise as
 * mrip_run (which is mrip_run_range(model, dps, n_dp, 0, n_reps, seed)).
 * 0 <= rep_lo < rep_hi <= 2^32. */
mrip_status mrip_run_range(mrip_model *model, const double *design_points, int32_t n_dp,
                           int64_t rep_lo, int64_t rep_hi, uint64_t seed);

/* Same as mrip_run with design_points already on the device. */
mrip_status mrip_run_device(mrip_model *model, const double *d_design_points, int32_t n_dp,
                            int64_t n_reps, uint64_t seed);

/* Synchronous.  Per-design-point intervals of the last run at confidence
 * `conf` in (0, 1) into the caller's host array out[n_dp].  Returns
 * MRIP_ESTEPCAP if a replication hit its step cap, MRIP_ESTATE before any
 * run. */
mrip_status mrip_stats(mrip_model *model, double conf, mrip_stat *out);

/* Synchronous.  The last run's per-design-point (n, mean, M2) triples
 * (FP64, as mrip_stats_reduce) into the caller's host array nmm2_out[n_dp][3]: the
 * exact input of mrip_stats_merge when shards of one experiment are
 * combined.  Errors as mrip_stats. */
mrip_status mrip_moments(mrip_model *model, double *nmm2_out);

/* Synchronous.  Copy output plane `which` of the last run into dst
 * (dst_bytes must be at least its size; on_device != 0: dst is a device
 * pointer).  Planes: MM1 0 wait, 1 idle, 2 system (double); TANDEM3 0 Y
 * (double), 1 features (double, 8 planes); FOREST_FIRE 0 burning counts
 * (int32, rep-major, T per replication), 1 per-replication scalar (double);
 * WALK 0 tau (int64).  Sizes: mrip_output_bytes. */
mrip_status mrip_outputs(mrip_model *model, int which, void *dst, size_t dst_bytes,
                         int on_device);
mrip_status mrip_output_bytes(const mrip_model *model, int which, size_t *bytes);

/* Choose the mapping and launch shape of this handle's model: plan_json is a
 * small JSON object, e.g. {"mapping": 5, "warps_per_cta": 8, "ctas_per_sm": 2,
 * "chunk": 64}; unknown keys are rejected.  mrip_get_plan writes the current
 * plan (NUL-terminated) into buf. */
mrip_status mrip_set_plan(mrip_model *model, const char *plan_json);
mrip_status mrip_get_plan(const mrip_model *model, char *buf, size_t buf_bytes);

/* Synchronous.  Time every candidate plan for (design_points, n_dp, n_reps)
 * with CUDA events (best of `trials`), check that every candidate gives the
 * same per-replication outputs as the first, keep the fastest and record it
 * in the cache file `cache_path` (JSON lines, may be NULL).  The WLP mapping
 * of the paper (Section 3) is one of the candidates. */
mrip_status mrip_autotune(mrip_model *model, const double *design_points, int32_t n_dp,
                          int64_t n_reps, uint64_t seed, int trials, const char *cache_path);

/* Learned control variate (engine extension; the paper's estimator is the
 * plain mean of Section 1, which stays the fallback and the yardstick).
 * Synchronous.  Steps:
 *   1. runs the n_reps replications of every design point and writes the
 *      plain intervals (all n_reps) into plain_out;
 *   2. trains the network d_in -> 64 -> 64 -> 1 (d_in 8 for TANDEM3: lambda,
 *      mu1..3 and the means of the first `window` gaps and services; 6 for
 *      FOREST_FIRE: log10 p_grow, log10 p_lightning and the mean burning
 *      fraction of the four quarters of the first `window` steps) with
 *      mrip_mlp_train on the first n_fit of the n_train = ceil(train_frac
 *      n_reps) training replications of every design point; the other
 *      n_val = ceil(val_frac n_train) are the validation set (early stop,
 *      `patience`).  Inputs and target are standardised with the fit set's
 *      FP64 mean and population standard deviation;
 *   3. from the validation replications, estimates rho^2, the pooled
 *      within-design-point squared correlation of Y and the prediction g
 *      (each design point's deviations divided by its own standard
 *      deviations of Y and g over its fit replications, so that every
 *      design point weighs the same), and sizes the control runs: m_ctrl = 0 asks for
 *      M = ceil(n_held rho^2 / (0.1 (1 - rho^2))), clamped to
 *      [2, 100 n_held], so that the control mean adds at most a tenth to
 *      the residual variance (10 n_held without validation);
 *   4. gate != 0: after the first ceil(64 / steps per epoch) epochs (at
 *      least 64 Adam steps; only if that is fewer than `epochs`), a
 *      validation rho^2 below a quarter of the break-even
 *      1 - n_held / (1.1 n_reps) declines at once (report->declined = 2, no
 *      further training; the run otherwise resumes exactly); after training,
 *      predicts the variance ratio of the control-variate and plain
 *      estimators at this n, n_reps ((1 - rho^2) / n_held + rho^2 / M),
 *      and when it is >= 1 declines (report->declined = 1).  Declined:
 *      cv_out gets the plain intervals (m = 0, beta = 0);
 *   5. otherwise predicts g for the n_held = n_reps - n_train held-out
 *      replications and for the M control runs -- the replications
 *      n_reps .. n_reps + M - 1 of the same streams (tag 0), simulated for
 *      the early window only -- and writes per design point
 *      beta = Cov(Y, g) / Var(g), mean(Y) - beta (mean(g) - mean(g_ctrl)),
 *      var = s_r^2 / n_held + beta^2 Var(g_ctrl) / M and the Student-t
 *      interval on n_held - 2 degrees of freedom into cv_out.
 * report (may be NULL) receives the counts, losses, rho^2 and the CUDA-event
 * time of each phase. */
typedef struct {
    double train_frac;   /* in (0, 1), e.g. 0.1                                 */
    double val_frac;     /* in [0, 1): share of the training replications kept  */
                         /* for validation; 0: no validation, no gate           */
    int32_t epochs;      /* >= 1 (the maximum when validating)                  */
    int32_t patience;    /* >= 0: early stop on the validation loss (0: never)  */
    int32_t batch;       /* >= 1                                                */
    int32_t gate;        /* != 0: decline the control variate when it cannot    */
                         /* beat the plain estimator at this n                  */
    float lr, beta1, beta2, eps;
    int64_t m_ctrl;      /* control runs per design point: 0 = sized as above,  */
                         /* else >= 2                                           */
    double conf;         /* interval confidence in (0, 1)                       */
    uint64_t net_seed;   /* network initialisation and minibatch order          */
} mrip_cv_params;

typedef struct {
    int32_t declined;    /* 0 kept; 1 declined after training, 2 by the screen   */
                         /* after the first epochs: cv_out = plain intervals   */
    int32_t epochs_run;
    int32_t best_epoch;  /* the epoch whose parameters were kept (1-based)      */
    int32_t n_val;       /* validation replications per design point            */
    int64_t m_ctrl;      /* control runs per design point (0 when declined)     */
    float train_loss;    /* mean minibatch loss of the last epoch run           */
    float val_loss;      /* validation loss of the kept epoch (NaN: none)       */
    double val_rho2;     /* pooled within-design-point rho^2 (NaN: none)        */
    double var_ratio;    /* predicted Var(control variate) / Var(plain) (NaN)   */
    double ms_simulate;  /* plain run and intervals                             */
    double ms_train;     /* features, standardisation, training, validation     */
    double ms_control;   /* control runs and their features                     */
    double ms_infer;     /* predictions of held-out and control replications    */
    double ms_estimate;  /* per-design-point estimator and read-back            */
} mrip_cv_report;

mrip_status mrip_run_cv(mrip_model *model, const double *design_points, int32_t n_dp,
                        int64_t n_reps, uint64_t seed, const mrip_cv_params *params,
                        mrip_stat *plain_out, mrip_cv_stat *cv_out, mrip_cv_report *report);

/* Synchronous.  The network of the handle's last mrip_run_cv: its
 * parameters (host float[mrip_mlp_param_count(d_in)], may be NULL) and the
 * standardisation (host double[2 (d_in + 1)]: mean and std of each input,
 * then of the target; may be NULL).  MRIP_ESTATE before any mrip_run_cv. */
mrip_status mrip_cv_network(mrip_model *model, float *theta_out, double *norm_out);

void mrip_destroy(mrip_model *model);

/* Thread-local message of the last failure on this thread ("" if none). */
const char *mrip_last_error(void);

/* ------------------------------------------------------------------------ */
/* Stage entry points (the low-level API): one per step of the hot path,     */
/* device buffers owned by the caller.                                       */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 of n counters.  d_ctr: device uint32 n x 4; d_key: device
 * uint32 n x 2; d_out: device uint32 n x 4. */
mrip_status mrip_philox(const uint32_t *d_ctr, const uint32_t *d_key, int64_t n,
                        uint32_t *d_out, void *stream);

/* u = top 53 bits of hi:lo times 2^-53 and the exponential variate
 * -log(1 - u) / rate (paper, Section 5.1: the M/M/1 arrival gaps and service
 * times are exponential).  All arrays device, length n. */
mrip_status mrip_expo(const uint32_t *d_lo, const uint32_t *d_hi, const double *d_rate,
                      int64_t n, double *d_u, double *d_e, void *stream);

/* M/M/1 replications (paper, Section 5.1, second model).  d_dps: device
 * n_dp x 2 (lambda, mu).  Replications rep0 .. rep0 + n_reps - 1 (indices
 * < 2^32; output column r is replication rep0 + r).  Client n uses block
 * (c0 = 0, c1 = n): words 0,1 ->
 * service S_n ~ Exp(mu), words 2,3 -> gap A_{n+1} ~ Exp(lambda); W_0 = 0,
 * W_{n+1} = max(0, W_n + S_n - A_{n+1}).  Outputs (device, n_dp * n_reps,
 * any may be NULL): mean wait W, mean idle max(0, A_{n+1} - W_n - S_n),
 * mean time in system W + S over n < n_clients.  mapping: THREAD,
 * WARP_1LANE, WARP_COOP or CTA (one replication per CTA of up to 1,024
 * threads, ~4 clients each, block scan of the maps; for a few replications
 * whose latency matters).  AUTO = THREAD. */
mrip_status mrip_mm1_simulate(const double *d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                              int64_t n_clients, uint64_t seed, int mapping,
                              double *d_wait, double *d_idle, double *d_system, void *stream);

/* Tandem of three M/M/1 stations.  d_dps: device n_dp x 4 (lambda, mu1..3).
 * Client n: block (0, n) words 0,1 -> gap A_n, 2,3 -> S_{n,1}; block (1, n)
 * -> S_{n,2}, S_{n,3}.  V_{n,j} = max(V_{n-1,j} - A_n, V_{n,j-1}) + S_{n,j},
 * V_{n,0} = 0, V_{-1,j} = -inf; Y = mean_n V_{n,3}.  Replications
 * rep0 .. rep0 + n_reps - 1 of stream `tag`.  d_y: device n_dp * n_reps;
 * d_feat (may be NULL): device 8 planes of n_dp * n_reps: lambda, mu1..3 and
 * the means over the first min(window, n_clients) clients of A, S1, S2, S3.
 * If n_clients == window only the early window is simulated (control runs).
 * mapping: THREAD, WARP_1LANE, WARP_COOP (one replication per warp: lanes
 * take 32 contiguous client segments, a warp scan of their max-plus maps gives
 * each segment's entry state) or CTA (the same over up to 1,024 threads, ~4
 * clients each, with a block scan); the last two are for few replications of
 * many clients.  AUTO = THREAD. */
mrip_status mrip_tandem3_simulate(const double *d_dps, int32_t n_dp, int64_t rep0,
                                  int64_t n_reps, int64_t n_clients, int64_t window,
                                  uint64_t seed, uint32_t tag, int mapping, double *d_y,
                                  double *d_feat, void *stream);

/* Forest-fire automaton, one CTA per replication, lattice bit-packed in
 * registers and shared memory.  d_dps: device n_dp x 2 (p_grow,
 * p_lightning).  Replications rep0 .. rep0 + n_reps - 1 (indices < 2^32;
 * output row r is replication rep0 + r).  L multiple of 32 in 32..512,
 * n_steps >= 0.
 * Initial state from tag 1 (tree iff word < floor(density 2^32)), or from
 * d_init (device uint8 L*L per replication, states 0/1/2; may be NULL).
 * Step t uses word (i mod 4) of block (i div 4, t) for cell i = y L + x:
 * burning -> empty; tree -> burning if a von Neumann neighbour burns or the
 * word < floor(p_lightning 2^32); empty -> tree iff word < floor(p_grow
 * 2^32).  Outputs (device, may be NULL): d_counts int32 [n_dp*n_reps][n_steps]
 * burning cells after each step; d_scalar double [n_dp*n_reps] =
 * sum_t counts / (n_steps L^2); d_final uint8 [n_dp*n_reps][L*L]. */
mrip_status mrip_forest_fire_simulate(const double *d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                                      int32_t L, int32_t n_steps, double density,
                                      uint64_t seed, const uint8_t *d_init,
                                      int32_t *d_counts, double *d_scalar, uint8_t *d_final,
                                      void *stream);

/* Forest fire with skip-sampled events (an engine variant; the paper has no
 * lattice model).  Same rules, arguments, outputs and initial state (tag 1)
 * as mrip_forest_fire_simulate, but each step t draws its growth and
 * lightning event sets as gaps between successes over the cells
 * i = y L + x: gap j is K_j = floor(E_j / mu), mu = -log1p(-p), E_j the
 * exponential variate -log(1 - u) of words 2(j mod 2), 2(j mod 2)+1 of block
 * (c0 = j div 2, c1 = t) under tag 5 (p_grow) or tag 6 (p_light); events at
 * K_0, K_0 + 1 + K_1, ... below L^2.  An empty cell with a growth event
 * becomes a tree; a tree without a burning neighbour ignites on a lightning
 * event.  Per cell and step the law is the per-cell model's with the exact
 * probabilities; the work per step is p L^2 variates instead of L^2 words.
 * p <= 0 (or NaN): no events; p >= 1: every cell. */
mrip_status mrip_forest_fire_skip_simulate(const double *d_dps, int32_t n_dp, int64_t rep0, int64_t n_reps,
                                           int32_t L, int32_t n_steps, double density,
                                           uint64_t seed, const uint8_t *d_init, int32_t *d_counts,
                                           double *d_scalar, uint8_t *d_final, void *stream);

/* L1-exit walk: simple random walk on Z^2 from the origin; move m reads the
 * 2-bit field k = m mod 64 of block (0, m div 64): word k div 16, bits
 * 2(k mod 16)..+1; 0:+x 1:-x 2:+y 3:-y.  tau = moves made when |x|+|y|
 * first reaches R.  Replications rep0 .. rep0 + n_reps - 1 (indices < 2^32;
 * output column r is replication rep0 + r).  radii: HOST array n_dp
 * (integers 1..65536).  d_tau:
 * device int64 n_dp * n_reps (-1 where max_steps was reached, and the call's
 * later status check reports MRIP_ESTEPCAP).  mapping: THREAD, WARP_1LANE,
 * WARP_COOP or PERSISTENT (AUTO = PERSISTENT); warps_per_cta, ctas_per_sm and
 * chunk (replications per ticket) shape PERSISTENT (0 = default: 32 warps,
 * one CTA per SM, chunks of 16; when no replications are left, a warp
 * finishes its last walkers with all 32 lanes on one walker at a time). */
mrip_status mrip_walk_simulate(const double *radii, int32_t n_dp, int64_t rep0, int64_t n_reps,
                               uint64_t seed, int64_t max_steps, int mapping,
                               int32_t warps_per_cta, int32_t ctas_per_sm, int32_t chunk,
                               int64_t *d_tau, void *stream);

/* Same walk, same arguments and outputs as mrip_walk_simulate, for callers
 * that cannot allocate device memory: code running inside a framework or
 * memory pool that owns every device allocation, or a latency-critical loop
 * where cudaMalloc (which can synchronize the device and can fail) is not
 * allowed.  The paper has no counterpart; it is a deployment variant.
 * The call allocates nothing: its scratch (work-stealing ticket, step-cap
 * flag, radius and design-point tables) is a fixed array of 8,448 bytes
 * inside the library, present on every GPU that loads it until the process
 * exits.  Limit: n_dp <= 1024 (larger values return MRIP_EINVAL).  Each call
 * looks the current device's address of the array up
 * (cudaGetSymbolAddress), then enqueues a small set-up kernel that writes
 * the tables (passed as its argument) and clears the ticket and the flag,
 * then the walk; it copies nothing from host memory and does not wait for
 * the GPU.  The first lookup on a device can load the library's device
 * code, so make the first call on each device before any stream capture on
 * that device.
 * Every call reuses the same array, so two calls whose work overlaps on the
 * GPU (different streams, or another thread) race and must not be issued
 * concurrently; calls on one stream run one after the other.  A replication
 * that reaches max_steps is written as -1; mrip_check_device_flags does
 * not see it (scan d_tau for -1). */
mrip_status mrip_walk_simulate_noalloc(const double *radii, int32_t n_dp, int64_t rep0,
                                       int64_t n_reps, uint64_t seed, int64_t max_steps,
                                       int mapping, int32_t warps_per_cta, int32_t ctas_per_sm,
                                       int32_t chunk, int64_t *d_tau, void *stream);

/* Area walk: the paper's random-walk model (Section 5.1, third model) and
 * its WLP-versus-TLP experiment (Section 5.3).  A walker on a 60 x 50
 * periodic map split into 30 areas of 10 x 10 cells (area x/10 + 6 (y/10))
 * starts at (30, 25); move m reads field m mod 64 of block (0, m div 64) of
 * replication rep0 + r (output column r), design point 0 (0:+x 1:-x 2:+y 3:-y); after every move
 * its area's visit count grows by one.  d_final_area: device int32 n_reps;
 * d_visits: device int32 30 planes of n_reps (may be NULL).  mapping: THREAD
 * (one replication per thread), WARP_1LANE (one per warp, lane 0 -- the
 * paper's WLP) or WARP_COOP (one per warp, lanes share 512-move rounds);
 * AUTO = THREAD.  n_steps <= 2^30. */
mrip_status mrip_area_walk_simulate(int64_t rep0, int64_t n_reps, int32_t n_steps, uint64_t seed,
                                    int mapping, int32_t *d_final_area, int32_t *d_visits,
                                    void *stream);

/* Monte Carlo pi (paper, Section 5.1, first model).  Draw k of replication
 * rep0 + r (output r; design point 0) uses words 2(k mod 2), 2(k mod 2)+1 of block
 * (0, k div 2) as integers x, y in [0, 2^32); it hits iff x^2 + y^2 < 2^64.
 * d_hits: device int64 n_reps (cleared, then filled with the hit counts;
 * pi ~ 4 hits / n_draws).  n_draws <= 2^33. */
mrip_status mrip_pi_simulate(int64_t rep0, int64_t n_reps, int64_t n_draws, uint64_t seed,
                             int64_t *d_hits, void *stream);

/* Synchronous.  MRIP_ESTEPCAP if any walk launched since the last check hit
 * its step cap (and clears the flag), else MRIP_OK. */
mrip_status mrip_check_device_flags(void);

/* Synchronous (waits for the whole device).  Bounds checks of a debug build
 * (the library compiled with -DMRIP_DEBUG; compute-sanitizer's stand-in):
 * kernels check their data-dependent indices -- event positions, the walk's
 * work-item decoding, minibatch sample indices, map cells, output ranges --
 * and the use of dynamically sized shared memory against the launch's
 * actual size; a failed check records (site, index) and skips the access.
 * *enabled: 1 in a debug build, 0 otherwise (then *first is 0).  *first:
 * (site << 40) | (index mod 2^40) of the first failed check since the last
 * call (sites: forest fire 1xx, queues 2xx, walk 3xx, network 4xx, control
 * variate 5xx, area walk 6xx, statistics 7xx), 0 if none; the records are
 * cleared. */
mrip_status mrip_debug_checks(int32_t *enabled, uint64_t *first);

/* Synchronous.  Measured throughput of the widening 32 x 32 -> 64-bit
 * multiply (two per Philox4x32-10 round; the unit that bounds the Philox
 * stream): a kernel filling every SM with independent chains of one such
 * multiply and one logic operation, timed with CUDA events on `stream`
 * (about a millisecond).  *warp_products_per_s: warp-wide multiplies (32
 * products each) per second on this GPU at its current clocks.  Errors:
 * MRIP_EINVAL for a null argument, MRIP_ENOMEM, MRIP_ECUDA. */
mrip_status mrip_probe_mul_wide(double *warp_products_per_s, void *stream);

/* Debug build only: records one deliberately failed check (site 999, index
 * 12345) that guards no access, so a test can see the record travel to
 * mrip_debug_checks.  A release build returns MRIP_EINVAL. */
mrip_status mrip_debug_selftest(void);

/* Per-design-point (n, mean, M2) of d_x (device double [n_dp][n_reps]) by
 * the two-pass definition (mean = sum / n, then M2 = sum of squared
 * deviations from it), each sum in a fixed order over 256 threads; more than
 * 4,096 replications are cut into slices (one CTA each) whose triples are
 * merged in slice order by Chan's pairwise formula (deterministic).  d_out: device double [n_dp][3].  The slice
 * partials live in library scratch memory, which a later call may grow:
 * capture this call in a CUDA graph only if that graph is replayed before
 * any larger reduction runs (4,096 replications or fewer need no scratch).
 * With n_reps == 0 d_x may be NULL and every triple is (0, 0, 0). */
mrip_status mrip_stats_reduce(const double *d_x, int32_t n_dp, int64_t n_reps,
                              double *d_out, void *stream);

/* mrip_stats_reduce for int64 outputs (the walk's exit times). */
mrip_status mrip_stats_reduce_i64(const int64_t *d_x, int32_t n_dp, int64_t n_reps,
                                  double *d_out, void *stream);

/* Host, synchronous: intervals from host (n, mean, M2) triples. */
mrip_status mrip_stats_finalize(const double *nmm2, int32_t n_dp, double conf,
                                mrip_stat *out);

/* Host, synchronous: merge per-design-point (n, mean, M2) triples of n_parts
 * disjoint replication sets -- e.g. the shards of several GPUs or a resumed
 * run -- into one set (Chan, Golub, LeVeque pairwise update, parts merged
 * in index order, so the result does not depend on arrival order).
 * parts: host double [n_parts][n_dp][3]; out: host double [n_dp][3].
 * Empty parts (n = 0) are allowed. */
mrip_status mrip_stats_merge(const double *parts, int32_t n_parts, int32_t n_dp, double *out);

/* Host: Student-t critical value t with P(T > t) = (1 - conf) / 2, df >= 1. */
mrip_status mrip_t_crit(double conf, int64_t df, double *out);

/* ----- learned control variate: network stages (device, caller-owned) ---- */
/* Flat FP32 parameter vector of d_in -> 64 -> 64 -> 1:
 * W1 [64][d_in], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]. */
int64_t mrip_mlp_param_count(int32_t d_in);

/* He-uniform initialisation from stream tag 3 (weights), zero biases. */
mrip_status mrip_mlp_init(int32_t d_in, uint64_t seed, float *d_theta, void *stream);

/* Forward pass of n samples.  d_x: device float [d_in][n] planes
 * (standardised inputs); d_yhat: device float n.  BF16 operands, FP32
 * accumulation. */
mrip_status mrip_mlp_forward(const float *d_theta, int32_t d_in, const float *d_x,
                             int64_t n, float *d_yhat, void *stream);

/* Loss mean (yhat - y)^2 over the B samples idx[0..B) (device int64, may be
 * NULL = 0..B-1) and its gradient.  d_grad: device float param_count;
 * d_loss: device float 1 (may be NULL). */
mrip_status mrip_mlp_loss_grad(const float *d_theta, int32_t d_in, const float *d_x,
                               const float *d_y, int64_t n, const int64_t *d_idx,
                               int64_t B, float *d_grad, float *d_loss, void *stream);

/* Training of the network on the tensor cores: the kernel mrip_run_cv uses.
 * One launch on a cluster of 8 CTAs runs every Adam step (Kingma & Ba, with
 * bias correction, steps counted from 1) of every epoch; the four 64-wide
 * contractions of a 128-sample tile run as tcgen05 MMAs with BF16 operands
 * and FP32 accumulators in tensor memory.  Epoch e visits the n samples in
 * the order pi(i) = (a i + b) mod n from block (0, e) of stream tag 4 under
 * order_seed (a = 1 + w0 mod (n - 1), stepped up to the first value coprime
 * with n; b = w1 mod n); minibatch k is positions k B .. min(k B + B, n) - 1,
 * the loss the mean of (yhat - y)^2 over it.  With a validation set
 * (n_val > 0), the mean squared error over it is evaluated after every
 * epoch; the parameters of the epoch with the lowest value are kept, and
 * training stops after `patience` epochs without a lower value (0: never).
 * Arguments (device unless stated; "may be NULL" outputs are skipped):
 *   d_x, d_y      float, d_in planes of n, and n (standardised inputs/target)
 *   d_xv, d_yv    the validation set, d_in planes of n_val, and n_val
 *   d_theta       in: initial parameters (mrip_mlp_param_count floats);
 *                 out: the trained ones (the kept epoch's with validation)
 *   d_m_in, d_v_in  Adam's moments to resume from (may be NULL: zero) --
 *                 with params->epoch0 = e this continues a run stopped after
 *                 e epochs: epoch order and Adam's step count go on from there
 *   d_losses      per Adam step (may be NULL; room for every step run)
 *   d_grad        the gradient of the last step (may be NULL)
 *   d_m, d_v      Adam's moments after the last step (may be NULL)
 *   d_val_losses  per epoch (may be NULL)
 *   info_out      HOST int32[3]: epochs run, epoch kept (1-based), steps run
 *                 (may be NULL)
 * Synchronous (it reads back the kernel's status).  An MMA that does not
 * complete within its wait limit returns MRIP_ECUDA. */
typedef struct {
    int64_t batch;        /* minibatch size >= 1                              */
    int32_t epochs;       /* >= 1 (epochs of this call)                       */
    int32_t patience;     /* >= 0; early stop on the validation loss          */
    int64_t max_steps;    /* > 0: stop after this many Adam steps; 0: none    */
    float lr, beta1, beta2, eps;
    uint64_t order_seed;  /* minibatch order (stream tag 4)                   */
    int32_t epoch0;       /* >= 0: index of this call's first epoch (resume)  */
    int32_t pad;
} mrip_train_params;
mrip_status mrip_mlp_train(int32_t d_in, const float *d_x, const float *d_y, int64_t n,
                           const float *d_xv, const float *d_yv, int64_t n_val,
                           const mrip_train_params *params, float *d_theta,
                           const float *d_m_in, const float *d_v_in, float *d_losses,
                           float *d_grad, float *d_m, float *d_v, float *d_val_losses,
                           int32_t *info_out, void *stream);

/* One Adam step (Kingma & Ba) with bias correction; step t >= 1. */
mrip_status mrip_adam_step(float *d_theta, float *d_m, float *d_v, const float *d_grad,
                           int64_t n, int64_t t, float lr, float beta1, float beta2,
                           float eps, void *stream);

/* Control-variate estimator of n_dp design points (FP64, device): d_y, d_g
 * [n_dp][n]; d_gc [n_dp][m].  d_out: device double [n_dp][5] =
 * (beta, mean, var, y_mean, 0); the host adds the t critical value. */
mrip_status mrip_cv_reduce(const double *d_y, const double *d_g, int64_t n,
                           const double *d_gc, int64_t m, int32_t n_dp, double *d_out,
                           void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MRIP_H */
