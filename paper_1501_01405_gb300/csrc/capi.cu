// Model handles: the high-level C ABI (mrip_create_model, mrip_run,
// mrip_stats, ...).  A handle owns the device buffers of its runs, picks the
// replication mapping from its plan, and replays a CUDA graph of
// "simulate + reduce" captured on first use for a given shape and seed.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "model.cuh"


namespace mrip {

int dp_dim(int kind) {
    switch (kind) {
        case MRIP_MM1: return 2;
        case MRIP_TANDEM3: return 4;
        case MRIP_FOREST_FIRE: return 2;
        case MRIP_WALK_L1_EXIT: return 1;
    }
    return 0;
}

mrip_status check_dps(int kind, const double* dps, int32_t n_dp) {
    const int k = dp_dim(kind);
    for (int32_t i = 0; i < n_dp; ++i) {
        for (int j = 0; j < k; ++j) {
            const double v = dps[static_cast<size_t>(i) * k + j];
            if (kind == MRIP_MM1 || kind == MRIP_TANDEM3) {
                if (!(std::isfinite(v) && v > 0.0))
                    return fail(MRIP_EINVAL, "design point " + std::to_string(i) +
                                                 ": rates must be finite and > 0");
            } else if (kind == MRIP_FOREST_FIRE) {
                if (!(v >= 0.0 && v < 1.0))
                    return fail(MRIP_EINVAL, "design point " + std::to_string(i) +
                                                 ": probabilities must be in [0, 1)");
            } else if (kind == MRIP_WALK_L1_EXIT) {
                if (!(v >= 1.0 && v <= 65536.0) || v != std::floor(v))
                    return fail(MRIP_EINVAL, "design point " + std::to_string(i) +
                                                 ": R must be an integer in 1..65536");
            }
        }
    }
    return MRIP_OK;
}

size_t plane_bytes(const mrip_model* m, int which) {
    const size_t items = static_cast<size_t>(m->n_dp) * m->n_reps;
    switch (m->kind) {
        case MRIP_MM1: return which >= 0 && which < 3 ? items * sizeof(double) : 0;
        case MRIP_TANDEM3: return which == 0 ? items * sizeof(double) : which == 1 ? 8 * items * sizeof(double) : 0;
        case MRIP_FOREST_FIRE:
            return which == 0 ? items * m->ff.n_steps * sizeof(int32_t) : which == 1 ? items * sizeof(double) : 0;
        case MRIP_WALK_L1_EXIT: return which == 0 ? items * sizeof(int64_t) : 0;
    }
    return 0;
}

// Enqueue simulate + reduce for the current buffers (capturable).
mrip_status enqueue_run(mrip_model* m, uint64_t seed) {
    const int32_t n_dp = m->n_dp;
    const int64_t n_reps = m->n_reps;
    const long long items = static_cast<long long>(n_dp) * n_reps;
    cudaStream_t st = m->stream;
    const double* d_dps = m->dps.as<double>();
    mrip_status s = MRIP_OK;
    switch (m->kind) {
        case MRIP_MM1: {
            double* w = m->out0.as<double>();
            s = mrip_mm1_simulate(d_dps, n_dp, m->rep0, n_reps, m->mm1.n_clients, seed, m->plan.mapping, w,
                                  w + items, w + 2 * items, st);
            if (s == MRIP_OK) s = stats_reduce_double(w, n_dp, n_reps, m->nmm2.as<double>(), st, m->spart.as<double>());
            break;
        }
        case MRIP_TANDEM3: {
            s = mrip_tandem3_simulate(d_dps, n_dp, m->rep0, n_reps, m->tandem.n_clients, m->tandem.window,
                                      seed, 0, m->plan.mapping, m->out0.as<double>(),
                                      m->out1.as<double>(), st);
            if (s == MRIP_OK)
                s = stats_reduce_double(m->out0.as<double>(), n_dp, n_reps, m->nmm2.as<double>(), st, m->spart.as<double>());
            break;
        }
        case MRIP_FOREST_FIRE: {
            s = mrip_forest_fire_simulate(d_dps, n_dp, m->rep0, n_reps, m->ff.L, m->ff.n_steps, m->ff.density,
                                          seed, nullptr, m->out0.as<int32_t>(), m->out1.as<double>(),
                                          nullptr, st);
            if (s == MRIP_OK)
                s = stats_reduce_double(m->out1.as<double>(), n_dp, n_reps, m->nmm2.as<double>(), st, m->spart.as<double>());
            break;
        }
        case MRIP_WALK_L1_EXIT: {
            const int32_t* tab = m->walk_tab.as<int32_t>();
            s = walk_launch(tab, tab + n_dp, n_dp, m->rep0, n_reps, seed, m->walk.max_steps, m->plan.mapping,
                            m->plan.warps_per_cta, m->plan.ctas_per_sm, m->plan.chunk,
                            m->out0.as<int64_t>(), m->ticket.as<unsigned long long>(), st);
            if (s == MRIP_OK)
                s = stats_reduce_int64(m->out0.as<int64_t>(), n_dp, n_reps, m->nmm2.as<double>(), st, m->spart.as<double>());
            break;
        }
        default: s = fail(MRIP_EINVAL, "unknown model kind");
    }
    return s;
}

bool same_plan(const Plan& a, const Plan& b) {
    return a.mapping == b.mapping && a.warps_per_cta == b.warps_per_cta &&
           a.ctas_per_sm == b.ctas_per_sm && a.chunk == b.chunk;
}

// Size buffers and upload the per-shape tables; host_dps already validated.
mrip_status prepare(mrip_model* m, int32_t n_dp, int64_t n_reps) {
    const size_t items = static_cast<size_t>(n_dp) * n_reps;
    m->n_dp = n_dp;
    m->n_reps = n_reps;
    bool ok = m->dps.ensure(static_cast<size_t>(n_dp) * dp_dim(m->kind) * sizeof(double)) &&
              m->nmm2.ensure(static_cast<size_t>(n_dp) * 3 * sizeof(double));
    const size_t spart = stats_scratch_bytes(n_dp, n_reps);
    if (spart) ok = ok && m->spart.ensure(spart);
    switch (m->kind) {
        case MRIP_MM1: ok = ok && m->out0.ensure(3 * items * sizeof(double)); break;
        case MRIP_TANDEM3:
            ok = ok && m->out0.ensure(items * sizeof(double)) && m->out1.ensure(8 * items * sizeof(double));
            break;
        case MRIP_FOREST_FIRE:
            ok = ok && m->out0.ensure(items * m->ff.n_steps * sizeof(int32_t)) &&
                 m->out1.ensure(items * sizeof(double));
            break;
        case MRIP_WALK_L1_EXIT:
            ok = ok && m->out0.ensure(items * sizeof(int64_t)) &&
                 m->walk_tab.ensure(2 * static_cast<size_t>(n_dp) * sizeof(int32_t)) &&
                 m->ticket.ensure(sizeof(unsigned long long));
            break;
    }
    if (!ok) return fail(MRIP_ENOMEM, "mrip_run: device allocation failed");
    return MRIP_OK;
}

mrip_status run_common(mrip_model* m, int32_t n_dp, int64_t n_reps, uint64_t seed) {
    if (m->kind == MRIP_WALK_L1_EXIT) {
        std::vector<int32_t> r_by_pos, dp_by_pos;
        mrip_status s = walk_tables(m->host_dps.data(), n_dp, r_by_pos, dp_by_pos);
        if (s != MRIP_OK) return s;
        std::vector<int32_t> tab(r_by_pos);
        tab.insert(tab.end(), dp_by_pos.begin(), dp_by_pos.end());
        cudaError_t e = cudaMemcpyAsync(m->walk_tab.p, tab.data(), tab.size() * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return cuda_status(e, "mrip_run: table upload");
        if (!device_error_flags()) return fail(MRIP_ENOMEM, "device error flags");
    }
    const bool reuse = m->exec && m->g_n_dp == n_dp && m->g_n_reps == n_reps && m->g_rep0 == m->rep0 &&
                       m->g_seed == seed && same_plan(m->g_plan, m->plan);
    if (!reuse) {
        if (m->exec) {
            cudaGraphExecDestroy(m->exec);
            m->exec = nullptr;
        }
        // the stage launchers touch lazily created tables; create them before capture
        sm_count();
        LogTable tab;
        mrip_status ts = log_table(&tab);
        if (ts != MRIP_OK) return ts;
        cudaStream_t cap = m->stream;
        bool own = false;
        if (cap == nullptr) {  // the legacy stream cannot be captured
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
                return cuda_status(cudaGetLastError(), "mrip_run: stream");
            own = true;
        }
        cudaStream_t saved = m->stream;
        m->stream = cap;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        mrip_status s = MRIP_OK;
        if (e == cudaSuccess) {
            s = enqueue_run(m, seed);
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (s == MRIP_OK && e2 != cudaSuccess) s = cuda_status(e2, "mrip_run: capture");
        } else {
            s = cuda_status(e, "mrip_run: begin capture");
        }
        m->stream = saved;
        if (own) cudaStreamDestroy(cap);
        if (s != MRIP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        e = cudaGraphInstantiate(&m->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            m->exec = nullptr;
            return cuda_status(e, "mrip_run: instantiate");
        }
        m->g_n_dp = n_dp;
        m->g_n_reps = n_reps;
        m->g_rep0 = m->rep0;
        m->g_seed = seed;
        m->g_plan = m->plan;
    }
    cudaError_t e = cudaGraphLaunch(m->exec, m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_run: graph launch");
    m->has_run = true;
    return MRIP_OK;
}

mrip_status check_shape(mrip_model* m, int32_t n_dp, int64_t n_reps, int64_t rep0 = 0) {
    if (n_dp < 1 || n_dp >= (1 << 24)) return fail(MRIP_EINVAL, "mrip_run: n_dp in 1..2^24-1");
    if (n_reps < 1 || n_reps > 0xFFFFFFFFll) return fail(MRIP_EINVAL, "mrip_run: n_reps in 1..2^32-1");
    if (rep0 < 0 || rep0 + n_reps > 0x100000000ll)
        return fail(MRIP_EINVAL, "mrip_run_range: 0 <= rep_lo < rep_hi <= 2^32");
    if (m->kind == MRIP_FOREST_FIRE && static_cast<long long>(n_dp) * n_reps > 0x7FFFFFFFll)
        return fail(MRIP_EINVAL, "mrip_run: forest fire needs n_dp * n_reps < 2^31");
    return MRIP_OK;
}

// ---- tiny JSON object parser for plans: {"key": int, ...} ----
bool parse_plan(const char* js, Plan& p, std::string& err) {
    Plan out = p;
    std::string s(js ? js : "");
    size_t i = s.find('{');
    if (i == std::string::npos) {
        err = "plan: expected a JSON object";
        return false;
    }
    ++i;
    while (true) {
        while (i < s.size() && isspace(static_cast<unsigned char>(s[i]))) ++i;
        if (i < s.size() && s[i] == '}') break;
        if (i >= s.size() || s[i] != '"') {
            err = "plan: expected a key";
            return false;
        }
        size_t j = s.find('"', i + 1);
        if (j == std::string::npos) {
            err = "plan: unterminated key";
            return false;
        }
        std::string key = s.substr(i + 1, j - i - 1);
        i = s.find(':', j);
        if (i == std::string::npos) {
            err = "plan: expected ':'";
            return false;
        }
        ++i;
        char* endp = nullptr;
        long v = std::strtol(s.c_str() + i, &endp, 10);
        if (endp == s.c_str() + i) {
            err = "plan: value of " + key + " must be an integer";
            return false;
        }
        i = endp - s.c_str();
        if (key == "mapping") out.mapping = static_cast<int>(v);
        else if (key == "warps_per_cta") out.warps_per_cta = static_cast<int>(v);
        else if (key == "ctas_per_sm") out.ctas_per_sm = static_cast<int>(v);
        else if (key == "chunk") out.chunk = static_cast<int>(v);
        else {
            err = "plan: unknown key '" + key + "'";
            return false;
        }
        while (i < s.size() && isspace(static_cast<unsigned char>(s[i]))) ++i;
        if (i < s.size() && s[i] == ',') {
            ++i;
            continue;
        }
        if (i < s.size() && s[i] == '}') break;
        err = "plan: expected ',' or '}'";
        return false;
    }
    if (out.mapping < 0 || out.mapping > MRIP_MAP_PERSISTENT || out.warps_per_cta < 0 ||
        out.warps_per_cta > 32 || out.ctas_per_sm < 0 || out.ctas_per_sm > 64 || out.chunk < 0 ||
        out.chunk > (1 << 20)) {
        err = "plan: value out of range";
        return false;
    }
    p = out;
    return true;
}

std::string plan_json(const Plan& p) {
    char buf[160];
    std::snprintf(buf, sizeof(buf),
                  "{\"mapping\": %d, \"warps_per_cta\": %d, \"ctas_per_sm\": %d, \"chunk\": %d}",
                  p.mapping, p.warps_per_cta, p.ctas_per_sm, p.chunk);
    return buf;
}

bool mapping_allowed(int kind, int mapping) {
    switch (kind) {
        case MRIP_MM1:
            return mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_THREAD ||
                   mapping == MRIP_MAP_WARP_1LANE || mapping == MRIP_MAP_WARP_COOP || mapping == MRIP_MAP_CTA;
        case MRIP_TANDEM3:
            return mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_THREAD || mapping == MRIP_MAP_WARP_1LANE ||
                   mapping == MRIP_MAP_WARP_COOP || mapping == MRIP_MAP_CTA;
        case MRIP_FOREST_FIRE: return mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_CTA;
        case MRIP_WALK_L1_EXIT:
            return mapping == MRIP_MAP_AUTO || mapping == MRIP_MAP_THREAD || mapping == MRIP_MAP_WARP_1LANE ||
                   mapping == MRIP_MAP_WARP_COOP || mapping == MRIP_MAP_PERSISTENT;
    }
    return false;
}

std::vector<Plan> candidates(int kind) {
    std::vector<Plan> c;
    auto add = [&](int mapping, int w, int k, int ch) {
        Plan p;
        p.mapping = mapping;
        p.warps_per_cta = w;
        p.ctas_per_sm = k;
        p.chunk = ch;
        c.push_back(p);
    };
    switch (kind) {
        case MRIP_MM1:
            add(MRIP_MAP_THREAD, 0, 0, 0);
            add(MRIP_MAP_CTA, 0, 0, 0);
            add(MRIP_MAP_WARP_COOP, 0, 0, 0);
            add(MRIP_MAP_WARP_1LANE, 0, 0, 0);
            break;
        case MRIP_TANDEM3:
            add(MRIP_MAP_THREAD, 0, 0, 0);
            add(MRIP_MAP_CTA, 0, 0, 0);
            add(MRIP_MAP_WARP_COOP, 0, 0, 0);
            add(MRIP_MAP_WARP_1LANE, 0, 0, 0);
            break;
        case MRIP_FOREST_FIRE: add(MRIP_MAP_CTA, 0, 0, 0); break;
        case MRIP_WALK_L1_EXIT:
            for (int w : {8, 16, 32})
                for (int k : {1, 2, 4})
                    for (int ch : {16, 64}) add(MRIP_MAP_PERSISTENT, w, k, ch);
            add(MRIP_MAP_THREAD, 0, 0, 0);
            add(MRIP_MAP_WARP_COOP, 0, 0, 0);
            add(MRIP_MAP_WARP_1LANE, 0, 0, 0);
            break;
    }
    return c;
}

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    return prop.name;
}

}  // namespace mrip

using namespace mrip;

extern "C" mrip_status mrip_create_model(int kind, const void* params, size_t params_bytes,
                                         mrip_model** out) {
    if (!out) return fail(MRIP_EINVAL, "mrip_create_model: null output");
    *out = nullptr;
    if (!params) return fail(MRIP_EINVAL, "mrip_create_model: null params");
    mrip_model* m = new (std::nothrow) mrip_model();
    if (!m) return fail(MRIP_ENOMEM, "mrip_create_model: host allocation failed");
    m->kind = kind;
    switch (kind) {
        case MRIP_MM1:
            if (params_bytes != sizeof(mrip_mm1_params)) break;
            std::memcpy(&m->mm1, params, sizeof(m->mm1));
            if (m->mm1.n_clients < 1 || m->mm1.n_clients > 0xFFFFFFFFll) {
                delete m;
                return fail(MRIP_EINVAL, "mrip_create_model: n_clients in 1..2^32-1");
            }
            *out = m;
            return MRIP_OK;
        case MRIP_TANDEM3:
            if (params_bytes != sizeof(mrip_tandem3_params)) break;
            std::memcpy(&m->tandem, params, sizeof(m->tandem));
            if (m->tandem.n_clients < 1 || m->tandem.n_clients > 0xFFFFFFFFll || m->tandem.window < 1) {
                delete m;
                return fail(MRIP_EINVAL, "mrip_create_model: n_clients in 1..2^32-1, window >= 1");
            }
            *out = m;
            return MRIP_OK;
        case MRIP_FOREST_FIRE: {
            if (params_bytes != sizeof(mrip_forest_fire_params)) break;
            std::memcpy(&m->ff, params, sizeof(m->ff));
            const int L = m->ff.L;
            if (!(L == 32 || L == 64 || L == 128 || L == 256 || L == 512) || m->ff.n_steps < 1 ||
                !(m->ff.density >= 0.0 && m->ff.density < 1.0) || m->ff.window < 0 ||
                m->ff.window > m->ff.n_steps) {
                delete m;
                return fail(MRIP_EINVAL,
                            "mrip_create_model: L in {32,64,128,256,512}, n_steps >= 1, density in [0,1), "
                            "0 <= window <= n_steps");
            }
            *out = m;
            return MRIP_OK;
        }
        case MRIP_WALK_L1_EXIT:
            if (params_bytes != sizeof(mrip_walk_params)) break;
            std::memcpy(&m->walk, params, sizeof(m->walk));
            if (m->walk.max_steps < 1 || m->walk.max_steps > (1LL << 38)) {
                delete m;
                return fail(MRIP_EINVAL, "mrip_create_model: max_steps in 1..2^38");
            }
            m->plan.mapping = MRIP_MAP_PERSISTENT;
            *out = m;
            return MRIP_OK;
        default:
            delete m;
            return fail(MRIP_EINVAL, "mrip_create_model: unknown kind " + std::to_string(kind));
    }
    delete m;
    return fail(MRIP_EINVAL, "mrip_create_model: params_bytes does not match the kind's struct");
}

extern "C" mrip_status mrip_set_stream(mrip_model* m, void* cuda_stream) {
    if (!m) return fail(MRIP_EINVAL, "mrip_set_stream: null model");
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    return MRIP_OK;
}

extern "C" mrip_status mrip_run_range(mrip_model* m, const double* design_points, int32_t n_dp, int64_t rep_lo,
                                      int64_t rep_hi, uint64_t seed) {
    if (!m || !design_points) return fail(MRIP_EINVAL, "mrip_run: null argument");
    NvtxRange range("mrip_run");
    const int64_t n_reps = rep_hi - rep_lo;
    mrip_status s = check_shape(m, n_dp, n_reps, rep_lo);
    if (s != MRIP_OK) return s;
    m->rep0 = rep_lo;
    s = check_dps(m->kind, design_points, n_dp);
    if (s != MRIP_OK) return s;
    const size_t nval = static_cast<size_t>(n_dp) * dp_dim(m->kind);
    m->host_dps.assign(design_points, design_points + nval);
    s = prepare(m, n_dp, n_reps);
    if (s != MRIP_OK) return s;
    cudaError_t e = cudaMemcpyAsync(m->dps.p, m->host_dps.data(), nval * sizeof(double),
                                    cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_run: design point upload");
    return run_common(m, n_dp, n_reps, seed);
}

extern "C" mrip_status mrip_run(mrip_model* m, const double* design_points, int32_t n_dp, int64_t n_reps,
                                uint64_t seed) {
    return mrip_run_range(m, design_points, n_dp, 0, n_reps, seed);
}

extern "C" mrip_status mrip_run_device(mrip_model* m, const double* d_design_points, int32_t n_dp,
                                       int64_t n_reps, uint64_t seed) {
    if (!m || !d_design_points) return fail(MRIP_EINVAL, "mrip_run_device: null argument");
    mrip_status s = check_shape(m, n_dp, n_reps);
    if (s != MRIP_OK) return s;
    m->rep0 = 0;
    const size_t nval = static_cast<size_t>(n_dp) * dp_dim(m->kind);
    s = prepare(m, n_dp, n_reps);
    if (s != MRIP_OK) return s;
    // validation and the walk's processing order need the values on the host
    m->host_dps.resize(nval);
    cudaError_t e = cudaMemcpyAsync(m->host_dps.data(), d_design_points, nval * sizeof(double),
                                    cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_run_device: design point read");
    s = check_dps(m->kind, m->host_dps.data(), n_dp);
    if (s != MRIP_OK) return s;
    e = cudaMemcpyAsync(m->dps.p, d_design_points, nval * sizeof(double), cudaMemcpyDeviceToDevice,
                        m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_run_device: design point copy");
    return run_common(m, n_dp, n_reps, seed);
}

extern "C" mrip_status mrip_stats(mrip_model* m, double conf, mrip_stat* out) {
    if (!m || !out) return fail(MRIP_EINVAL, "mrip_stats: null argument");
    if (!m->has_run) return fail(MRIP_ESTATE, "mrip_stats: no run yet");
    if (!(conf > 0.0 && conf < 1.0)) return fail(MRIP_EINVAL, "mrip_stats: conf in (0, 1)");
    std::vector<double> h(static_cast<size_t>(m->n_dp) * 3);
    cudaError_t e = cudaMemcpyAsync(h.data(), m->nmm2.p, h.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_stats");
    mrip_status s = mrip_stats_finalize(h.data(), m->n_dp, conf, out);
    if (s != MRIP_OK) return s;
    if (m->kind == MRIP_WALK_L1_EXIT) return mrip_check_device_flags();
    return MRIP_OK;
}

extern "C" mrip_status mrip_moments(mrip_model* m, double* nmm2_out) {
    if (!m || !nmm2_out) return fail(MRIP_EINVAL, "mrip_moments: null argument");
    if (!m->has_run) return fail(MRIP_ESTATE, "mrip_moments: no run yet");
    cudaError_t e = cudaMemcpyAsync(nmm2_out, m->nmm2.p, static_cast<size_t>(m->n_dp) * 3 * sizeof(double),
                                    cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_moments");
    if (m->kind == MRIP_WALK_L1_EXIT) return mrip_check_device_flags();
    return MRIP_OK;
}

extern "C" mrip_status mrip_output_bytes(const mrip_model* m, int which, size_t* bytes) {
    if (!m || !bytes) return fail(MRIP_EINVAL, "mrip_output_bytes: null argument");
    if (!m->has_run) return fail(MRIP_ESTATE, "mrip_output_bytes: no run yet");
    *bytes = plane_bytes(m, which);
    if (*bytes == 0) return fail(MRIP_EINVAL, "mrip_output_bytes: no such output plane");
    return MRIP_OK;
}

extern "C" mrip_status mrip_outputs(mrip_model* m, int which, void* dst, size_t dst_bytes, int on_device) {
    if (!m || !dst) return fail(MRIP_EINVAL, "mrip_outputs: null argument");
    if (!m->has_run) return fail(MRIP_ESTATE, "mrip_outputs: no run yet");
    const size_t bytes = plane_bytes(m, which);
    if (bytes == 0) return fail(MRIP_EINVAL, "mrip_outputs: no such output plane");
    if (dst_bytes < bytes) return fail(MRIP_EINVAL, "mrip_outputs: destination too small");
    const size_t items = static_cast<size_t>(m->n_dp) * m->n_reps;
    const char* src = nullptr;
    switch (m->kind) {
        case MRIP_MM1: src = m->out0.as<char>() + which * items * sizeof(double); break;
        case MRIP_TANDEM3: src = which == 0 ? m->out0.as<char>() : m->out1.as<char>(); break;
        case MRIP_FOREST_FIRE: src = which == 0 ? m->out0.as<char>() : m->out1.as<char>(); break;
        case MRIP_WALK_L1_EXIT: src = m->out0.as<char>(); break;
    }
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_status(e, "mrip_outputs");
    if (m->kind == MRIP_WALK_L1_EXIT) return mrip_check_device_flags();
    return MRIP_OK;
}

extern "C" mrip_status mrip_set_plan(mrip_model* m, const char* plan_json_str) {
    if (!m || !plan_json_str) return fail(MRIP_EINVAL, "mrip_set_plan: null argument");
    Plan p = m->plan;
    std::string err;
    if (!parse_plan(plan_json_str, p, err)) return fail(MRIP_EINVAL, err);
    if (!mapping_allowed(m->kind, p.mapping))
        return fail(MRIP_EINVAL, "mrip_set_plan: mapping not available for this model");
    m->plan = p;
    return MRIP_OK;
}

extern "C" mrip_status mrip_get_plan(const mrip_model* m, char* buf, size_t buf_bytes) {
    if (!m || !buf) return fail(MRIP_EINVAL, "mrip_get_plan: null argument");
    std::string s = plan_json(m->plan);
    if (buf_bytes < s.size() + 1) return fail(MRIP_EINVAL, "mrip_get_plan: buffer too small");
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return MRIP_OK;
}

namespace {
bool outputs_match(int kind, const std::vector<char>& a, const std::vector<char>& b) {
    if (a.size() != b.size()) return false;
    if (kind == MRIP_WALK_L1_EXIT || kind == MRIP_FOREST_FIRE) return std::memcmp(a.data(), b.data(), a.size()) == 0;
    const double* x = reinterpret_cast<const double*>(a.data());
    const double* y = reinterpret_cast<const double*>(b.data());
    for (size_t i = 0; i < a.size() / sizeof(double); ++i) {
        const double tol = 1e-12 * std::fmax(std::fabs(x[i]), std::fabs(y[i])) + 1e-300;
        if (!(std::fabs(x[i] - y[i]) <= tol)) return false;
    }
    return true;
}
}  // namespace

extern "C" mrip_status mrip_autotune(mrip_model* m, const double* design_points, int32_t n_dp, int64_t n_reps,
                                     uint64_t seed, int trials, const char* cache_path) {
    if (!m || !design_points) return fail(MRIP_EINVAL, "mrip_autotune: null argument");
    if (trials < 1) trials = 1;
    char key[256];
    std::snprintf(key, sizeof(key), "kind=%d;n_dp=%d;n_reps=%lld;p=%lld;gpu=%s", m->kind, n_dp,
                  static_cast<long long>(n_reps),
                  static_cast<long long>(m->kind == MRIP_MM1 ? m->mm1.n_clients
                                         : m->kind == MRIP_TANDEM3 ? m->tandem.n_clients
                                         : m->kind == MRIP_FOREST_FIRE ? m->ff.L * 100000LL + m->ff.n_steps
                                                                       : m->walk.max_steps),
                  device_name().c_str());
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            const std::string tag = std::string("\"key\": \"") + key + "\"";
            if (line.find(tag) == std::string::npos) continue;
            size_t at = line.find("\"plan\": ");
            if (at == std::string::npos) continue;
            Plan p;
            std::string err;
            if (parse_plan(line.c_str() + at + 8, p, err) && mapping_allowed(m->kind, p.mapping)) {
                m->plan = p;
                return MRIP_OK;
            }
        }
    }
    const std::vector<Plan> cands = candidates(m->kind);
    const Plan saved = m->plan;
    float best_ms = 1e30f;
    Plan best = saved;
    std::vector<char> ref, cur;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    mrip_status s = MRIP_OK;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        m->plan = cands[ci];
        float cand_best = 1e30f;
        for (int t = 0; t < trials + 1 && s == MRIP_OK; ++t) {
            cudaEventRecord(e0, m->stream);
            s = mrip_run(m, design_points, n_dp, n_reps, seed);
            cudaEventRecord(e1, m->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (t > 0 && ms < cand_best) cand_best = ms;  // the first run captures the graph
        }
        if (s != MRIP_OK) break;
        size_t bytes = plane_bytes(m, 0);
        cur.resize(bytes);
        s = mrip_outputs(m, 0, cur.data(), bytes, 0);
        if (s != MRIP_OK) break;
        if (ci == 0) {
            ref = cur;
        } else if (!outputs_match(m->kind, ref, cur)) {
            s = fail(MRIP_ECUDA, "mrip_autotune: candidate " + plan_json(cands[ci]) +
                                     " disagrees with " + plan_json(cands[0]));
            break;
        }
        if (cand_best < best_ms) {
            best_ms = cand_best;
            best = cands[ci];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MRIP_OK) {
        m->plan = saved;
        return s;
    }
    m->plan = best;
    if (cache_path) {
        std::ofstream outf(cache_path, std::ios::app);
        outf << "{\"key\": \"" << key << "\", \"ms\": " << best_ms << ", \"plan\": " << plan_json(best)
             << "}\n";
    }
    return MRIP_OK;
}

extern "C" mrip_status mrip_run_cv(mrip_model* m, const double* design_points, int32_t n_dp, int64_t n_reps,
                                   uint64_t seed, const mrip_cv_params* params, mrip_stat* plain_out,
                                   mrip_cv_stat* cv_out, mrip_cv_report* report) {
    if (!m || !design_points || !params || !plain_out || !cv_out)
        return fail(MRIP_EINVAL, "mrip_run_cv: null argument");
    NvtxRange range("mrip_run_cv");
    return run_cv_impl(m, design_points, n_dp, n_reps, seed, params, plain_out, cv_out, report);
}

extern "C" mrip_status mrip_cv_network(mrip_model* m, float* theta_out, double* norm_out) {
    if (!m) return fail(MRIP_EINVAL, "mrip_cv_network: null model");
    if (m->cv_d_in == 0) return fail(MRIP_ESTATE, "mrip_cv_network: no mrip_run_cv yet");
    if (theta_out) {
        cudaError_t e = cudaMemcpyAsync(theta_out, m->cv_theta.p, mlp_params(m->cv_d_in) * sizeof(float),
                                        cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return cuda_status(e, "mrip_cv_network");
    }
    if (norm_out) std::memcpy(norm_out, m->cv_norm.data(), m->cv_norm.size() * sizeof(double));
    return MRIP_OK;
}

extern "C" void mrip_destroy(mrip_model* m) { delete m; }
