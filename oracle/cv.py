"""Oracle for the control-variate estimator -- FP64, numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's interval is the plain replication mean (Section 1).  The learned
control variate is the engine's addition; its reading:

Per design point, with n held-out replications (Y_i, g_i), g the network's
prediction from the replication's early window, and M control runs -- the
further replications n_reps .. n_reps + M - 1 of the same streams, simulated
for the early window only -- with predictions g'_m:
    beta  = Cov(Y, g) / Var(g)                (sample moments, n - 1; 0 if Var(g) = 0)
    Y_cv  = mean(Y) - beta (mean(g) - mean(g'))
    s_r^2 = sum_i (r_i - mean(r))^2 / (n - 2),  r_i = Y_i - beta g_i
    Var   = s_r^2 / n + beta^2 Var(g') / M     (Var(g') with M - 1)
    half  = t_{(1+conf)/2, n-2} sqrt(Var)
The control mean is estimated, not known, so its variance enters the
interval.  All sums are exactly rounded (math.fsum).
"""
import math

import numpy as np

from . import t_crit


def _mean(x):
    return math.fsum(np.asarray(x, dtype=np.float64).tolist()) / len(x)


def cv_estimate(y, g, g_ctrl, conf=0.95):
    """Control-variate estimate of one design point (dict)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    gc = np.asarray(g_ctrl, dtype=np.float64).reshape(-1)
    n, M = y.size, gc.size
    if n < 3 or M < 2:
        raise ValueError("need n >= 3 held-out and M >= 2 control runs")
    ybar, gbar, gcbar = _mean(y), _mean(g), _mean(gc)
    dy, dg = y - ybar, g - gbar
    cov = math.fsum((dy * dg).tolist()) / (n - 1)
    var_g = math.fsum((dg * dg).tolist()) / (n - 1)
    beta = cov / var_g if var_g > 0.0 else 0.0
    y_cv = ybar - beta * (gbar - gcbar)
    r = y - beta * g
    rbar = _mean(r)
    dr = r - rbar
    s_r2 = math.fsum((dr * dr).tolist()) / (n - 2)
    dgc = gc - gcbar
    var_gc = math.fsum((dgc * dgc).tolist()) / (M - 1)
    var = s_r2 / n + beta * beta * var_gc / M
    tc = t_crit(conf, n - 2)
    return dict(n=n, m=M, beta=beta, mean=y_cv, var=var, t_crit=tc,
                half_width=tc * math.sqrt(var), y_mean=ybar, g_mean=gbar, g_ctrl_mean=gcbar)


def ff_features(counts, p_grow, p_light, window, L):
    """Forest-fire network inputs of replications with burning counts (n, T):
    log10 p_grow, log10 p_lightning (probabilities floored at 1e-30) and the
    mean burning fraction of the four quarters of the first `window` steps
    (quarter q covers steps floor(q W/4) < t <= floor((q+1) W/4))."""
    counts = np.asarray(counts)
    n = counts.shape[0]
    f = np.empty((n, 6))
    f[:, 0] = np.log10(np.maximum(np.asarray(p_grow, dtype=np.float64), 1e-30))
    f[:, 1] = np.log10(np.maximum(np.asarray(p_light, dtype=np.float64), 1e-30))
    for q in range(4):
        a, b = (q * window) // 4, ((q + 1) * window) // 4
        s = counts[:, a:b].astype(np.int64).sum(axis=1)
        f[:, 2 + q] = s / (float(b - a) * float(L) * float(L)) if b > a else 0.0
    return f


def run_cv(kind, dps, n_reps, seed, n_clients=None, window=100, L=None, n_steps=None,
           density=0.5, train_frac=0.1, epochs=20, batch=1024, lr=1e-3, m_ctrl=None, conf=0.95,
           net_seed=None, threads=1):
    """The whole control-variate pipeline on the CPU (small sizes):
    simulate, build features, train the FP64 network on the first
    ceil(train_frac n) replications of every design point (design-point-major
    order), predict held-out and control runs, and estimate per design
    point.  Returns (plain intervals, cv dicts, last-epoch mean loss)."""
    import math as _m
    from . import all_items, forest_fire, tandem3
    from . import mlp as _mlp
    from . import stats as _st
    dps = np.asarray(dps, dtype=np.float64)
    n_dp = dps.shape[0]
    n_train = int(_m.ceil(train_frac * n_reps))
    n_held = n_reps - n_train
    if m_ctrl is None:
        m_ctrl = 10 * n_held
    net_seed = seed if net_seed is None else net_seed
    dp, rep = all_items(n_dp, n_reps)
    cdp, crep = all_items(n_dp, m_ctrl)
    crep = crep + n_reps
    if kind == "tandem3":
        y, feat = tandem3(dps, dp, rep, n_clients, seed, window=window, threads=threads)
        _, cfeat = tandem3(dps, cdp, crep, window, seed, window=window, threads=threads)
        d_in = 8
    else:
        counts = forest_fire(L, n_steps, dps, density, dp, rep, seed, threads=threads)
        y = counts.sum(axis=1) / (float(n_steps) * L * L)
        feat = ff_features(counts, dps[dp, 0], dps[dp, 1], window, L)
        ccounts = forest_fire(L, window, dps, density, cdp, crep, seed, threads=threads)
        cfeat = ff_features(ccounts, dps[cdp, 0], dps[cdp, 1], window, L)
        d_in = 6
    Y = y.reshape(n_dp, n_reps)
    F = feat.reshape(n_dp, n_reps, d_in)
    plain = [_st.ci(Y[d], conf) for d in range(n_dp)]
    Xtr = F[:, :n_train].reshape(-1, d_in)
    ytr = Y[:, :n_train].reshape(-1)
    theta, norm, losses = _mlp.train(Xtr, ytr, d_in, net_seed, epochs, batch=batch, lr=lr)
    steps_per_epoch = -(-Xtr.shape[0] // batch)
    last = losses[-steps_per_epoch:]
    sizes = np.array([min(batch, Xtr.shape[0] - k * batch) for k in range(steps_per_epoch)], float)
    loss = float((last * sizes).sum() / sizes.sum())
    g_ho = _mlp.predict(theta, F[:, n_train:].reshape(-1, d_in), norm, d_in).reshape(n_dp, n_held)
    g_c = _mlp.predict(theta, cfeat, norm, d_in).reshape(n_dp, m_ctrl)
    g_ho = _mlp.f32(g_ho)
    g_c = _mlp.f32(g_c)
    cv = [cv_estimate(Y[d, n_train:], g_ho[d], g_c[d], conf) for d in range(n_dp)]
    return plain, cv, loss
