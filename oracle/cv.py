"""Oracle for the control-variate estimator -- FP64, numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's interval is the plain replication mean (Section 1).  The learned
control variate is the engine's addition; its reading:

Per design point, with n held-out replications (Y_i, g_i), g the network's
prediction from the replication's early window, and M control runs -- the
further replications n_reps .. n_reps + M - 1 of the same streams (tag 0),
simulated for the early window only -- with predictions g'_m:
    beta  = Cov(Y, g) / Var(g)                (sample moments, n - 1; 0 if Var(g) = 0)
    Y_cv  = mean(Y) - beta (mean(g) - mean(g'))
    s_r^2 = sum_i (r_i - mean(r))^2 / (n - 2),  r_i = Y_i - beta g_i
    Var   = s_r^2 / n + beta^2 Var(g') / M     (Var(g') with M - 1)
    half  = t_{(1+conf)/2, n-2} sqrt(Var)
The control mean is estimated, not known, so its variance enters the
interval.  All sums are exactly rounded (math.fsum).

Sizing and gate (the plain estimator of Section 1 stays the fallback): with
rho^2 the pooled within-design-point squared correlation of Y and g on
validation replications (never used by the estimator; each design point's
deviations scaled by its fit-set standard deviations, so that design points
of large variance do not outweigh the others), the optimal beta
leaves a residual variance (1 - rho^2) s^2 and the control mean adds about
rho^2 s^2 / M, so M = ceil(n rho^2 / (0.1 (1 - rho^2))) keeps that term to a
tenth of the residual one, and the control-variate estimator beats the
plain one on all n_reps replications only if
n_reps ((1 - rho^2) / n + rho^2 / M) < 1, i.e. (M sized so) rho^2 above
about 1 - n / (1.1 n_reps).  A network trained for the first
ceil(64 / steps per epoch) epochs whose validation rho^2 is below a quarter
of that declines without further training.
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


def within_rho2(y, g, y_fit=None, g_fit=None):
    """Pooled within-design-point squared correlation of (y, g), both shaped
    (n_dp, n): per design point the sums of products of deviations from its
    own means, added over the design points in order.  With y_fit, g_fit
    (n_dp, n_fit) each design point's deviations are first divided by its
    population standard deviations over those, so that every design point
    weighs the same (a design point with a constant y_fit or g_fit is
    left out)."""
    y = np.asarray(y, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    syg = syy = sgg = 0.0
    for d, (yr, gr) in enumerate(zip(y, g)):
        sy = sg = 1.0
        if y_fit is not None:
            yf = np.asarray(y_fit[d], dtype=np.float64)
            gf = np.asarray(g_fit[d], dtype=np.float64)
            sy = math.sqrt(math.fsum(((yf - _mean(yf)) ** 2).tolist()) / len(yf))
            sg = math.sqrt(math.fsum(((gf - _mean(gf)) ** 2).tolist()) / len(gf))
            if not (sy > 0.0 and sg > 0.0):
                continue
        dy = (yr - _mean(yr)) / sy
        dg = (gr - _mean(gr)) / sg
        syg += math.fsum((dy * dg).tolist())
        syy += math.fsum((dy * dy).tolist())
        sgg += math.fsum((dg * dg).tolist())
    return (syg * syg) / (syy * sgg) if syy > 0.0 and sgg > 0.0 else 0.0


def control_runs(rho2, n_held):
    """Control runs per design point: the control mean's variance term
    beta^2 Var(g') / M ~ rho^2 s^2 / M kept to a tenth of the residual term
    (1 - rho^2) s^2 / n_held, within [2, 100 n_held]; 10 n_held without a
    validation estimate."""
    if rho2 is None or not rho2 >= 0.0:
        return 10 * n_held
    r = min(rho2, 0.999999)
    m = min(math.ceil(n_held * r / (0.1 * (1.0 - r))), 100 * n_held)
    return max(2, int(m))


def var_ratio(rho2, n_reps, n_held, M):
    """Predicted Var(control variate) / Var(plain) at n_reps replications."""
    return n_reps * ((1.0 - rho2) / n_held + rho2 / M)


def run_cv(kind, dps, n_reps, seed, n_clients=None, window=100, L=None, n_steps=None,
           density=0.5, train_frac=0.1, val_frac=0.0, epochs=20, patience=0, batch=1024, lr=1e-3,
           gate=False, m_ctrl=None, conf=0.95, net_seed=None, theta=None, threads=1):
    """The whole control-variate pipeline on the CPU (small sizes):
    simulate; build features; split each design point's replications into
    fit [0, n_fit), validation [n_fit, n_train) and held-out [n_train, n_reps)
    (n_train = ceil(train_frac n_reps), n_val = ceil(val_frac n_train));
    standardise with the fit set's moments; train the FP64 network on the fit
    set (design-point-major order) with early stopping on the validation set
    -- or, with `theta` given, take that network; estimate the pooled
    within-design-point rho^2 on the validation set; size the control runs
    (m_ctrl None or 0: control_runs); with `gate`, decline right after
    the first ceil(64 / steps per epoch) epochs when the validation rho^2
    is below a quarter of the break-even 1 - n_held / (1.1 n_reps) (the
    screen), and after training when the
    predicted variance ratio is >= 1 (cv = the plain intervals); else
    predict held-out and control runs and estimate per design point.
    Returns (plain intervals, cv dicts, info dict)."""
    import math as _m
    from . import all_items, forest_fire, tandem3
    from . import mlp as _mlp
    from . import stats as _st
    dps = np.asarray(dps, dtype=np.float64)
    n_dp = dps.shape[0]
    n_train = int(_m.ceil(train_frac * n_reps))
    n_held = n_reps - n_train
    n_val = int(_m.ceil(val_frac * n_train)) if val_frac > 0 else 0
    n_fit = n_train - n_val
    net_seed = seed if net_seed is None else net_seed
    dp, rep = all_items(n_dp, n_reps)
    if kind == "tandem3":
        y, feat = tandem3(dps, dp, rep, n_clients, seed, window=window, threads=threads)
        d_in = 8
    else:
        counts = forest_fire(L, n_steps, dps, density, dp, rep, seed, threads=threads)
        y = counts.sum(axis=1) / (float(n_steps) * L * L)
        feat = ff_features(counts, dps[dp, 0], dps[dp, 1], window, L)
        d_in = 6
    Y = y.reshape(n_dp, n_reps)
    F = feat.reshape(n_dp, n_reps, d_in)
    plain = [_st.ci(Y[d], conf) for d in range(n_dp)]
    Xfit = F[:, :n_fit].reshape(-1, d_in)
    yfit = Y[:, :n_fit].reshape(-1)
    Xval = F[:, n_fit:n_train].reshape(-1, d_in)
    yval = Y[:, n_fit:n_train].reshape(-1)
    def val_rho2(th, nrm):
        g_val = _mlp.f32(_mlp.predict(th, Xval, nrm, d_in)).reshape(n_dp, n_val)
        g_fit = _mlp.f32(_mlp.predict(th, Xfit, nrm, d_in)).reshape(n_dp, n_fit)
        return within_rho2(Y[:, n_fit:n_train], g_val, Y[:, :n_fit], g_fit)

    # the screen: after the first ceil(64 / steps per epoch) epochs (at least
    # 64 Adam steps), a validation rho^2 below a quarter of the break-even
    # value 1 - n_held / (1.1 n_reps) declines at once
    rho2_be = 1.0 - n_held / (1.1 * n_reps)
    screen = {"rho2": None}
    spe = -(-Xfit.shape[0] // batch)
    screen_epochs = min(epochs, -(-64 // spe))

    def after_epoch(e, th, nrm):
        if e != screen_epochs or not gate or screen_epochs >= epochs or n_val < 2:
            return False
        screen["rho2"] = val_rho2(th, nrm)
        return screen["rho2"] < 0.25 * rho2_be

    if theta is None:
        theta, norm, losses, tinfo = _mlp.train(Xfit, yfit, d_in, net_seed, epochs, batch=batch,
                                                lr=lr, X_val=Xval if n_val else None,
                                                y_val=yval if n_val else None, patience=patience,
                                                after_epoch=after_epoch)
        spe = -(-Xfit.shape[0] // batch)
        last = losses[(tinfo["epochs_run"] - 1) * spe:tinfo["epochs_run"] * spe]
        sizes = np.array([min(batch, Xfit.shape[0] - k * batch) for k in range(spe)], float)
        loss = float((last * sizes).sum() / sizes.sum())
    else:
        theta = np.asarray(theta, dtype=np.float64)
        xm, xs = _mlp.standardizer(Xfit)
        ym, ys = _mlp.standardizer(yfit)
        norm = (xm, xs, ym[0], ys[0])
        tinfo, loss = dict(val_losses=np.array([]), epochs_run=0, best_epoch=0), float("nan")
    screened = bool(tinfo.get("stopped_by_callback"))
    rho2 = None
    if n_val >= 2:
        rho2 = screen["rho2"] if screened else val_rho2(theta, norm)
    M = int(m_ctrl) if m_ctrl else control_runs(rho2, n_held)
    ratio = var_ratio(rho2, n_reps, n_held, M) if rho2 is not None else None
    info = dict(loss=loss, val_rho2=rho2, var_ratio=ratio, m_ctrl=M, theta=theta, norm=norm,
                declined=False, screened=screened, **tinfo)
    if gate and ratio is not None and (screened or ratio >= 1.0):
        info.update(declined=True, m_ctrl=0)
        cv = [dict(n=p["n"], m=0, beta=0.0, mean=p["mean"], var=p["var"] / p["n"],
                   half_width=p["half_width"], t_crit=p["t_crit"]) for p in plain]
        return plain, cv, info
    cdp, crep = all_items(n_dp, M)
    crep = crep + n_reps
    if kind == "tandem3":
        _, cfeat = tandem3(dps, cdp, crep, window, seed, window=window, threads=threads)
    else:
        ccounts = forest_fire(L, window, dps, density, cdp, crep, seed, threads=threads)
        cfeat = ff_features(ccounts, dps[cdp, 0], dps[cdp, 1], window, L)
    g_ho = _mlp.predict(theta, F[:, n_train:].reshape(-1, d_in), norm, d_in).reshape(n_dp, n_held)
    g_c = _mlp.predict(theta, cfeat, norm, d_in).reshape(n_dp, M)
    g_ho = _mlp.f32(g_ho)
    g_c = _mlp.f32(g_c)
    cv = [cv_estimate(Y[d, n_train:], g_ho[d], g_c[d], conf) for d in range(n_dp)]
    return plain, cv, info
