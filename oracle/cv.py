"""Oracle for the control-variate estimator -- FP64, numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's interval is the plain replication mean (Section 1).  The learned
control variate is the engine's addition; its reading:

Per design point, with n held-out replications (Y_i, g_i), g the network's
prediction from the replication's early window, and M independent control
runs of the early window only (tag 2) with predictions g'_m:
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
