"""Oracle statistics: per-design-point mean, variance and Student-t interval.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper builds a confidence interval from replications by the Central Limit
Theorem and recommends at least 30 replications (Section 1).  With the
variance estimated from the same replications the interval is
mean +/- t_{(1+conf)/2, n-1} * sqrt(s^2 / n).  Everything here is the
two-pass definition with exactly rounded sums (math.fsum), FP64: s^2 is the
sum of squared deviations from the exact mean; the deviations are taken
from the rounded mean m and the sum d of those deviations removes its
rounding, sum (x - mean)^2 = sum (x - m)^2 - d^2 / n (an identity).
"""
import math

import numpy as np

from . import t_crit


def dp_stats(x):
    """(n, mean, unbiased variance) of one design point's outputs, two-pass."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    n = x.size
    if n == 0:
        raise ValueError("no replications")
    mean = math.fsum(x.tolist()) / n
    if n < 2:
        return n, mean, float("nan")
    dev = x - mean
    d = math.fsum(dev.tolist())
    var = (math.fsum((dev * dev).tolist()) - d * d / n) / (n - 1)
    return n, mean, var


def ci(x, conf=0.95):
    """Student-t interval of one design point: dict(n, mean, var, t_crit, half_width)."""
    n, mean, var = dp_stats(x)
    if n < 2:
        return dict(n=n, mean=mean, var=var, t_crit=float("nan"), half_width=float("nan"))
    tc = t_crit(conf, n - 1)
    return dict(n=n, mean=mean, var=var, t_crit=tc, half_width=tc * math.sqrt(var / n))


def ci_table(values, conf=0.95):
    """Row-wise ci() of a (n_dp, n_reps) array."""
    values = np.asarray(values, dtype=np.float64)
    return [ci(row, conf) for row in values]
