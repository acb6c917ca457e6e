"""Seeded synthetic inputs shared by the tests, the bench and the oracle side.

This module holds workload definitions (sizes, rates, probabilities) and
seeded generators of input arrays.  It contains none of the method's
arithmetic: no random stream of the method, no model, no statistic.  Design
points that the workloads draw at random come from numpy's PCG64
(``numpy.random.default_rng``) and are then passed, as plain inputs, to both
the CUDA path and the oracle.

Workloads (one per model; sizes follow the MRIP experiments of the paper,
Section 5, scaled to a modern GPU):

* ``mm1_32``        M/M/1 via Lindley, lambda=0.9, mu=1, 1,000 clients,
                    32 replications, 1 design point, seed 42.
* ``mm1_64k``       the same model with 2^16 replications (the throughput
                    row beside the latency-bound 32).
* ``ff128``         forest fire 128x128, p_grow=0.01, p_lightning=1e-5,
                    density 0.5, 1,000 steps, 1,024 replications.
* ``walk8``         L1-exit walk, R in {16,32,48,64,96,128,192,256},
                    2^17 replications each.
* ``tandem_cv``     3-station tandem, 4,096 design points lambda~U[0.5,0.95],
                    mu_j~U[1.0,1.5], 256 replications x 10,000 clients,
                    network 8-64-64-1 trained on 10 % of the replications.
* ``ff256_cv``      forest fire 256x256, 64 design points p_grow geometric
                    from 1e-3 to 5e-2 (endpoints included), p_lightning=1e-5,
                    2,000 steps, 128 replications each (8,192 in total),
                    network 6-64-64-1.
"""
import numpy as np

SEED = 42

WALK_RADII = (16, 32, 48, 64, 96, 128, 192, 256)


def tandem_design_points(n_dp=4096, seed=SEED):
    """(n_dp, 4) array of (lambda, mu1, mu2, mu3), uniform as stated above."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(0.5, 0.95, size=n_dp)
    mu = rng.uniform(1.0, 1.5, size=(n_dp, 3))
    return np.ascontiguousarray(np.column_stack([lam, mu]), dtype=np.float64)


def ff_cv_design_points(n_dp=64, p_light=1e-5):
    """(n_dp, 2) array of (p_grow, p_lightning): p_grow = 1e-3 * 50^(i/(n_dp-1))."""
    i = np.arange(n_dp, dtype=np.float64)
    p_grow = 1e-3 * np.power(50.0, i / max(n_dp - 1, 1))
    return np.ascontiguousarray(np.column_stack([p_grow, np.full(n_dp, p_light)]))


WORKLOADS = {
    "mm1_32": dict(kind="mm1", dps=np.array([[0.9, 1.0]]), n_reps=32, n_clients=1000,
                   seed=SEED),
    "mm1_64k": dict(kind="mm1", dps=np.array([[0.9, 1.0]]), n_reps=1 << 16, n_clients=1000,
                    seed=SEED),
    "ff128": dict(kind="forest_fire", L=128, n_steps=1000, dps=np.array([[0.01, 1e-5]]),
                  density=0.5, n_reps=1024, seed=SEED),
    "walk8": dict(kind="walk", dps=np.array(WALK_RADII, dtype=np.float64)[:, None],
                  n_reps=1 << 17, seed=SEED),
    "tandem_cv": dict(kind="tandem3", dps=None, n_dp=4096, n_reps=256, n_clients=10000,
                      window=100, train_frac=0.1, seed=SEED),
    "ff256_cv": dict(kind="forest_fire", L=256, n_steps=2000, dps=None, n_dp=64,
                     density=0.5, n_reps=128, window=100, train_frac=0.1, seed=SEED),
}


def workload(name):
    """A copy of a workload definition with its design points filled in."""
    w = dict(WORKLOADS[name])
    if name == "tandem_cv":
        w["dps"] = tandem_design_points(w["n_dp"], w["seed"])
    elif name == "ff256_cv":
        w["dps"] = ff_cv_design_points(w["n_dp"])
    w["dps"] = np.ascontiguousarray(np.asarray(w["dps"], dtype=np.float64))
    w["n_dp"] = w["dps"].shape[0]
    return w


# ---------------------------------------------------------------------------
# Seeded arrays for stage-level checks (network, estimator, statistics)
# ---------------------------------------------------------------------------
def random_matrix(shape, seed, scale=1.0, loc=0.0):
    """Gaussian array of the given shape."""
    rng = np.random.default_rng(seed)
    return loc + scale * rng.standard_normal(size=shape)


def random_uniform(shape, seed, lo=0.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape)


def correlated_pair(n, rho, seed, loc=(5.0, 1.0), scale=(2.0, 0.5)):
    """(y, g) with correlation rho, for estimator checks."""
    rng = np.random.default_rng(seed)
    z1 = rng.standard_normal(n)
    z2 = rng.standard_normal(n)
    g = z1
    y = rho * z1 + np.sqrt(max(1.0 - rho * rho, 0.0)) * z2
    return loc[0] + scale[0] * y, loc[1] + scale[1] * g
