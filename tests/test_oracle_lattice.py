"""Pins for the oracle's forest-fire automaton and L1-exit walk (CPU only).

Forest fire: a deterministic fire front on a full forest (4t burning cells at
step t until the front wraps, every tree burns once), conservation and rule
invariants from random states, the rates of growth and lightning, and the
exact distribution of the whole 2x2 lattice after two steps (81 states,
enumerated here) against the oracle's empirical frequencies.

Walk: R = 1 and R = 2 in closed form, the exact distribution of the exit time
for R <= 6 by dynamic programming over the interior of the L1 ball, and the
parity tau = R (mod 2).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle

EMPTY, TREE, BURN = 0, 1, 2


# ---------------------------------------------------------------- forest fire
def test_fire_front_on_full_forest():
    L = 32
    s0 = np.full((L, L), TREE, np.uint8)
    s0[16, 16] = BURN
    counts, final = oracle.forest_fire_rep(L, 40, 0.0, 0.0, 0.5, 42, 0, 0, init_state=s0)
    for t in range(1, L // 2):
        assert counts[t - 1] == 4 * t
    assert counts.sum() == L * L - 1        # every tree burns exactly once
    assert counts[-1] == 0 and np.all(final == EMPTY)


def test_no_fire_without_lightning_and_binomial_density():
    L, reps = 32, 400
    counts = oracle.forest_fire(L, 20, [[0.05, 0.0]], 0.5, np.zeros(reps, np.int32),
                                np.arange(reps), 42)
    assert np.all(counts == 0)
    trees = np.array([np.count_nonzero(oracle.forest_fire_rep(L, 0, 0.0, 0.0, 0.5, 42, 0, r)[1]
                                       == TREE) for r in range(reps)])
    # Binomial(L^2, 1/2): mean and variance
    assert abs(trees.mean() - L * L / 2) < 5 * math.sqrt(L * L / 4 / reps)
    assert 0.7 < trees.var() / (L * L / 4) < 1.3


def test_one_step_rules_from_random_states():
    L = 48
    rng = np.random.default_rng(3)
    pg, pl = 0.2, 0.1
    moved = dict(grow=[0, 0], light=[0, 0])
    for rep in range(30):
        s = rng.integers(0, 3, size=(L, L)).astype(np.uint8)
        counts, s1 = oracle.forest_fire_rep(L, 1, pg, pl, 0.5, 42, 0, rep, init_state=s)
        assert counts[0] == np.count_nonzero(s1 == BURN)
        nb = np.zeros((L, L), bool)
        for ax, sh in ((0, 1), (0, -1), (1, 1), (1, -1)):
            nb |= np.roll(s == BURN, sh, axis=ax)
        assert np.all(s1[s == BURN] == EMPTY)               # burning -> empty
        assert np.all(s1[(s == TREE) & nb] == BURN)         # fire spreads
        assert np.all(s1[s == EMPTY] != BURN)               # empty never ignites
        assert np.all(s1[s == TREE] != EMPTY)               # trees never vanish
        iso = (s == TREE) & ~nb
        moved["light"][0] += np.count_nonzero(s1[iso] == BURN)
        moved["light"][1] += np.count_nonzero(iso)
        moved["grow"][0] += np.count_nonzero(s1[s == EMPTY] == TREE)
        moved["grow"][1] += np.count_nonzero(s == EMPTY)
    for key, p in (("grow", pg), ("light", pl)):
        k, n = moved[key]
        q = oracle.threshold(p) / 2.0**32
        assert abs(k - n * q) < 5 * math.sqrt(n * q * (1 - q)), key


def _exact_2x2(pg, pl, density, steps):
    """Distribution over the 81 states of the periodic 2x2 lattice."""
    qg = oracle.threshold(pg) / 2.0**32
    ql = oracle.threshold(pl) / 2.0**32
    qd = oracle.threshold(density) / 2.0**32
    states = list(itertools.product((EMPTY, TREE, BURN), repeat=4))
    index = {s: i for i, s in enumerate(states)}

    def neighbours(i):
        y, x = divmod(i, 2)
        return [(1 - y) * 2 + x, y * 2 + (1 - x)]   # up = down, left = right on 2x2

    P = np.zeros((81, 81))
    for s in states:
        per_cell = []
        for i in range(4):
            if s[i] == BURN:
                per_cell.append({EMPTY: 1.0})
            elif s[i] == TREE:
                if any(s[j] == BURN for j in neighbours(i)):
                    per_cell.append({BURN: 1.0})
                else:
                    per_cell.append({BURN: ql, TREE: 1.0 - ql})
            else:
                per_cell.append({TREE: qg, EMPTY: 1.0 - qg})
        for combo in itertools.product(*[list(d.items()) for d in per_cell]):
            nxt = tuple(c[0] for c in combo)
            P[index[s], index[nxt]] += np.prod([c[1] for c in combo])
    p0 = np.zeros(81)
    for s in itertools.product((EMPTY, TREE), repeat=4):
        p0[index[s]] = np.prod([qd if c == TREE else 1.0 - qd for c in s])
    dist = p0
    for _ in range(steps):
        dist = dist @ P
    return dist, index


def test_2x2_lattice_distribution_brute_force():
    pg, pl, dens, steps, reps = 0.3, 0.2, 0.5, 2, 40000
    exact, index = _exact_2x2(pg, pl, dens, steps)
    assert exact.sum() == pytest.approx(1.0, abs=1e-12)
    hist = np.zeros(81)
    for r in range(reps):
        _, fin = oracle.forest_fire_rep(2, steps, pg, pl, dens, 42, 0, r)
        hist[index[tuple(int(v) for v in fin.reshape(-1))]] += 1
    expect = exact * reps
    keep = expect >= 5
    obs = np.append(hist[keep], hist[~keep].sum())
    exp = np.append(expect[keep], expect[~keep].sum())
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
        assert hist[~keep].sum() == 0
    assert stats.chisquare(obs, exp).pvalue > 1e-4


# ---------------------------------------------------------------- walk
def _exact_exit_distribution(R, kmax):
    pts = [(x, y) for x in range(-R, R + 1) for y in range(-R, R + 1) if abs(x) + abs(y) < R]
    idx = {p: i for i, p in enumerate(pts)}
    assert len(pts) == 2 * R * R - 2 * R + 1
    dist = np.zeros(len(pts))
    dist[idx[(0, 0)]] = 1.0
    out = np.zeros(kmax + 1)
    for k in range(1, kmax + 1):
        new = np.zeros_like(dist)
        exit_p = 0.0
        for (x, y), i in idx.items():
            if dist[i] == 0.0:
                continue
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                q = (x + dx, y + dy)
                if q in idx:
                    new[idx[q]] += 0.25 * dist[i]
                else:
                    exit_p += 0.25 * dist[i]
        out[k] = exit_p
        dist = new
    return out


def test_walk_radius_one_and_two():
    n = 4000
    tau1 = oracle.walk([1.0], np.zeros(n, np.int32), np.arange(n), 42)
    assert np.all(tau1 == 1)
    tau2 = oracle.walk([2.0], np.zeros(n, np.int32), np.arange(n), 42)
    assert np.all(tau2 % 2 == 0) and tau2.min() == 2
    # P(tau = 2k) = 3/4 (1/4)^(k-1), E[tau] = 8/3
    k = tau2 // 2
    hist = np.bincount(k, minlength=8)[1:]
    probs = np.array([0.75 * 0.25 ** (j - 1) for j in range(1, len(hist) + 1)])
    exp = probs * n
    keep = exp >= 5
    obs = np.append(hist[keep], hist[~keep].sum())
    ex = np.append(exp[keep], n - exp[keep].sum())
    assert stats.chisquare(obs, ex).pvalue > 1e-4
    assert abs(tau2.mean() - 8 / 3) < 5 * math.sqrt(np.var(tau2) / n)


@pytest.mark.parametrize("R", [3, 4, 6])
def test_walk_exact_distribution_small_radius(R):
    n = 20000
    tau = oracle.walk([float(R)], np.zeros(n, np.int32), np.arange(n), 42)
    assert np.all(tau % 2 == R % 2)
    kmax = max(int(tau.max()) + 50, 60 * R * R)
    p = _exact_exit_distribution(R, kmax)
    assert p.sum() == pytest.approx(1.0, abs=1e-9)
    exp = p * n
    hist = np.bincount(tau, minlength=kmax + 1).astype(float)
    keep = exp >= 5
    obs = np.append(hist[keep], hist[~keep].sum())
    ex = np.append(exp[keep], n - exp[keep].sum())
    assert stats.chisquare(obs, ex).pvalue > 1e-4
    mean_exact = float((np.arange(kmax + 1) * p).sum())
    assert abs(tau.mean() - mean_exact) < 5 * math.sqrt(np.var(tau) / n)


def _exit_survival_1d(R, kmax):
    """P(T > k), k = 0..kmax, for a +-1 walk from 0 and T the first k with
    |position| >= R (dynamic programming over the 2R - 1 inner sites)."""
    p = np.zeros(2 * R - 1)
    p[R - 1] = 1.0
    surv = np.empty(kmax + 1)
    surv[0] = 1.0
    for k in range(1, kmax + 1):
        q = np.zeros_like(p)
        q[1:] += 0.5 * p[:-1]
        q[:-1] += 0.5 * p[1:]
        p = q
        surv[k] = p.sum()
    return surv


@pytest.mark.parametrize("R", [16, 33])
def test_walk_exact_distribution_by_diagonal_coordinates(R):
    """In u = x + y, v = x - y a move steps u and v by independent fair +-1
    (u's sign is bit 0, v's the xor of the two bits) and |x| + |y| >= R iff
    max(|u|, |v|) >= R, so P(tau > k) = P(T > k)^2 with T the exit time of a
    1-D walk from (-R, R): an exact law at the radii the GPU tests use,
    derived independently of the 2-D dynamic programming above."""
    n = 20000
    tau = oracle.walk([float(R)], np.zeros(n, np.int32), np.arange(n), 7)
    kmax = int(tau.max()) + 40 * R * R
    surv = _exit_survival_1d(R, kmax) ** 2
    p = np.append(surv[:-1] - surv[1:], surv[-1])  # P(tau = k), k = 1..kmax, then the rest
    # bins of roughly equal probability along the exact CDF
    cdf = np.cumsum(p)
    edges = np.searchsorted(cdf, np.linspace(0, 1, 41)[1:-1]) + 1
    edges = np.unique(np.concatenate([[1], edges, [kmax + 1]]))
    ex = np.array([p[lo - 1:hi - 1].sum() for lo, hi in zip(edges[:-1], edges[1:])]) * n
    obs = np.array([np.count_nonzero((tau >= lo) & (tau < hi)) for lo, hi in zip(edges[:-1], edges[1:])])
    ex[-1] += n * p[kmax:].sum()
    assert np.all(ex >= 5) and obs.sum() == n
    assert stats.chisquare(obs, ex * n / ex.sum()).pvalue > 1e-4
    mean_exact = float(surv[:-1].sum())  # E[tau] = sum_k P(tau > k)
    assert abs(tau.mean() - mean_exact) < 5 * math.sqrt(np.var(tau) / n)


def test_walk_parity_large_radius_and_cap():
    radii = [16.0, 33.0]
    dp = np.repeat(np.arange(2, dtype=np.int32), 300)
    rep = np.tile(np.arange(300), 2)
    tau = oracle.walk(radii, dp, rep, 42)
    assert np.all(tau[dp == 0] % 2 == 0) and np.all(tau[dp == 1] % 2 == 1)
    assert np.all(tau[dp == 0] >= 16) and np.all(tau[dp == 1] >= 33)
    # E[tau] grows like R^2: between R^2/2 and R^2
    for d, R in enumerate(radii):
        assert 0.4 * R * R < tau[dp == d].mean() < 1.0 * R * R
    capped = oracle.walk([64.0], [0], [0], 42, max_steps=10)
    assert capped[0] == -1


# ---------------------------------------------------------------- area walk
def _area_walk_exact(n_steps, W=60, Hh=50, cell=10):
    """Exact position law of the walk on the W x H torus by dynamic
    programming; returns (final-area probabilities, expected visits)."""
    p = np.zeros((Hh, W))
    p[Hh // 2, W // 2] = 1.0
    area = (np.arange(W)[None, :] // cell) + (W // cell) * (np.arange(Hh)[:, None] // cell)
    visits = np.zeros(30)
    for _ in range(n_steps):
        p = 0.25 * (np.roll(p, 1, 1) + np.roll(p, -1, 1) + np.roll(p, 1, 0) + np.roll(p, -1, 0))
        visits += np.bincount(area.ravel(), weights=p.ravel(), minlength=30)
    final = np.bincount(area.ravel(), weights=p.ravel(), minlength=30)
    return final, visits


def test_area_walk_counts_and_exact_law():
    n, steps = 20000, 1000
    final, visits = oracle.area_walk(np.arange(n), steps, 42, threads=oracle.host_threads())
    assert np.all(visits.sum(axis=1) == steps)
    assert final.min() >= 0 and final.max() < 30
    p_final, e_visits = _area_walk_exact(steps)
    assert p_final.sum() == pytest.approx(1.0, abs=1e-12)
    hist = np.bincount(final, minlength=30).astype(float)
    exp = p_final * n
    keep = exp >= 5
    obs = np.append(hist[keep], hist[~keep].sum())
    ex = np.append(exp[keep], n - exp[keep].sum())
    assert stats.chisquare(obs, ex).pvalue > 1e-4
    # mean visit counts per area against the exact expectation
    m = visits.mean(axis=0)
    se = visits.std(axis=0, ddof=1) / math.sqrt(n)
    z = np.abs(m - e_visits) / np.maximum(se, 1e-12)
    assert np.all(z[se > 0] < 5) and np.all(m[se == 0] == e_visits[se == 0].round())


def test_area_walk_one_step_and_long_run_uniformity():
    final, visits = oracle.area_walk(np.arange(400), 1, 7)
    # one move from (30, 25) stays in area 3 + 6*2 = 15 unless it leaves the block
    assert set(np.unique(final)) <= {14, 15}
    n, steps = 64, 200000
    _, visits = oracle.area_walk(np.arange(n), steps, 3, threads=oracle.host_threads())
    frac = visits.sum(axis=0) / (n * steps)
    assert np.all(np.abs(frac - 1 / 30) < 0.012)  # stationary law: uniform over the torus
