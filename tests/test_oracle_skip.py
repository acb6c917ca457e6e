"""Pins for the oracle's skip-sampled forest fire (CPU only).

The variant keeps the automaton's rules and replaces one random word per
cell by the gaps between successive events of each step's growth and
lightning sets.  Pinned here, against facts that do not come from the
oracle: each event set is iid Bernoulli(p) over the cells (count law, per
cell frequency, pair independence, the geometric gap law), the
deterministic fire front with no events, the one-step rule invariants from
random states with the exact rates p (no 2^-32 rounding), and the exact
distribution of the whole 2x2 lattice after two steps (81 states,
enumerated here) -- the same law as the per-cell automaton.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle

EMPTY, TREE, BURN = 0, 1, 2


def _grown_set(L, p, rep, t_steps=1):
    """Cells grown in one step from an empty lattice = that step's growth set."""
    s0 = np.zeros((L, L), np.uint8)
    counts, fin, ties = oracle.forest_fire_skip_rep(L, t_steps, p, 0.0, 0.5, 42, 0, rep, init_state=s0)
    assert ties == 0
    return fin.reshape(-1) == TREE


@pytest.mark.parametrize("p", [0.01, 0.3, 0.9])
def test_growth_set_is_iid_bernoulli(p):
    L, reps = 32, 1500
    n = L * L
    sets = np.array([_grown_set(L, p, r) for r in range(reps)])
    k = sets.sum(axis=1)
    # count ~ Binomial(n, p)
    assert abs(k.mean() - n * p) < 5 * math.sqrt(n * p * (1 - p) / reps)
    assert 0.85 < k.var() / (n * p * (1 - p)) < 1.15
    # every cell has frequency p (chi-square over the cells)
    per_cell = sets.sum(axis=0)
    chi = ((per_cell - reps * p) ** 2 / (reps * p * (1 - p))).sum()
    assert stats.chi2.sf(chi, n) > 1e-4
    # neighbours in index order are independent (the gap structure links them)
    both = (sets[:, :-1] & sets[:, 1:]).sum()
    m = reps * (n - 1)
    assert abs(both - m * p * p) < 5 * math.sqrt(m * p * p * (1 - p * p))


def test_gap_law_is_geometric():
    L, p, reps = 64, 0.05, 300
    gaps = []
    for r in range(reps):
        pos = np.flatnonzero(_grown_set(L, p, r))
        gaps.extend(np.diff(np.concatenate(([-1], pos))) - 1)
    gaps = np.asarray(gaps)
    kmax = 60
    obs = np.array([np.count_nonzero(gaps == k) for k in range(kmax)] + [np.count_nonzero(gaps >= kmax)])
    pk = np.array([p * (1 - p) ** k for k in range(kmax)] + [(1 - p) ** kmax])
    # the last gap of a step is cut by the lattice end; it is excluded by
    # construction (only gaps that end in an event are listed)
    exp = pk * gaps.size
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_lightning_set_rate_and_growth_independent_streams():
    L, reps, pl = 32, 400, 0.02
    s0 = np.full((L, L), TREE, np.uint8)
    hits = 0
    for r in range(reps):
        counts, fin, ties = oracle.forest_fire_skip_rep(L, 1, 0.0, pl, 0.5, 42, 0, r, init_state=s0)
        assert counts[0] == np.count_nonzero(fin == BURN)
        hits += counts[0]
    n = reps * L * L
    assert abs(hits - n * pl) < 5 * math.sqrt(n * pl * (1 - pl))
    # growth and lightning use different streams: same p, different sets
    g = _grown_set(L, pl, 0)
    _, fin, _ = oracle.forest_fire_skip_rep(L, 1, 0.0, pl, 0.5, 42, 0, 0, init_state=s0)
    assert not np.array_equal(g, fin.reshape(-1) == BURN)


def test_no_events_gives_the_deterministic_front():
    L = 32
    s0 = np.full((L, L), TREE, np.uint8)
    s0[16, 16] = BURN
    counts, final, ties = oracle.forest_fire_skip_rep(L, 40, 0.0, 0.0, 0.5, 42, 0, 0, init_state=s0)
    for t in range(1, L // 2):
        assert counts[t - 1] == 4 * t
    assert counts.sum() == L * L - 1
    assert np.all(final == EMPTY) and ties == 0
    # and the initial state is the per-cell automaton's (tag 1)
    _, f_skip, _ = oracle.forest_fire_skip_rep(L, 0, 0.1, 0.1, 0.4, 42, 3, 7)
    _, f_cell = oracle.forest_fire_rep(L, 0, 0.1, 0.1, 0.4, 42, 3, 7)
    assert np.array_equal(f_skip, f_cell)


def test_one_step_rules_from_random_states():
    L = 48
    rng = np.random.default_rng(5)
    pg, pl = 0.2, 0.1
    moved = dict(grow=[0, 0], light=[0, 0])
    for rep in range(30):
        s = rng.integers(0, 3, size=(L, L)).astype(np.uint8)
        counts, s1, _ = oracle.forest_fire_skip_rep(L, 1, pg, pl, 0.5, 42, 0, rep, init_state=s)
        assert counts[0] == np.count_nonzero(s1 == BURN)
        nb = np.zeros((L, L), bool)
        for ax, sh in ((0, 1), (0, -1), (1, 1), (1, -1)):
            nb |= np.roll(s == BURN, sh, axis=ax)
        assert np.all(s1[s == BURN] == EMPTY)
        assert np.all(s1[(s == TREE) & nb] == BURN)
        assert np.all(s1[s == EMPTY] != BURN)
        assert np.all(s1[s == TREE] != EMPTY)
        iso = (s == TREE) & ~nb
        moved["light"][0] += np.count_nonzero(s1[iso] == BURN)
        moved["light"][1] += np.count_nonzero(iso)
        moved["grow"][0] += np.count_nonzero(s1[s == EMPTY] == TREE)
        moved["grow"][1] += np.count_nonzero(s == EMPTY)
    for key, q in (("grow", pg), ("light", pl)):
        k, n = moved[key]
        assert abs(k - n * q) < 5 * math.sqrt(n * q * (1 - q)), key


def _exact_2x2(qg, ql, qd, steps):
    """Distribution over the 81 states of the periodic 2x2 lattice."""
    states = list(itertools.product((EMPTY, TREE, BURN), repeat=4))
    index = {s: i for i, s in enumerate(states)}

    def neighbours(i):
        y, x = divmod(i, 2)
        return [(1 - y) * 2 + x, y * 2 + (1 - x)]

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
    exact, index = _exact_2x2(pg, pl, oracle.threshold(dens) / 2.0**32, steps)
    hist = np.zeros(81)
    for r in range(reps):
        _, fin, _ = oracle.forest_fire_skip_rep(2, steps, pg, pl, dens, 42, 0, r)
        hist[index[tuple(int(v) for v in fin.reshape(-1))]] += 1
    expect = exact * reps
    keep = expect >= 5
    obs = np.append(hist[keep], hist[~keep].sum())
    exp = np.append(expect[keep], expect[~keep].sum())
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
        assert hist[~keep].sum() == 0
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_batch_matches_single_and_ties_are_rare():
    dps = [[0.01, 1e-5], [0.05, 1e-4]]
    dp = np.array([0, 1, 1], np.int32)
    rep = np.array([0, 2, 5], np.int64)
    counts, ties = oracle.forest_fire_skip(64, 200, dps, 0.5, dp, rep, 42)
    for i in range(3):
        c, _, t = oracle.forest_fire_skip_rep(64, 200, *dps[dp[i]], 0.5, 42, dp[i], rep[i])
        assert np.array_equal(counts[i], c) and ties[i] == t
    assert ties.sum() == 0
