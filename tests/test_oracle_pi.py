"""Pins for the oracle's Monte Carlo pi (paper, Section 5.1, first model).

* the overflow-free inside test equals the definition x^2 + y^2 < 2^64
  evaluated with unbounded integers, draw by draw;
* hits are Binomial(n, pi/4) (the lattice of 2^64 points deviates from the
  disc by far less than the binomial spread): total frequency and spread;
* the 99 % Student-t interval of 64 replications covers pi.
"""
import math

import numpy as np

import oracle
import oracle.stats as ostats


def test_inside_test_matches_unbounded_integers():
    n = 3001
    blocks = oracle.stream_block(42, 0, 0, 5, np.arange((n + 1) // 2), 0)
    hits = 0
    for k in range(n):
        w = blocks[k // 2]
        x, y = int(w[2 * (k % 2)]), int(w[2 * (k % 2) + 1])
        hits += x * x + y * y < 2**64
    assert oracle.pi_hits([5], n, 42)[0] == hits
    assert oracle.pi_hits([5], 0, 42)[0] == 0


def test_binomial_law_and_interval_covers_pi():
    n_draws, reps = 10**6, 64
    h = oracle.pi_hits(np.arange(reps), n_draws, 7, threads=oracle.host_threads())
    p = math.pi / 4
    tot = h.sum()
    assert abs(tot - reps * n_draws * p) < 5 * math.sqrt(reps * n_draws * p * (1 - p))
    assert 0.6 < h.var(ddof=1) / (n_draws * p * (1 - p)) < 1.5
    c = ostats.ci(4.0 * h / n_draws, 0.99)
    assert abs(c["mean"] - math.pi) <= c["half_width"]
