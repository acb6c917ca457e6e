"""Pins for the oracle's variates, M/M/1 and tandem queues (CPU only).

* u53 / exponential: exact grid, boundary words, mean and KS against the
  exponential law.
* M/M/1 (paper, Section 5.1): the Lindley recurrence equals an event-driven
  simulation written here on the same variates; long runs cover the textbook
  steady state (mean wait rho/(mu-lambda), idle per client (1-rho)/lambda,
  time in system 1/(mu-lambda)).
* Tandem: the arrival-relative recurrence equals an absolute-clock
  event-driven simulation; with stations 2 and 3 made instantaneous it is an
  M/M/1 sojourn; long runs cover the Jackson-network sum of 1/(mu_j-lambda).
"""
import heapq
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.stats as ostats


# ---------------------------------------------------------------- variates
def test_u53_grid_and_bounds():
    rng = np.random.default_rng(1)
    lo = rng.integers(0, 2**32, 100000, dtype=np.uint64).astype(np.uint32)
    hi = rng.integers(0, 2**32, 100000, dtype=np.uint64).astype(np.uint32)
    u, _ = oracle.u53_expo(lo, hi, 1.0)
    k = u * 2.0**53
    assert np.all(k == np.floor(k)) and np.all(u >= 0) and np.all(u < 1)
    # the integer is the top 53 bits of hi:lo
    expect = ((hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)) >> np.uint64(11)
    assert np.array_equal(k.astype(np.uint64), expect)
    u0, e0 = oracle.u53_expo([0], [0], 2.0)
    assert u0[0] == 0.0 and e0[0] == 0.0
    u1, e1 = oracle.u53_expo([0xFFFFFFFF], [0xFFFFFFFF], 1.0)
    assert u1[0] == 1.0 - 2.0**-53
    assert e1[0] == pytest.approx(53 * math.log(2.0), rel=1e-15)


def test_exponential_law():
    n = 200000
    blk = oracle.stream_block(42, 0, 0, 0, np.arange(n), 0)
    for rate in (0.5, 1.0, 3.0):
        _, e = oracle.u53_expo(blk[:, 0], blk[:, 1], rate)
        z = (e.mean() - 1.0 / rate) / (1.0 / rate / math.sqrt(n))
        assert abs(z) < 5.0
        assert stats.kstest(e, "expon", args=(0, 1.0 / rate)).pvalue > 1e-4
    # small u: -log(1-u) ~ u, so E ~ u/rate
    u, e = oracle.u53_expo([1 << 11], [0], 4.0)
    assert e[0] == pytest.approx(2.0**-53 / 4.0, rel=1e-15)


def test_threshold():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(0.5) == 1 << 31
    assert oracle.threshold(0.25) == 1 << 30
    assert oracle.threshold(1e-5) == math.floor(1e-5 * 2**32)
    # (1 - 2^-40) * 2^32 = 2^32 - 2^-8, whose floor is 2^32 - 1
    assert oracle.threshold(1.0 - 2.0**-40) == 2**32 - 1
    # a Bernoulli(p) built on the threshold has frequency p
    n = 1 << 18
    blk = oracle.stream_block(3, 0, 0, 0, np.arange(n // 4), 0).reshape(-1)
    for p in (0.01, 0.3):
        hits = int(np.count_nonzero(blk < oracle.threshold(p)))
        assert abs(hits - n * p) < 5 * math.sqrt(n * p * (1 - p))


# ---------------------------------------------------------------- helpers
def _mm1_variates(seed, dp, rep, n, lam, mu):
    blk = oracle.stream_block(seed, 0, dp, rep, np.arange(n), 0)
    _, s = oracle.u53_expo(blk[:, 0], blk[:, 1], mu)
    _, a = oracle.u53_expo(blk[:, 2], blk[:, 3], lam)
    return s, a  # a[n] is the gap after client n


def _event_driven_mm1(s, a_after):
    """Single-server FIFO queue driven by an event list on an absolute clock.
    Client 0 arrives at time 0; client n+1 arrives a_after[n] after client n."""
    n = len(s)
    events = [(0.0, 0, "arrive", 0)]
    seq = 1
    queue = []
    busy = False
    arrival_time = {}
    start_time = {}
    idle_after = {}
    last_departure = None
    last_departed = None
    while events:
        t, _, kind, c = heapq.heappop(events)
        if kind == "arrive":
            arrival_time[c] = t
            if c + 1 < n:
                heapq.heappush(events, (t + a_after[c], seq, "arrive", c + 1)); seq += 1
            if last_departure is not None and not busy and last_departed == c - 1:
                idle_after[c - 1] = t - last_departure
            if not busy:
                busy = True
                start_time[c] = t
                heapq.heappush(events, (t + s[c], seq, "depart", c)); seq += 1
            else:
                queue.append(c)
        else:
            last_departure, last_departed = t, c
            if queue:
                nxt = queue.pop(0)
                start_time[nxt] = t
                heapq.heappush(events, (t + s[nxt], seq, "depart", nxt)); seq += 1
            else:
                busy = False
    wait = np.array([start_time[c] - arrival_time[c] for c in range(n)])
    system = wait + np.asarray(s)
    # idle between departure of c and arrival of c+1 (the last client's idle
    # uses the gap to a client n that is not simulated)
    idle = np.zeros(n)
    for c in range(n - 1):
        idle[c] = idle_after.get(c, 0.0)
    dep_last = start_time[n - 1] + s[n - 1]
    idle[n - 1] = max(0.0, (arrival_time[n - 1] + a_after[n - 1]) - dep_last)
    return wait, idle, system


# ---------------------------------------------------------------- M/M/1
@pytest.mark.parametrize("lam,mu,rep", [(0.9, 1.0, 0), (0.9, 1.0, 5), (0.5, 1.0, 3),
                                        (1.3, 1.0, 1)])
def test_mm1_equals_event_driven(lam, mu, rep):
    n = 40
    s, a = _mm1_variates(42, 0, rep, n, lam, mu)
    wait, idle, system = _event_driven_mm1(s, a)
    w, i, y = oracle.mm1([[lam, mu]], [0], [rep], n, 42)
    assert w[0] == pytest.approx(wait.mean(), rel=1e-12, abs=1e-14)
    assert i[0] == pytest.approx(idle.mean(), rel=1e-12, abs=1e-14)
    assert y[0] == pytest.approx(system.mean(), rel=1e-12, abs=1e-14)


def test_mm1_light_traffic_and_single_client():
    # one client: it never waits; time in system is its service time
    s, a = _mm1_variates(42, 0, 0, 1, 0.9, 1.0)
    w, i, y = oracle.mm1([[0.9, 1.0]], [0], [0], 1, 42)
    assert w[0] == 0.0 and y[0] == s[0] and i[0] == max(0.0, a[0] - s[0])
    # arrivals far apart: nobody waits
    w, i, y = oracle.mm1([[1e-9, 1.0]], [0, 0], [0, 1], 1000, 42)
    assert np.all(w == 0.0)


def _ci_covers(values, truth, conf=0.99):
    c = ostats.ci(values, conf)
    return abs(c["mean"] - truth) <= c["half_width"], c


def test_mm1_steady_state_light_load():
    lam, mu = 0.5, 1.0
    reps = 16
    w, i, y = oracle.mm1([[lam, mu]], np.zeros(reps, np.int32), np.arange(reps), 10**6, 7,
                         threads=oracle.host_threads())
    rho = lam / mu
    ok, c = _ci_covers(w, rho / (mu - lam)); assert ok, c
    ok, c = _ci_covers(i, (1 - rho) / lam); assert ok, c
    ok, c = _ci_covers(y, 1.0 / (mu - lam)); assert ok, c


def test_mm1_steady_state_heavy_load():
    lam, mu = 0.9, 1.0
    reps = 8
    w, _, y = oracle.mm1([[lam, mu]], np.zeros(reps, np.int32), np.arange(reps), 2 * 10**6, 11,
                         threads=oracle.host_threads())
    ok, c = _ci_covers(w, 0.9 / 0.1); assert ok, c
    ok, c = _ci_covers(y, 1.0 / 0.1); assert ok, c


# ---------------------------------------------------------------- tandem
def _tandem_variates(seed, tag, dp, rep, n, par):
    b0 = oracle.stream_block(seed, tag, dp, rep, np.arange(n), 0)
    b1 = oracle.stream_block(seed, tag, dp, rep, np.arange(n), 1)
    _, a = oracle.u53_expo(b0[:, 0], b0[:, 1], par[0])
    _, s1 = oracle.u53_expo(b0[:, 2], b0[:, 3], par[1])
    _, s2 = oracle.u53_expo(b1[:, 0], b1[:, 1], par[2])
    _, s3 = oracle.u53_expo(b1[:, 2], b1[:, 3], par[3])
    return a, (s1, s2, s3)


def _event_driven_tandem(a, s):
    """Absolute-clock event simulation of three FIFO stations in series."""
    n = len(a)
    arrive = np.cumsum(a)  # client n arrives at A_0 + ... + A_n
    events = []
    seq = 0
    for c in range(n):
        heapq.heappush(events, (arrive[c], seq, 0, c)); seq += 1
    queues = [[], [], []]
    busy = [False, False, False]
    leave = np.zeros(n)
    while events:
        t, _, station, c = heapq.heappop(events)
        if station < 3:  # client c reaches `station`
            if busy[station]:
                queues[station].append(c)
            else:
                busy[station] = True
                heapq.heappush(events, (t + s[station][c], seq, 10 + station, c)); seq += 1
        else:  # departure from station (code - 10)
            st = station - 10
            if st == 2:
                leave[c] = t
            else:
                heapq.heappush(events, (t, seq, st + 1, c)); seq += 1
            if queues[st]:
                nxt = queues[st].pop(0)
                heapq.heappush(events, (t + s[st][nxt], seq, 10 + st, nxt)); seq += 1
            else:
                busy[st] = False
    return leave - arrive


@pytest.mark.parametrize("par,rep", [((0.7, 1.0, 1.2, 1.4), 0), ((0.95, 1.0, 1.0, 1.0), 3),
                                     ((1.2, 1.0, 2.0, 0.8), 2)])
def test_tandem_equals_event_driven(par, rep):
    n = 40
    a, s = _tandem_variates(42, 0, 0, rep, n, par)
    soj = _event_driven_tandem(a, s)
    y, feat = oracle.tandem3([par], [0], [rep], n, 42, window=10)
    assert y[0] == pytest.approx(soj.mean(), rel=1e-12)
    assert np.array_equal(feat[0, :4], np.array(par))
    assert feat[0, 4] == pytest.approx(a[:10].mean(), rel=1e-15)
    for j in range(3):
        assert feat[0, 5 + j] == pytest.approx(s[j][:10].mean(), rel=1e-15)


def test_tandem_window_longer_than_run_and_tag():
    y, feat = oracle.tandem3([[0.5, 1, 1, 1]], [0], [0], 5, 42, window=100)
    a, s = _tandem_variates(42, 0, 0, 0, 5, (0.5, 1, 1, 1))
    assert feat[0, 4] == pytest.approx(a.mean(), rel=1e-15)
    # tag 2 draws from another stream
    y2, _ = oracle.tandem3([[0.5, 1, 1, 1]], [0], [0], 5, 42, window=100, tag=2)
    assert y2[0] != y[0]


def test_tandem_reduces_to_mm1_when_later_stations_instant():
    par = (0.8, 1.0, 1e12, 1e12)
    n = 200
    a, s = _tandem_variates(42, 0, 0, 4, n, par)
    # single station sojourn by Lindley on an absolute clock
    arrive = np.cumsum(a)
    dep = np.zeros(n)
    for c in range(n):
        start = arrive[c] if c == 0 else max(arrive[c], dep[c - 1])
        dep[c] = start + s[0][c]
    y, _ = oracle.tandem3([par], [0], [4], n, 42)
    assert y[0] == pytest.approx((dep - arrive).mean(), rel=1e-9)


def test_tandem_jackson_steady_state():
    par = (0.5, 1.0, 1.2, 1.5)
    reps = 8
    y, _ = oracle.tandem3([par], np.zeros(reps, np.int32), np.arange(reps), 10**6, 5,
                          threads=oracle.host_threads())
    truth = sum(1.0 / (m - par[0]) for m in par[1:])
    ok, c = _ci_covers(y, truth)
    assert ok, (c, truth)
