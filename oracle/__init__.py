"""CPU oracle for the MRIP hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA path (the package
``paper_1501_01405_gb300``) and never imports it.

The replication recurrences (Philox4x32-10 streams, M/M/1, tandem, forest
fire, L1-exit walk) and the Student-t critical value are plain C in
``mrip_oracle.c``; the statistics, the network and the control-variate
estimator are numpy in ``stats.py``, ``mlp.py`` and ``cv.py``.  All are FP64
except where the method itself rounds to BF16 (the network's weights and
matmul operands).

The batch helpers below split a list of (design point, replication) items
into contiguous chunks and run them on Python threads; ctypes releases the GIL
during each foreign call, so the chunks run on separate host cores.
"""
import ctypes
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_c = ctypes


def lib():
    """Load (building if needed) the oracle's shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    L.or_philox_batch.argtypes = [_c.c_int64, _u32p, _u32p, _u32p]
    L.or_philox_batch.restype = None
    L.or_expo_batch.argtypes = [_c.c_int64, _u32p, _u32p, _f64p, _f64p, _f64p]
    L.or_expo_batch.restype = None
    L.or_threshold.argtypes = [_c.c_double]
    L.or_threshold.restype = _c.c_uint32
    L.or_mm1_batch.argtypes = [_f64p, _c.c_int64, _i32p, _i64p, _c.c_int64, _c.c_uint64,
                               _f64p, _f64p, _f64p]
    L.or_mm1_batch.restype = None
    L.or_tandem3_batch.argtypes = [_f64p, _c.c_int64, _i32p, _i64p, _c.c_int64, _c.c_int64,
                                   _c.c_uint64, _c.c_uint32, _f64p, _f64p]
    L.or_tandem3_batch.restype = None
    L.or_forest_fire_rep.argtypes = [_c.c_int32, _c.c_int32, _c.c_double, _c.c_double,
                                     _c.c_double, _c.c_uint64, _c.c_uint32, _c.c_uint32,
                                     _c.c_void_p, _i32p, _c.c_void_p]
    L.or_forest_fire_rep.restype = _c.c_int
    L.or_forest_fire_batch.argtypes = [_c.c_int32, _c.c_int32, _f64p, _c.c_double,
                                       _c.c_int64, _i32p, _i64p, _c.c_uint64, _i32p]
    L.or_forest_fire_batch.restype = _c.c_int
    L.or_forest_fire_skip_rep.argtypes = [_c.c_int32, _c.c_int32, _c.c_double, _c.c_double,
                                          _c.c_double, _c.c_uint64, _c.c_uint32, _c.c_uint32,
                                          _c.c_void_p, _i32p, _c.c_void_p, _i64p]
    L.or_forest_fire_skip_rep.restype = _c.c_int
    L.or_forest_fire_skip_batch.argtypes = [_c.c_int32, _c.c_int32, _f64p, _c.c_double,
                                            _c.c_int64, _i32p, _i64p, _c.c_uint64, _i32p, _i64p]
    L.or_forest_fire_skip_batch.restype = _c.c_int
    L.or_walk_batch.argtypes = [_f64p, _c.c_int64, _i32p, _i64p, _c.c_uint64, _c.c_int64,
                                _i64p]
    L.or_walk_batch.restype = None
    L.or_area_walk_batch.argtypes = [_c.c_int64, _i64p, _c.c_int32, _c.c_uint64, _i32p, _i32p]
    L.or_area_walk_batch.restype = None
    L.or_pi_batch.argtypes = [_c.c_int64, _i64p, _c.c_int64, _c.c_uint64, _i64p]
    L.or_pi_batch.restype = None
    L.or_t_cdf.argtypes = [_c.c_double, _c.c_int64]
    L.or_t_cdf.restype = _c.c_double
    L.or_t_crit.argtypes = [_c.c_double, _c.c_int64]
    L.or_t_crit.restype = _c.c_double
    L.or_t_quantile.argtypes = [_c.c_double, _c.c_int64]
    L.or_t_quantile.restype = _c.c_double
    _lib = L
    return L


# ---------------------------------------------------------------------------
# Random streams (Philox4x32-10 keyed on seed, design point, replication, step)
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 of counters ``ctr`` (n, 4) under keys ``key`` (n, 2)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    if key.shape[0] == 1 and ctr.shape[0] > 1:
        key = np.ascontiguousarray(np.repeat(key, ctr.shape[0], axis=0))
    out = np.empty_like(ctr)
    lib().or_philox_batch(ctr.shape[0], ctr.reshape(-1), key.reshape(-1), out.reshape(-1))
    return out


def stream_block(seed, tag, dp, rep, step, sub):
    """The four words of block (c0 = sub, c1 = step) of (tag, dp, rep)."""
    step = np.atleast_1d(np.asarray(step, dtype=np.uint64))
    sub = np.broadcast_to(np.asarray(sub, dtype=np.uint64), step.shape)
    ctr = np.stack([sub.astype(np.uint32), step.astype(np.uint32),
                    np.full(step.shape, rep, dtype=np.uint32),
                    np.full(step.shape, (tag << 24) | dp, dtype=np.uint32)], axis=1)
    key = np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint32)
    return philox4x32_10(ctr, key)


def u53_expo(lo, hi, rate):
    """(u, -log(1-u)/rate) for u = top 53 bits of hi:lo times 2^-53."""
    lo = np.ascontiguousarray(np.asarray(lo, dtype=np.uint32).reshape(-1))
    hi = np.ascontiguousarray(np.asarray(hi, dtype=np.uint32).reshape(-1))
    rate = np.ascontiguousarray(np.broadcast_to(np.asarray(rate, dtype=np.float64), lo.shape))
    u = np.empty(lo.shape, np.float64)
    e = np.empty(lo.shape, np.float64)
    lib().or_expo_batch(lo.size, lo, hi, rate, u, e)
    return u, e


def threshold(p):
    """T(p) = floor(p * 2^32) for p in [0, 1)."""
    return int(lib().or_threshold(float(p)))


# ---------------------------------------------------------------------------
# Threaded batch driver
# ---------------------------------------------------------------------------
def _chunks(n, threads):
    threads = max(1, min(int(threads), n if n > 0 else 1))
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    return [(int(bounds[i]), int(bounds[i + 1])) for i in range(threads)
            if bounds[i + 1] > bounds[i]]


def _run_chunks(fn, n, threads):
    parts = _chunks(n, threads)
    if len(parts) <= 1:
        for lo, hi in parts:
            fn(lo, hi)
        return
    with ThreadPoolExecutor(max_workers=len(parts)) as ex:
        list(ex.map(lambda p: fn(*p), parts))


def _items(dp_idx, rep_idx):
    dp_idx = np.ascontiguousarray(np.asarray(dp_idx, dtype=np.int32).reshape(-1))
    rep_idx = np.ascontiguousarray(np.asarray(rep_idx, dtype=np.int64).reshape(-1))
    if dp_idx.shape != rep_idx.shape:
        raise ValueError("dp_idx and rep_idx must have the same length")
    return dp_idx, rep_idx


def all_items(n_dp, n_reps):
    """Every (dp, rep) pair, design-point-major."""
    dp = np.repeat(np.arange(n_dp, dtype=np.int32), n_reps)
    rep = np.tile(np.arange(n_reps, dtype=np.int64), n_dp)
    return dp, rep


# ---------------------------------------------------------------------------
# Models
# ---------------------------------------------------------------------------
def mm1(dps, dp_idx, rep_idx, n_clients, seed, threads=1):
    """M/M/1 per replication: (mean wait, mean idle, mean time in system)."""
    dps = np.ascontiguousarray(np.asarray(dps, dtype=np.float64).reshape(-1, 2))
    dp_idx, rep_idx = _items(dp_idx, rep_idx)
    n = dp_idx.size
    wait, idle, system = (np.empty(n, np.float64) for _ in range(3))

    def run(lo, hi):
        lib().or_mm1_batch(dps.reshape(-1), hi - lo, dp_idx[lo:hi], rep_idx[lo:hi],
                           int(n_clients), int(seed), wait[lo:hi], idle[lo:hi],
                           system[lo:hi])
    _run_chunks(run, n, threads)
    return wait, idle, system


def tandem3(dps, dp_idx, rep_idx, n_clients, seed, window=100, tag=0, threads=1):
    """Tandem-3 per replication: (mean sojourn Y, features (n, 8))."""
    dps = np.ascontiguousarray(np.asarray(dps, dtype=np.float64).reshape(-1, 4))
    dp_idx, rep_idx = _items(dp_idx, rep_idx)
    n = dp_idx.size
    y = np.empty(n, np.float64)
    feat = np.empty((n, 8), np.float64)

    def run(lo, hi):
        lib().or_tandem3_batch(dps.reshape(-1), hi - lo, dp_idx[lo:hi], rep_idx[lo:hi],
                               int(n_clients), int(window), int(seed), int(tag), y[lo:hi],
                               feat[lo:hi].reshape(-1))
    _run_chunks(run, n, threads)
    return y, feat


def forest_fire_rep(L, n_steps, p_grow, p_light, density, seed, dp, rep, init_state=None):
    """One forest-fire replication: (burning counts (T,), final state (L, L))."""
    counts = np.empty(n_steps, np.int32)
    final = np.empty((L, L), np.uint8)
    init_ptr = None
    if init_state is not None:
        init_state = np.ascontiguousarray(np.asarray(init_state, dtype=np.uint8).reshape(L, L))
        init_ptr = init_state.ctypes.data
    rc = lib().or_forest_fire_rep(int(L), int(n_steps), float(p_grow), float(p_light),
                                  float(density), int(seed), int(dp), int(rep), init_ptr,
                                  counts, final.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle forest fire: allocation failed")
    return counts, final


def forest_fire(L, n_steps, dps, density, dp_idx, rep_idx, seed, threads=1):
    """Forest fire per replication: burning counts (n, T)."""
    dps = np.ascontiguousarray(np.asarray(dps, dtype=np.float64).reshape(-1, 2))
    dp_idx, rep_idx = _items(dp_idx, rep_idx)
    n = dp_idx.size
    counts = np.empty((n, n_steps), np.int32)

    def run(lo, hi):
        rc = lib().or_forest_fire_batch(int(L), int(n_steps), dps.reshape(-1), float(density),
                                        hi - lo, dp_idx[lo:hi], rep_idx[lo:hi], int(seed),
                                        counts[lo:hi].reshape(-1))
        if rc != 0:
            raise MemoryError("oracle forest fire: allocation failed")
    _run_chunks(run, n, threads)
    return counts


def forest_fire_skip_rep(L, n_steps, p_grow, p_light, density, seed, dp, rep, init_state=None):
    """One skip-sampled forest-fire replication: (counts (T,), final (L, L),
    near_ties)."""
    counts = np.empty(n_steps, np.int32)
    final = np.empty((L, L), np.uint8)
    ties = np.zeros(1, np.int64)
    init_ptr = None
    if init_state is not None:
        init_state = np.ascontiguousarray(np.asarray(init_state, dtype=np.uint8).reshape(L, L))
        init_ptr = init_state.ctypes.data
    rc = lib().or_forest_fire_skip_rep(int(L), int(n_steps), float(p_grow), float(p_light),
                                       float(density), int(seed), int(dp), int(rep), init_ptr,
                                       counts, final.ctypes.data, ties)
    if rc != 0:
        raise MemoryError("oracle forest fire: allocation failed")
    return counts, final, int(ties[0])


def forest_fire_skip(L, n_steps, dps, density, dp_idx, rep_idx, seed, threads=1):
    """Skip-sampled forest fire per replication: (counts (n, T), near_ties (n,))."""
    dps = np.ascontiguousarray(np.asarray(dps, dtype=np.float64).reshape(-1, 2))
    dp_idx, rep_idx = _items(dp_idx, rep_idx)
    n = dp_idx.size
    counts = np.empty((n, n_steps), np.int32)
    ties = np.zeros(n, np.int64)

    def run(lo, hi):
        rc = lib().or_forest_fire_skip_batch(int(L), int(n_steps), dps.reshape(-1), float(density),
                                             hi - lo, dp_idx[lo:hi], rep_idx[lo:hi], int(seed),
                                             counts[lo:hi].reshape(-1), ties[lo:hi])
        if rc != 0:
            raise MemoryError("oracle forest fire: allocation failed")
    _run_chunks(run, n, threads)
    return counts, ties


def walk(radii, dp_idx, rep_idx, seed, max_steps=1 << 38, threads=1):
    """L1-exit walk per replication: exit time tau (int64; -1 if capped)."""
    radii = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
    dp_idx, rep_idx = _items(dp_idx, rep_idx)
    n = dp_idx.size
    tau = np.empty(n, np.int64)

    def run(lo, hi):
        lib().or_walk_batch(radii, hi - lo, dp_idx[lo:hi], rep_idx[lo:hi], int(seed),
                            int(max_steps), tau[lo:hi])
    _run_chunks(run, n, threads)
    return tau


def area_walk(rep_idx, n_steps, seed, threads=1):
    """Area walk per replication: (final area (n,), visits (n, 30))."""
    rep_idx = np.ascontiguousarray(np.asarray(rep_idx, dtype=np.int64).reshape(-1))
    n = rep_idx.size
    final = np.empty(n, np.int32)
    visits = np.empty((n, 30), np.int32)

    def run(lo, hi):
        lib().or_area_walk_batch(hi - lo, rep_idx[lo:hi], int(n_steps), int(seed), final[lo:hi],
                                 visits[lo:hi].reshape(-1))
    _run_chunks(run, n, threads)
    return final, visits


def pi_hits(rep_idx, n_draws, seed, threads=1):
    """Monte Carlo pi per replication: number of the n_draws points inside."""
    rep_idx = np.ascontiguousarray(np.asarray(rep_idx, dtype=np.int64).reshape(-1))
    hits = np.empty(rep_idx.size, np.int64)

    def run(lo, hi):
        lib().or_pi_batch(hi - lo, rep_idx[lo:hi], int(n_draws), int(seed), hits[lo:hi])
    _run_chunks(run, rep_idx.size, threads)
    return hits


# ---------------------------------------------------------------------------
# Student-t
# ---------------------------------------------------------------------------
def t_cdf(t, nu):
    return float(lib().or_t_cdf(float(t), int(nu)))


def t_crit(conf, nu):
    """t > 0 with P(T > t) = (1 - conf)/2, nu degrees of freedom."""
    return float(lib().or_t_crit(float(conf), int(nu)))


def t_quantile(p, nu):
    return float(lib().or_t_quantile(float(p), int(nu)))


def host_threads():
    """Host cores available to this process."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1
