"""Multi-rank logic on the CPU (gloo, world size 2).

Replications are pure functions of (seed, design point, replication), so a
partition of the replications across ranks changes nothing but the order in
which per-design-point (n, mean, M2) triples are merged.  These tests check
the shard ranges, the engine's host merge against the oracle's two-pass
statistics, a real two-process gloo exchange, and failure handling done on
the host: a rank that dies before publishing is detected through the store
and its shard is recomputed by the survivor, with the same result.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
import oracle.stats as ostats

pytest.importorskip("torch")


def _engine():
    import paper_1501_01405_gb300 as eng
    try:
        eng.lib()
    except eng.MripLibraryMissing:
        from paper_1501_01405_gb300 import build
        build.build()
    return eng


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _triples(x):
    x = np.asarray(x, dtype=np.float64).reshape(x.shape[0], -1)
    out = []
    for row in x:
        n = row.size
        if n == 0:
            out.append([0.0, 0.0, 0.0])
            continue
        m = row.mean()
        out.append([n, m, float(((row - m) ** 2).sum())])
    return np.array(out)


DPS = np.array([[0.9, 1.0], [0.6, 1.0], [0.3, 0.5]])
N_REPS, N_CLIENTS, SEED = 50, 300, 11


def _shard_outputs(lo, hi):
    dp = np.repeat(np.arange(3, dtype=np.int32), hi - lo)
    rep = np.tile(np.arange(lo, hi), 3)
    w, _, _ = oracle.mm1(DPS, dp, rep, N_CLIENTS, SEED)
    return w.reshape(3, hi - lo)


def test_shard_range_covers_once():
    from paper_1501_01405_gb300.distributed import shard_range
    for n in (0, 1, 7, 50, 1 << 17):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [h - l for l, h in got]
            assert max(sizes) - min(sizes) <= 1


def test_merge_of_shards_equals_two_pass():
    eng = _engine()
    from paper_1501_01405_gb300.distributed import shard_range
    full = _shard_outputs(0, N_REPS)
    for world in (1, 2, 3, 5):
        parts = np.stack([_triples(_shard_outputs(*shard_range(N_REPS, r, world)))
                          for r in range(world)])
        merged = eng.mrip_stats_merge(parts)
        for d in range(3):
            n, mean, var = ostats.dp_stats(full[d])
            assert merged[d, 0] == n
            assert merged[d, 1] == pytest.approx(mean, rel=1e-14)
            assert merged[d, 2] / (n - 1) == pytest.approx(var, rel=1e-13)
    # an empty part changes nothing
    t = _triples(full)
    merged = eng.mrip_stats_merge(np.stack([np.zeros_like(t), t]))
    assert np.array_equal(merged, t)


def _rank_main(rank, world, port, mode, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        import datetime
        import torch.distributed as dist
        from paper_1501_01405_gb300 import distributed as D
        from paper_1501_01405_gb300 import mrip_stats_finalize
        lo, hi = D.shard_range(N_REPS, rank, world)
        if mode == "gloo":
            dist.init_process_group("gloo", rank=rank, world_size=world,
                                    timeout=datetime.timedelta(seconds=30))
            merged = D.gather_merge_stats(_triples(_shard_outputs(lo, hi)))
            tmax = D.max_over_ranks(float(rank) + 0.5)
            ci = mrip_stats_finalize(merged, 0.95)
            dist.destroy_process_group()
            q.put((rank, merged.tolist(), tmax, [c["half_width"] for c in ci]))
        else:  # one rank dies before publishing its shard
            import torch.distributed as dist
            store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                                  timeout=datetime.timedelta(seconds=30))
            if rank == 1:
                os._exit(0)  # dies without publishing or reporting
            merged, failed = D.collect_with_recovery(
                store, rank, world, _triples(_shard_outputs(lo, hi)),
                lambda r: _triples(_shard_outputs(*D.shard_range(N_REPS, r, world))),
                timeout_s=3.0)
            q.put((rank, merged.tolist(), failed, None))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, "error", repr(e), None))


def _run_ranks(mode, world=2, reporting=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world if reporting is None else reporting):
        r = q.get(timeout=90)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return res


def _expected():
    full = _shard_outputs(0, N_REPS)
    return full, [ostats.ci(full[d]) for d in range(3)]


def test_two_rank_gloo_exchange_matches_single_run():
    _engine()
    res = _run_ranks("gloo")
    full, ci = _expected()
    for r in (0, 1):
        assert res[r][1] != "error", res[r]
        merged = np.array(res[r][1])
        assert res[r][2] == 1.5  # max over ranks of rank + 0.5
        for d in range(3):
            assert merged[d, 1] == pytest.approx(ci[d]["mean"], rel=1e-14)
            assert res[r][3][d] == pytest.approx(ci[d]["half_width"], rel=1e-12)


def test_dead_rank_detected_and_shard_recomputed():
    _engine()
    res = _run_ranks("failure", reporting=1)
    assert res[0][1] != "error", res[0]
    merged = np.array(res[0][1])
    assert res[0][2] == [1]
    full, ci = _expected()
    for d in range(3):
        assert merged[d, 0] == N_REPS
        assert merged[d, 1] == pytest.approx(ci[d]["mean"], rel=1e-14)
