"""Sharding one experiment (GPU): replications split into ranges give exactly
the per-replication outputs of one run, and their statistics merge to the
one-run statistics.

Every replication is a pure function of (seed, design point, replication
index), so for every model and mapping the outputs of the ranges [0, lo) and
[lo, n) -- and of three ragged ranges -- laid side by side per design point
must equal the outputs of one call over [0, n) bit for bit (FP64 included:
the same replication runs the same instructions whichever range it is in).
Through the model handle, mrip_run_range's (n, mean, M2) triples merged
with mrip_stats_merge must equal the one-run triples within 1e-13, and two
gloo ranks on this GPU, each running its shard through the engine, must
agree on the merged interval.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import mrip_inputs

pytestmark = pytest.mark.gpu

SPLITS = ([13], [5, 23])  # cut points inside [0, n)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1501_01405_gb300 as eng
    eng.lib()
    return eng, torch


def _ranges(n, cuts):
    edges = [0] + list(cuts) + [n]
    return list(zip(edges[:-1], edges[1:]))


def _check_sharded(n, n_dp, run, cuts_list=SPLITS):
    """run(rep0, n_reps) -> array shaped (n_dp, n_reps, ...) of outputs."""
    full = run(0, n)
    assert full.shape[:2] == (n_dp, n)
    for cuts in cuts_list:
        parts = [run(lo, hi - lo) for lo, hi in _ranges(n, cuts)]
        got = np.concatenate(parts, axis=1)
        assert np.array_equal(got, full), cuts


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP", "CTA"])
def test_mm1_shards(env, mapping):
    eng, torch = env
    dps = torch.tensor([[0.9, 1.0], [0.5, 1.0], [0.02, 9.0]], dtype=torch.float64, device="cuda")
    m = getattr(eng, "MRIP_MAP_" + mapping)

    def run(rep0, k):
        w = torch.empty(3 * k, dtype=torch.float64, device="cuda")
        i = torch.empty_like(w)
        s = torch.empty_like(w)
        eng.mrip_mm1_simulate(dps, k, 201, 42, m, w, i, s, rep0=rep0)
        return torch.stack([w, i, s], 1).view(3, k, 3).cpu().numpy()
    _check_sharded(37, 3, run)


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_COOP", "CTA"])
def test_tandem_shards(env, mapping):
    eng, torch = env
    dps = torch.tensor(mrip_inputs.tandem_design_points(3, seed=4), device="cuda")
    m = getattr(eng, "MRIP_MAP_" + mapping)

    def run(rep0, k):
        y = torch.empty(3 * k, dtype=torch.float64, device="cuda")
        f = torch.empty(8 * 3 * k, dtype=torch.float64, device="cuda")
        eng.mrip_tandem3_simulate(dps, rep0, k, 150, 40, 42, 0, m, y, f)
        return torch.cat([y.view(1, -1), f.view(8, -1)]).T.reshape(3, k, 9).cpu().numpy()
    _check_sharded(37, 3, run)


@pytest.mark.parametrize("skip", [False, True])
def test_forest_fire_shards(env, skip):
    eng, torch = env
    dps = torch.tensor([[0.05, 0.001], [0.01, 1e-5]], dtype=torch.float64, device="cuda")
    fn = eng.mrip_forest_fire_skip_simulate if skip else eng.mrip_forest_fire_simulate
    L, T = 64, 50

    def run(rep0, k):
        c = torch.empty(2 * k * T, dtype=torch.int32, device="cuda")
        sc = torch.empty(2 * k, dtype=torch.float64, device="cuda")
        fin = torch.empty(2 * k * L * L, dtype=torch.uint8, device="cuda")
        fn(dps, k, L, T, 0.5, 42, counts=c, scalar=sc, final=fin, rep0=rep0)
        out = np.concatenate([c.view(2, k, T).cpu().numpy().astype(np.float64),
                              sc.view(2, k, 1).cpu().numpy(),
                              fin.view(2, k, L * L).cpu().numpy().astype(np.float64)], axis=2)
        return out
    _check_sharded(7, 2, run, ([3], [1, 4]))


@pytest.mark.parametrize("mapping", ["PERSISTENT", "THREAD", "WARP_COOP"])
@pytest.mark.parametrize("noalloc", [False, True])
def test_walk_shards(env, mapping, noalloc):
    eng, torch = env
    radii = [5.0, 12.0, 9.0]
    m = getattr(eng, "MRIP_MAP_" + mapping)
    fn = eng.mrip_walk_simulate_noalloc if noalloc else eng.mrip_walk_simulate

    def run(rep0, k):
        tau = torch.empty(3 * k, dtype=torch.int64, device="cuda")
        fn(radii, k, 42, 1 << 30, m, tau, chunk=7, rep0=rep0)
        torch.cuda.synchronize()
        return tau.view(3, k).cpu().numpy()
    _check_sharded(301, 3, run, ([150], [17, 200]))


def test_pi_shards(env):
    eng, torch = env

    def run(rep0, k):
        h = torch.empty(k, dtype=torch.int64, device="cuda")
        eng.mrip_pi_simulate(k, 100_003, 42, h, rep0=rep0)
        return h.view(1, k).cpu().numpy()
    _check_sharded(9, 1, run, ([4], [1, 6]))


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP"])
def test_area_walk_shards(env, mapping):
    eng, torch = env
    m = getattr(eng, "MRIP_MAP_" + mapping)

    def run(rep0, k):
        fa = torch.empty(k, dtype=torch.int32, device="cuda")
        vis = torch.empty(30 * k, dtype=torch.int32, device="cuda")
        eng.mrip_area_walk_simulate(k, 700, 42, m, fa, vis, rep0=rep0)
        return torch.cat([fa.view(1, k), vis.view(30, k)]).T.reshape(1, k, 31).cpu().numpy()
    _check_sharded(100, 1, run, ([33], [10, 64]))


def _handle_cases(eng):
    return [
        (eng.MRIP_MM1, dict(n_clients=300), [[0.9, 1.0], [0.5, 1.0]], 0, np.float64),
        (eng.MRIP_TANDEM3, dict(n_clients=120, window=30), mrip_inputs.tandem_design_points(2, seed=8),
         0, np.float64),
        (eng.MRIP_FOREST_FIRE, dict(L=32, n_steps=40, density=0.5, window=8),
         [[0.05, 0.001], [0.02, 0.0]], 1, np.float64),
        (eng.MRIP_WALK_L1_EXIT, dict(max_steps=1 << 30), [7.0, 3.0, 16.0], 0, np.int64),
    ]


def test_handle_run_range_merges_to_one_run(env):
    eng, torch = env
    n, seed = 41, 42
    for kind, params, dps, plane, dtype in _handle_cases(eng):
        n_dp = len(dps)
        m = eng.Model(kind, **params)
        m.run(dps, n, seed)
        full_out = m.outputs(plane, dtype=dtype).reshape(n_dp, n)
        full = m.moments()
        one = m.stats()
        for cuts in ([20], [1, 30], [10, 11, 40]):
            parts, outs = [], []
            for lo, hi in _ranges(n, cuts):
                m.run_range(dps, lo, hi, seed)
                parts.append(m.moments())
                outs.append(m.outputs(plane, dtype=dtype).reshape(n_dp, hi - lo))
            assert np.array_equal(np.concatenate(outs, axis=1), full_out), (kind, cuts)
            merged = eng.mrip_stats_merge(np.stack(parts))
            assert np.array_equal(merged[:, 0], full[:, 0])
            np.testing.assert_allclose(merged[:, 1], full[:, 1], rtol=1e-13, atol=0)
            np.testing.assert_allclose(merged[:, 2], full[:, 2], rtol=1e-13, atol=0)
            for g, r in zip(eng.mrip_stats_finalize(merged), one):
                assert g["half_width"] == pytest.approx(r["half_width"], rel=1e-13)
        m.close()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, seed, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1501_01405_gb300 as eng
        from paper_1501_01405_gb300.distributed import sharded_stats
        torch.cuda.set_device(0)
        m = eng.Model(eng.MRIP_MM1, n_clients=500)
        stats, merged = sharded_stats(m, [[0.9, 1.0], [0.7, 1.0]], n, seed)
        q.put((rank, merged, [s["half_width"] for s in stats]))
        m.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_one_experiment(env):
    """Two processes on this GPU, each running its replication range through
    the engine; they exchange triples over gloo (host) -- no kernel of one
    waits for the other."""
    eng, torch = env
    n, seed = 75, 42
    m = eng.Model(eng.MRIP_MM1, n_clients=500)
    m.run([[0.9, 1.0], [0.7, 1.0]], n, seed)
    ref = m.moments()
    ref_hw = [s["half_width"] for s in m.stats()]
    m.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, seed, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, merged, hw in got:
        np.testing.assert_allclose(merged, ref, rtol=1e-13, atol=0)
        np.testing.assert_allclose(hw, ref_hw, rtol=1e-13)


def test_checkpoint_resume_matches_one_run(env, tmp_path):
    """An experiment interrupted after two ranges, saved, loaded and resumed
    in ranges of another size gives the one-run (n, mean, M2) within 1e-13
    (the merge order is the replication order either way)."""
    eng, torch = env
    from paper_1501_01405_gb300.checkpoint import Checkpoint, run_resumable
    path = str(tmp_path / "exp.json")
    for kind, params, dps in ((eng.MRIP_MM1, {"n_clients": 400}, [[0.9, 1.0], [0.6, 1.0]]),
                              (eng.MRIP_WALK_L1_EXIT, {"max_steps": 1 << 30}, [12.0, 5.0])):
        n, seed = 301, 42
        m = eng.Model(kind, **params)
        m.run(dps, n, seed)
        ref = m.moments()
        m.close()
        ck = Checkpoint(kind, params, dps, n, seed)
        part = run_resumable(ck, 64, path=path, max_chunks=2)
        assert np.all(part[:, 0] == 128) and not ck.complete()
        again = Checkpoint.load(path)
        assert again.missing() == [(128, n)]
        full = run_resumable(again, 50, path=path)
        assert again.complete() and Checkpoint.load(path).complete()
        assert np.array_equal(full[:, 0], ref[:, 0])
        np.testing.assert_allclose(full[:, 1:], ref[:, 1:], rtol=1e-13, atol=0)


def test_allocation_failure_is_reported_and_the_handle_recovers(env):
    """A run too large for any device (2^20 design points x 2^20 replications:
    24 TB of outputs) returns MRIP_ENOMEM from a failed allocation -- a
    normal error return, not a fault -- and the same handle then runs a
    small experiment."""
    eng, torch = env
    m = eng.Model(eng.MRIP_MM1, n_clients=10)
    big = np.tile([[0.5, 1.0]], (1 << 20, 1))
    with pytest.raises(eng.MripError) as e:
        m.run(big, 1 << 20, 42)
    assert e.value.code == 2
    m.run([[0.5, 1.0]], 8, 42)
    assert m.stats()[0]["n"] == 8
    m.close()
