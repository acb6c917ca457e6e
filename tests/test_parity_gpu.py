"""GPU parity: every stage of the CUDA path against the oracle, through the C ABI.

Integer and lattice outputs must match bit for bit; FP64 outputs within
1e-12 relative (the engine's log may differ from the C library's by an ulp,
and a warp-cooperative replay sums in another order).  Sizes span several
tiles with ragged tails; the full-size workloads run on the GPU in the
launch configuration the bench uses and are checked on every replication
(M/M/1, forest fire 128^2 and its skip-sampled variant, walk batch, tandem)
or on sampled ones (the 256^2 forest fire and its skip-sampled variant).
"""
import math

import numpy as np
import pytest

import mrip_inputs
import oracle
import oracle.stats as ostats

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available(), "GPU parity tests need CUDA"
    import paper_1501_01405_gb300 as e
    e.lib()  # fails loudly if the engine was not built
    return e


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def dev(torch, a, dtype=None):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def threads():
    return oracle.host_threads()


# ------------------------------------------------------------------ streams
def test_philox_bit_exact(eng, torch_mod):
    t = torch_mod
    rng = np.random.default_rng(1)
    n = (1 << 16) + 17
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]]
    out = t.empty((n, 4), dtype=t.int32, device="cuda")
    eng.mrip_philox(dev(t, ctr.view(np.int32)), dev(t, key.view(np.int32)), out)
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.philox4x32_10(ctr, key))


def test_expo_variates(eng, torch_mod):
    t = torch_mod
    rng = np.random.default_rng(2)
    n = 100003
    lo = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    hi = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    lo[:2], hi[:2] = [0, 0xFFFFFFFF], [0, 0xFFFFFFFF]
    rate = rng.uniform(0.3, 3.0, n)
    u = t.empty(n, dtype=t.float64, device="cuda")
    e = t.empty(n, dtype=t.float64, device="cuda")
    eng.mrip_expo(dev(t, lo.view(np.int32)), dev(t, hi.view(np.int32)), dev(t, rate), u, e)
    u_ref, e_ref = oracle.u53_expo(lo, hi, rate)
    assert np.array_equal(u.cpu().numpy(), u_ref)
    # The engine evaluates -log(1 - u) in 64-bit fixed point (absolute error
    # below 2^-56) and multiplies by a rounded 1/rate; the oracle calls the C
    # library's log and divides.  Bound: a few ulps plus 2^-55 / rate.
    got = e.cpu().numpy()
    bound = 4 * np.spacing(np.abs(e_ref)) + 2.0**-55 / rate
    assert np.all(np.abs(got - e_ref) <= bound)
    big = e_ref * rate > 1 / 16
    assert np.max(np.abs(got - e_ref)[big] / np.spacing(e_ref[big])) <= 3


# ------------------------------------------------------------------ M/M/1
MM1_DPS = np.array([[0.9, 1.0], [0.5, 1.0], [1.2, 1.0]])


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP", "CTA"])
@pytest.mark.parametrize("n_clients", [1, 31, 1000, 1337])
def test_mm1_all_mappings(eng, torch_mod, mapping, n_clients):
    t = torch_mod
    n_reps = 37
    items = oracle.all_items(3, n_reps)
    out = [t.empty(3 * n_reps, dtype=t.float64, device="cuda") for _ in range(3)]
    eng.mrip_mm1_simulate(dev(t, MM1_DPS), n_reps, n_clients, 42,
                          getattr(eng, "MRIP_MAP_" + mapping), *out)
    ref = oracle.mm1(MM1_DPS, *items, n_clients, 42, threads=threads())
    for g, r in zip(out, ref):
        np.testing.assert_allclose(g.cpu().numpy(), r, rtol=REL, atol=1e-300)


@pytest.mark.parametrize("n_clients", [3000, 5000, 100003])
def test_mm1_cta_fallbacks(eng, torch_mod, n_clients):
    """One replication per CTA with a block scan of fixed-point maps: slow
    rates (below 2^-6) and a queue whose wait passes 2^12 redo the
    replication in FP64; ~4 clients per thread up to 1,024 threads, then
    longer segments."""
    t = torch_mod
    dps = np.array([[0.9, 1.0], [0.005, 0.01], [3.0, 1.0], [0.5, 16.0]])
    n_reps = 5
    out = [t.empty(4 * n_reps, dtype=t.float64, device="cuda") for _ in range(3)]
    eng.mrip_mm1_simulate(dev(t, dps), n_reps, n_clients, 42, eng.MRIP_MAP_CTA, *out)
    ref = oracle.mm1(dps, *oracle.all_items(4, n_reps), n_clients, 42, threads=threads())
    for g, r in zip(out, ref):
        np.testing.assert_allclose(g.cpu().numpy(), r, rtol=REL, atol=1e-300)
    if n_clients >= 5000:
        assert ref[0][2 * n_reps:3 * n_reps].min() > 4096 / 4  # the unstable point really grows


def test_mm1_workload_full(eng, torch_mod):
    """32 replications x 1,000 clients, lambda 0.9, mu 1, seed 42: every value."""
    t = torch_mod
    w = mrip_inputs.workload("mm1_32")
    wait = t.empty(w["n_reps"], dtype=t.float64, device="cuda")
    eng.mrip_mm1_simulate(dev(t, w["dps"]), w["n_reps"], w["n_clients"], w["seed"],
                          eng.MRIP_MAP_WARP_COOP, wait)
    ref, _, _ = oracle.mm1(w["dps"], *oracle.all_items(1, w["n_reps"]), w["n_clients"], w["seed"])
    np.testing.assert_allclose(wait.cpu().numpy(), ref, rtol=REL)
    c = ostats.ci(ref, 0.95)
    m = eng.Model(eng.MRIP_MM1, n_clients=w["n_clients"])
    m.set_plan('{"mapping": 3}')
    m.run(w["dps"], w["n_reps"], w["seed"])
    s = m.stats(0.95)[0]
    assert s["n"] == 32
    assert s["mean"] == pytest.approx(c["mean"], rel=REL)
    assert s["half_width"] == pytest.approx(c["half_width"], rel=REL)


# ------------------------------------------------------------------ tandem
def test_tandem_thread_and_wlp(eng, torch_mod):
    t = torch_mod
    dps = mrip_inputs.tandem_design_points(5, seed=3)
    n_reps, n_clients, window = 7, 2000, 100
    ref_y, ref_f = oracle.tandem3(dps, *oracle.all_items(5, n_reps), n_clients, 42,
                                  window=window, threads=threads())
    for mapping in (eng.MRIP_MAP_THREAD, eng.MRIP_MAP_WARP_1LANE, eng.MRIP_MAP_WARP_COOP, eng.MRIP_MAP_CTA):
        y = t.empty(5 * n_reps, dtype=t.float64, device="cuda")
        f = t.empty(8 * 5 * n_reps, dtype=t.float64, device="cuda")
        eng.mrip_tandem3_simulate(dev(t, dps), 0, n_reps, n_clients, window, 42, 0, mapping, y, f)
        np.testing.assert_allclose(y.cpu().numpy(), ref_y, rtol=REL)
        np.testing.assert_allclose(f.cpu().numpy().reshape(8, -1).T, ref_f, rtol=REL)


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP", "CTA"])
def test_tandem_fixed_point_fallbacks(eng, torch_mod, mapping):
    """Times run in 48-bit fixed point; a slow rate (below 2^-6) sends a design
    point to FP64 and an unstable queue whose sojourn time passes 2^12
    restarts its replication in FP64.  All within 1e-12 of the oracle."""
    t = torch_mod
    dps = np.array([[0.9, 1.0, 1.1, 1.2],      # fixed point all the way
                    [0.005, 0.01, 0.02, 0.03],  # rates below 2^-6: FP64
                    [2.0, 1.0, 1.5, 1.5],       # unstable: passes 2^12 after ~8,000 clients
                    [0.5, 16.0, 1.0, 3.0],      # a service rate at the upper bound 2^4
                    [0.5, 2.0**30, 1.0, 3.0]])  # above it: FP64
    n_reps, n_clients, window = 3, 12000, 50
    ry, rf = oracle.tandem3(dps, *oracle.all_items(5, n_reps), n_clients, 42, window=window,
                            threads=threads())
    y = t.empty(5 * n_reps, dtype=t.float64, device="cuda")
    f = t.empty(8 * 5 * n_reps, dtype=t.float64, device="cuda")
    eng.mrip_tandem3_simulate(dev(t, dps), 0, n_reps, n_clients, window, 42, 0,
                              getattr(eng, "MRIP_MAP_" + mapping), y, f)
    np.testing.assert_allclose(y.cpu().numpy(), ry, rtol=REL)
    np.testing.assert_allclose(f.cpu().numpy().reshape(8, -1).T, rf, rtol=REL)
    assert ry[6:9].min() > 4096 / 4  # the unstable point really grows


def test_tandem_offset_tag_and_short_runs(eng, torch_mod):
    t = torch_mod
    dps = mrip_inputs.tandem_design_points(3, seed=4)
    # control runs: tag 2, replications 5..13, only the early window simulated
    y = t.empty(3 * 9, dtype=t.float64, device="cuda")
    f = t.empty(8 * 3 * 9, dtype=t.float64, device="cuda")
    eng.mrip_tandem3_simulate(dev(t, dps), 5, 9, 100, 100, 42, 2, eng.MRIP_MAP_THREAD, y, f)
    dp, rep = oracle.all_items(3, 9)
    ry, rf = oracle.tandem3(dps, dp, rep + 5, 100, 42, window=100, tag=2)
    np.testing.assert_allclose(y.cpu().numpy(), ry, rtol=REL)
    np.testing.assert_allclose(f.cpu().numpy().reshape(8, -1).T, rf, rtol=REL)
    # fewer clients than the window
    eng.mrip_tandem3_simulate(dev(t, dps), 0, 9, 7, 100, 42, 0, eng.MRIP_MAP_THREAD, y, f)
    ry, rf = oracle.tandem3(dps, *oracle.all_items(3, 9), 7, 42, window=100)
    np.testing.assert_allclose(f.cpu().numpy().reshape(8, -1).T, rf, rtol=REL)


@pytest.mark.parametrize("mapping", ["WARP_COOP", "CTA"])
@pytest.mark.parametrize("n_clients,window", [(1, 1), (31, 5), (33, 100), (1000, 64), (4099, 100),
                                              (100003, 4096)])
def test_tandem_warp_coop_ragged(eng, torch_mod, n_clients, window, mapping):
    """Warp scan over 32 client segments: fewer clients than lanes, a
    ragged last segment, window shorter and longer than a segment, a long
    horizon; offset replications and a non-zero stream tag."""
    t = torch_mod
    dps = mrip_inputs.tandem_design_points(3, seed=11)
    n_reps, rep0 = 4, 3
    dp, rep = oracle.all_items(3, n_reps)
    ry, rf = oracle.tandem3(dps, dp, rep + rep0, n_clients, 42, window=window, tag=2,
                            threads=threads())
    y = t.empty(3 * n_reps, dtype=t.float64, device="cuda")
    f = t.empty(8 * 3 * n_reps, dtype=t.float64, device="cuda")
    eng.mrip_tandem3_simulate(dev(t, dps), rep0, n_reps, n_clients, window, 42, 2,
                              getattr(eng, "MRIP_MAP_" + mapping), y, f)
    np.testing.assert_allclose(y.cpu().numpy(), ry, rtol=REL)
    np.testing.assert_allclose(f.cpu().numpy().reshape(8, -1).T, rf, rtol=REL)


def test_tandem_workload_full(eng, torch_mod):
    """4,096 design points x 256 replications x 10,000 clients on the GPU;
    every replication's output and 8 features against the oracle (about 40 s
    on 16 host cores)."""
    t = torch_mod
    w = mrip_inputs.workload("tandem_cv")
    n = w["n_dp"] * w["n_reps"]
    y = t.empty(n, dtype=t.float64, device="cuda")
    f = t.empty(8 * n, dtype=t.float64, device="cuda")
    eng.mrip_tandem3_simulate(dev(t, w["dps"]), 0, w["n_reps"], w["n_clients"], w["window"],
                              w["seed"], 0, eng.MRIP_MAP_THREAD, y, f)
    ry, rf = oracle.tandem3(w["dps"], *oracle.all_items(w["n_dp"], w["n_reps"]), w["n_clients"], w["seed"],
                            window=w["window"], threads=threads())
    gy = y.cpu().numpy()
    gf = f.cpu().numpy().reshape(8, -1).T
    np.testing.assert_allclose(gy, ry, rtol=REL)
    np.testing.assert_allclose(gf, rf, rtol=REL)


# ------------------------------------------------------------------ forest fire
@pytest.mark.parametrize("L", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("n_steps", [1, 64, 130])
def test_forest_fire_bit_exact(eng, torch_mod, L, n_steps):
    """Every lattice width the kernel has: 1 to 16 words per row (the widths of
    8 and 16 words take the carry-chain counter add and word-indexed
    neighbours), over one step, one 64-step chunk and a ragged count."""
    t = torch_mod
    if L == 512 and n_steps == 130:
        n_steps = 70
    dps = np.array([[0.05, 0.002], [0.3, 0.05]])
    n_reps = 3
    items = 2 * n_reps
    counts = t.empty(items * n_steps, dtype=t.int32, device="cuda")
    scalar = t.empty(items, dtype=t.float64, device="cuda")
    final = t.empty(items * L * L, dtype=t.uint8, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, dps), n_reps, L, n_steps, 0.5, 42, None, counts,
                                  scalar, final)
    gc = counts.cpu().numpy().reshape(items, n_steps)
    gs = final.cpu().numpy().reshape(items, L, L)
    gsc = scalar.cpu().numpy()
    for i, (d, r) in enumerate(zip(*oracle.all_items(2, n_reps))):
        rc, rs = oracle.forest_fire_rep(L, n_steps, dps[d, 0], dps[d, 1], 0.5, 42, d, r)
        assert np.array_equal(gc[i], rc)
        assert np.array_equal(gs[i], rs)
        assert gsc[i] == rc.sum() / (n_steps * L * L)


def test_forest_fire_from_given_states(eng, torch_mod):
    t = torch_mod
    L, n_steps, n_reps = 64, 70, 4
    rng = np.random.default_rng(5)
    init = rng.integers(0, 3, size=(n_reps, L, L)).astype(np.uint8)
    init[0] = 1
    init[0, 10, 10] = 2  # single fire front on a full forest
    dps = np.array([[0.0, 0.0]])
    counts = t.empty(n_reps * n_steps, dtype=t.int32, device="cuda")
    final = t.empty(n_reps * L * L, dtype=t.uint8, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, dps), n_reps, L, n_steps, 0.5, 7, dev(t, init), counts,
                                  None, final)
    gc = counts.cpu().numpy().reshape(n_reps, n_steps)
    for r in range(n_reps):
        rc, rs = oracle.forest_fire_rep(L, n_steps, 0.0, 0.0, 0.5, 7, 0, r, init_state=init[r])
        assert np.array_equal(gc[r], rc)
        assert np.array_equal(final.cpu().numpy().reshape(n_reps, L, L)[r], rs)
    assert gc[0, :31].tolist() == [4 * k for k in range(1, 32)]


def test_forest_fire_zero_steps_is_initial_state(eng, torch_mod):
    t = torch_mod
    L = 128
    final = t.empty(2 * L * L, dtype=t.uint8, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, [[0.01, 1e-5]]), 2, L, 0, 0.37, 42, None, None, None,
                                  final)
    for r in range(2):
        _, rs = oracle.forest_fire_rep(L, 0, 0.01, 1e-5, 0.37, 42, 0, r)
        assert np.array_equal(final.cpu().numpy().reshape(2, L, L)[r], rs)


def test_forest_fire_workload_full(eng, torch_mod):
    """128x128, 1,000 steps, 1,024 replications on the GPU; every replication's
    1,000 counts bit-exact against the oracle (about 7 s on 16 host cores)."""
    t = torch_mod
    w = mrip_inputs.workload("ff128")
    counts = t.empty(w["n_reps"] * w["n_steps"], dtype=t.int32, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, w["dps"]), w["n_reps"], w["L"], w["n_steps"],
                                  w["density"], w["seed"], None, counts)
    gc = counts.cpu().numpy().reshape(w["n_reps"], w["n_steps"])
    rc = oracle.forest_fire(w["L"], w["n_steps"], w["dps"], w["density"],
                            *oracle.all_items(1, w["n_reps"]), w["seed"], threads=threads())
    assert np.array_equal(gc, rc)
    assert gc.min() >= 0 and gc.max() <= w["L"] ** 2


def test_forest_fire_cv_workload_sampled(eng, torch_mod):
    """256x256, 2,000 steps, 64 design points x 128 replications on the GPU in
    the bench's launch; every design point's replications {0, 1, 127} at full
    length bit-exact against the oracle (192 replications)."""
    t = torch_mod
    w = mrip_inputs.workload("ff256_cv")
    n = w["n_dp"] * w["n_reps"]
    counts = t.empty(n * w["n_steps"], dtype=t.int32, device="cuda")
    scalar = t.empty(n, dtype=t.float64, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, w["dps"]), w["n_reps"], w["L"], w["n_steps"],
                                  w["density"], w["seed"], None, counts, scalar)
    gc = counts.cpu().numpy().reshape(n, w["n_steps"])
    dp = np.repeat(np.arange(w["n_dp"]), 3).astype(np.int32)
    rep = np.tile([0, 1, w["n_reps"] - 1], w["n_dp"])
    rc = oracle.forest_fire(w["L"], w["n_steps"], w["dps"], w["density"], dp, rep, w["seed"],
                            threads=threads())
    idx = dp * w["n_reps"] + rep
    assert np.array_equal(gc[idx], rc)
    sc = scalar.cpu().numpy()[idx]
    assert np.array_equal(sc, rc.sum(axis=1) / (w["n_steps"] * w["L"] ** 2))


def test_forest_fire_cv_workload_every_replication_short(eng, torch_mod):
    """The same 8,192 replications cut to 100 steps: every one bit-exact."""
    t = torch_mod
    w = mrip_inputs.workload("ff256_cv")
    n, steps = w["n_dp"] * w["n_reps"], 100
    counts = t.empty(n * steps, dtype=t.int32, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, w["dps"]), w["n_reps"], w["L"], steps, w["density"],
                                  w["seed"], None, counts)
    rc = oracle.forest_fire(w["L"], steps, w["dps"], w["density"],
                            *oracle.all_items(w["n_dp"], w["n_reps"]), w["seed"], threads=threads())
    assert np.array_equal(counts.cpu().numpy().reshape(n, steps), rc)


# ------------------------------------------------------------------ walk
WALK_MAPS = ["PERSISTENT", "THREAD", "WARP_1LANE", "WARP_COOP"]


@pytest.mark.parametrize("mapping", WALK_MAPS)
def test_walk_all_mappings_bit_exact(eng, torch_mod, mapping):
    t = torch_mod
    radii = [1.0, 2.0, 3.0, 16.0, 33.0, 5.0]
    n_reps = 301
    tau = t.empty(len(radii) * n_reps, dtype=t.int64, device="cuda")
    eng.mrip_walk_simulate(radii, n_reps, 42, 1 << 38, getattr(eng, "MRIP_MAP_" + mapping), tau,
                           warps_per_cta=4, ctas_per_sm=2, chunk=37)
    t.cuda.synchronize()
    eng.mrip_check_device_flags()
    ref = oracle.walk(radii, *oracle.all_items(len(radii), n_reps), 42, threads=threads())
    assert np.array_equal(tau.cpu().numpy(), ref)


@pytest.mark.parametrize("mapping", WALK_MAPS)
def test_walk_step_cap_reported(eng, torch_mod, mapping):
    t = torch_mod
    tau = t.empty(2 * 40, dtype=t.int64, device="cuda")
    eng.mrip_walk_simulate([200.0, 2.0], 40, 42, 100, getattr(eng, "MRIP_MAP_" + mapping), tau)
    t.cuda.synchronize()
    with pytest.raises(eng.MripError) as e:
        eng.mrip_check_device_flags()
    assert e.value.code == 4
    got = tau.cpu().numpy()
    ref = oracle.walk([200.0, 2.0], *oracle.all_items(2, 40), 42, max_steps=100)
    assert np.array_equal(got, ref) and np.all(got[:40] == -1)
    eng.mrip_check_device_flags()  # the flag was cleared


@pytest.mark.parametrize("shape", [(1, 1, 64), (0, 0, 0)])
def test_walk_step_cap_inside_rounds(eng, torch_mod, shape):
    """Exit times around the cap (E[tau] ~ 960 at R = 40, cap 1,000, not a
    multiple of 64 or 512): walkers exit before, at and after it, in the
    lane-parallel loop (one warp per SM takes 64 at a time, so lanes refill)
    and in the cooperative tail (512-move rounds). Bit-exact, -1 past the cap."""
    t = torch_mod
    radii, n_reps, cap = [40.0, 41.0], 3000, 1000
    tau = t.empty(len(radii) * n_reps, dtype=t.int64, device="cuda")
    w, k, ch = shape
    eng.mrip_walk_simulate(radii, n_reps, 5, cap, eng.MRIP_MAP_PERSISTENT, tau,
                           warps_per_cta=w, ctas_per_sm=k, chunk=ch)
    t.cuda.synchronize()
    with pytest.raises(eng.MripError) as e:
        eng.mrip_check_device_flags()
    assert e.value.code == 4
    got = tau.cpu().numpy()
    ref = oracle.walk(radii, *oracle.all_items(len(radii), n_reps), 5, max_steps=cap, threads=threads())
    assert np.array_equal(got, ref)
    assert np.any(got == -1) and np.any(got > 900)


def test_walk_workload_full(eng, torch_mod):
    """8 radii x 2^17 replications, persistent work stealing in the bench's
    launch; every replication bit-exact against the oracle (about 3 s on 16
    host cores), every tau has the parity of R."""
    t = torch_mod
    w = mrip_inputs.workload("walk8")
    radii = w["dps"][:, 0]
    n = len(radii) * w["n_reps"]
    tau = t.empty(n, dtype=t.int64, device="cuda")
    eng.mrip_walk_simulate(radii, w["n_reps"], w["seed"], 1 << 38, eng.MRIP_MAP_PERSISTENT, tau)
    t.cuda.synchronize()
    eng.mrip_check_device_flags()
    g = tau.cpu().numpy()
    dp = np.repeat(np.arange(len(radii)), w["n_reps"])
    assert np.all(g % 2 == radii[dp].astype(np.int64) % 2) and np.all(g >= radii[dp])
    ref = oracle.walk(radii, *oracle.all_items(len(radii), w["n_reps"]), w["seed"], threads=threads())
    assert np.array_equal(g, ref)


# ------------------------------------------------------------------ statistics
@pytest.mark.parametrize("n_reps", [1, 2, 255, 257, 4096, 4097, 12289, 1 << 17, 1 << 21])
def test_stats_reduce(eng, torch_mod, n_reps):
    """One CTA up to 4,096 replications, then slices merged in order (a ragged
    last slice at 4,097 and 12,289; 256 slices at 2^21)."""
    t = torch_mod
    n_dp = 5
    x = mrip_inputs.random_matrix((n_dp, n_reps), 3, scale=2.0, loc=7.0)
    out = t.empty(n_dp * 3, dtype=t.float64, device="cuda")
    eng.mrip_stats_reduce(dev(t, x), out)
    got = out.cpu().numpy().reshape(n_dp, 3)
    for d in range(n_dp):
        n, mean, var = ostats.dp_stats(x[d])
        assert got[d, 0] == n
        assert got[d, 1] == pytest.approx(mean, rel=1e-13)
        if n > 1:
            assert got[d, 2] / (n - 1) == pytest.approx(var, rel=1e-12)
        else:
            assert got[d, 2] == 0.0


@pytest.mark.parametrize("n_reps", [1000, 4097, 1 << 17])
def test_stats_reduce_large_mean_small_spread(eng, torch_mod, n_reps):
    """Mean 1e9, spread 1e-2: deviations taken from the rounded mean alone
    (an ulp of 1e9 is 1.2e-7) miss the variance by up to ~1e-10 relative; the
    corrected two-pass term (the sum of the deviations) removes that, on both
    sides."""
    t = torch_mod
    n_dp = 3
    x = mrip_inputs.random_matrix((n_dp, n_reps), 5, scale=1e-2, loc=1e9)
    out = t.empty(n_dp * 3, dtype=t.float64, device="cuda")
    eng.mrip_stats_reduce(dev(t, x), out)
    got = out.cpu().numpy().reshape(n_dp, 3)
    for d in range(n_dp):
        n, mean, var = ostats.dp_stats(x[d])
        assert got[d, 0] == n
        assert got[d, 1] == pytest.approx(mean, rel=1e-14)
        assert got[d, 2] / (n - 1) == pytest.approx(var, rel=1e-12)


def test_stats_reduce_i64(eng, torch_mod):
    t = torch_mod
    rng = np.random.default_rng(4)
    x = rng.integers(0, 1 << 40, size=(3, 50001), dtype=np.int64)
    out = t.empty(9, dtype=t.float64, device="cuda")
    eng.mrip_stats_reduce_i64(dev(t, x), out)
    got = out.cpu().numpy().reshape(3, 3)
    for d in range(3):
        n, mean, var = ostats.dp_stats(x[d].astype(np.float64))
        assert got[d, 0] == n
        assert got[d, 1] == pytest.approx(mean, rel=1e-13)
        assert got[d, 2] / (n - 1) == pytest.approx(var, rel=1e-12)


# ------------------------------------------------------------------ model handles
def test_handles_match_oracle_intervals(eng, torch_mod):
    # forest fire, 2 design points x 20 replications
    m = eng.Model(eng.MRIP_FOREST_FIRE, L=64, n_steps=120, density=0.5, window=25)
    dps = np.array([[0.02, 0.001], [0.2, 0.0001]])
    m.run(dps, 20, 9)
    st = m.stats(0.95)
    counts = m.outputs(0, np.int32).reshape(40, 120)
    rc = oracle.forest_fire(64, 120, dps, 0.5, *oracle.all_items(2, 20), 9, threads=threads())
    assert np.array_equal(counts, rc)
    y = rc.sum(axis=1) / (120 * 64 * 64)
    for d in range(2):
        c = ostats.ci(y[d * 20:(d + 1) * 20])
        assert st[d]["mean"] == pytest.approx(c["mean"], rel=REL)
        assert st[d]["half_width"] == pytest.approx(c["half_width"], rel=REL)
    m.close()
    # walk, plans and a second run of the same graph with a new seed
    wm = eng.Model(eng.MRIP_WALK_L1_EXIT, max_steps=1 << 38)
    radii = np.array([[12.0], [7.0], [20.0]])
    for plan in ('{"mapping": 5, "warps_per_cta": 4, "ctas_per_sm": 1, "chunk": 16}',
                 '{"mapping": 1}', '{"mapping": 3}'):
        for seed in (1, 2):
            wm.set_plan(plan)
            wm.run(radii, 100, seed)
            st = wm.stats(0.95)
            tau = wm.outputs(0, np.int64)
            ref = oracle.walk(radii[:, 0], *oracle.all_items(3, 100), seed)
            assert np.array_equal(tau, ref)
            for d in range(3):
                c = ostats.ci(ref[d * 100:(d + 1) * 100].astype(np.float64))
                assert st[d]["mean"] == pytest.approx(c["mean"], rel=REL)
                assert st[d]["half_width"] == pytest.approx(c["half_width"], rel=REL)
    wm.close()
    # tandem and M/M/1 handles
    tm = eng.Model(eng.MRIP_TANDEM3, n_clients=500, window=50)
    tdp = mrip_inputs.tandem_design_points(4, seed=8)
    tm.run(tdp, 9, 5)
    ty = tm.outputs(0).reshape(4, 9)
    ry, _ = oracle.tandem3(tdp, *oracle.all_items(4, 9), 500, 5, window=50)
    np.testing.assert_allclose(ty.reshape(-1), ry, rtol=REL)
    tm.set_plan('{"mapping": %d}' % eng.MRIP_MAP_WARP_COOP)
    tm.run(tdp, 9, 5)
    np.testing.assert_allclose(tm.outputs(0), ry, rtol=REL)
    tm.close()
    # M/M/1 handle in the CTA mapping (block scan), replayed as a graph twice
    qm = eng.Model(eng.MRIP_MM1, n_clients=777)
    qm.set_plan('{"mapping": %d}' % eng.MRIP_MAP_CTA)
    qdp = np.array([[0.9, 1.0], [0.6, 1.3]])
    rw, _, _ = oracle.mm1(qdp, *oracle.all_items(2, 40), 777, 6)
    for _ in range(2):
        qm.run(qdp, 40, 6)
        np.testing.assert_allclose(qm.outputs(0), rw, rtol=REL)
        st = qm.stats(0.95)
        for d in range(2):
            c = ostats.ci(rw[d * 40:(d + 1) * 40])
            assert st[d]["mean"] == pytest.approx(c["mean"], rel=REL)
    qm.close()


def test_autotune_queues_keep_results(eng, torch_mod, tmp_path):
    """The queue autotuners time THREAD, CTA / WARP_COOP and WARP_1LANE; whatever
    they pick reproduces the oracle."""
    qm = eng.Model(eng.MRIP_MM1, n_clients=3000)
    qdp = np.array([[0.9, 1.0]])
    qm.autotune(qdp, 8, 11, trials=1, cache_path=str(tmp_path / "q.jsonl"))
    assert '"mapping"' in qm.get_plan()
    qm.run(qdp, 8, 11)
    rw, _, _ = oracle.mm1(qdp, *oracle.all_items(1, 8), 3000, 11)
    np.testing.assert_allclose(qm.outputs(0), rw, rtol=REL)
    qm.close()
    tm = eng.Model(eng.MRIP_TANDEM3, n_clients=20000, window=100)
    tdp = mrip_inputs.tandem_design_points(2, seed=12)
    tm.autotune(tdp, 3, 13, trials=1, cache_path=str(tmp_path / "t.jsonl"))
    tm.run(tdp, 3, 13)
    ry, _ = oracle.tandem3(tdp, *oracle.all_items(2, 3), 20000, 13, window=100)
    np.testing.assert_allclose(tm.outputs(0), ry, rtol=REL)
    tm.close()


def test_autotune_keeps_results_and_picks_a_plan(eng, torch_mod, tmp_path):
    wm = eng.Model(eng.MRIP_WALK_L1_EXIT, max_steps=1 << 38)
    radii = np.array([[64.0], [16.0], [32.0]])
    cache = str(tmp_path / "plans.jsonl")
    wm.autotune(radii, 2000, 3, trials=1, cache_path=cache)
    plan = wm.get_plan()
    assert '"mapping"' in plan
    text = open(cache).read()
    assert text.count("\n") == 1
    # cached: a second autotune reads the file and times nothing
    wm2 = eng.Model(eng.MRIP_WALK_L1_EXIT, max_steps=1 << 38)
    wm2.autotune(radii, 2000, 3, trials=1, cache_path=cache)
    assert wm2.get_plan() == plan
    assert open(cache).read().count("\n") == 1
    wm2.run(radii, 2000, 3)
    ref = oracle.walk(radii[:, 0], *oracle.all_items(3, 2000), 3, threads=threads())
    assert np.array_equal(wm2.outputs(0, np.int64), ref)
    wm.close()
    wm2.close()


def test_errors_do_not_poison_the_context(eng, torch_mod):
    t = torch_mod
    with pytest.raises(eng.MripError):
        eng.mrip_mm1_simulate(dev(t, MM1_DPS), 2, 0, 42, eng.MRIP_MAP_THREAD,
                              t.empty(6, dtype=t.float64, device="cuda"))
    m = eng.Model(eng.MRIP_MM1, n_clients=10)
    with pytest.raises(eng.MripError):
        m.run(np.array([[0.5, -1.0]]), 4, 1)
    m.run(np.array([[0.5, 1.0]]), 4, 1)
    assert m.stats()[0]["n"] == 4
    m.close()


# ------------------------------------------------------------------ area walk
@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP"])
@pytest.mark.parametrize("n_steps", [0, 1, 17, 1000, 1537])
def test_area_walk_all_mappings_bit_exact(eng, torch_mod, mapping, n_steps):
    t = torch_mod
    n = 301
    fa = t.full((n,), -1, dtype=t.int32, device="cuda")
    vis = t.full((30 * n,), -1, dtype=t.int32, device="cuda")
    eng.mrip_area_walk_simulate(n, n_steps, 42, getattr(eng, "MRIP_MAP_" + mapping), fa, vis)
    ref_f, ref_v = oracle.area_walk(np.arange(n), n_steps, 42, threads=threads())
    if n_steps > 0:
        assert np.array_equal(fa.cpu().numpy(), ref_f)
    else:
        assert np.all(fa.cpu().numpy() == 15)
    assert np.array_equal(vis.cpu().numpy().reshape(30, n).T, ref_v)


# ------------------------------------------------------------------ Monte Carlo pi
@pytest.mark.parametrize("n_draws", [0, 1, 2, 3, 65535, 65536, 65537, 10**7])
def test_pi_bit_exact(eng, torch_mod, n_draws):
    t = torch_mod
    reps = 5 if n_draws < 10**7 else 3
    hits = t.full((reps,), -1, dtype=t.int64, device="cuda")
    eng.mrip_pi_simulate(reps, n_draws, 42, hits)
    ref = oracle.pi_hits(np.arange(reps), n_draws, 42, threads=threads())
    assert np.array_equal(hits.cpu().numpy(), ref)


# ------------------------------------------------------------------ skip-sampled forest fire
def _skip_run(eng, t, dps, n_reps, L, n_steps, density, seed, init=None):
    items = len(dps) * n_reps
    counts = t.empty(max(1, items * n_steps), dtype=t.int32, device="cuda")
    scalar = t.empty(items, dtype=t.float64, device="cuda")
    final = t.empty(items * L * L, dtype=t.uint8, device="cuda")
    eng.mrip_forest_fire_skip_simulate(dev(t, dps), n_reps, L, n_steps, density, seed,
                                       None if init is None else dev(t, init), counts, scalar, final)
    return (counts.cpu().numpy()[:items * n_steps].reshape(items, n_steps), scalar.cpu().numpy(),
            final.cpu().numpy().reshape(items, L, L))


@pytest.mark.parametrize("L", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("n_steps", [1, 64, 130])
def test_forest_fire_skip_bit_exact(eng, torch_mod, L, n_steps):
    """Event sets of tiny, moderate and large probabilities (several 64-gap
    rounds per step), over a ragged number of steps and every lattice size."""
    t = torch_mod
    if L == 512 and n_steps == 130:
        n_steps = 20
    dps = np.array([[0.01, 1e-5], [0.3, 0.05], [0.97, 0.0]])
    n_reps = 2
    gc, gsc, gs = _skip_run(eng, t, dps, n_reps, L, n_steps, 0.5, 42)
    compared = 0
    for i, (d, r) in enumerate(zip(*oracle.all_items(len(dps), n_reps))):
        rc, rs, ties = oracle.forest_fire_skip_rep(L, n_steps, dps[d, 0], dps[d, 1], 0.5, 42, d, r)
        if ties:
            continue
        compared += 1
        assert np.array_equal(gc[i], rc), (d, r)
        assert np.array_equal(gs[i], rs), (d, r)
        assert gsc[i] == rc.sum() / (n_steps * L * L)
    assert compared == len(dps) * n_reps


def test_forest_fire_skip_edges(eng, torch_mod):
    """No events (p = 0), every cell (p = 1), zero steps, given states."""
    t = torch_mod
    L, n_steps, n_reps = 64, 70, 3
    rng = np.random.default_rng(9)
    init = rng.integers(0, 3, size=(2 * n_reps, L, L)).astype(np.uint8)
    init[0] = 1
    init[0, 10, 10] = 2
    dps = np.array([[0.0, 0.0], [1.0, 0.5]])
    gc, _, gs = _skip_run(eng, t, dps, n_reps, L, n_steps, 0.5, 7, init=init)
    for i, (d, r) in enumerate(zip(*oracle.all_items(2, n_reps))):
        rc, rs, ties = oracle.forest_fire_skip_rep(L, n_steps, dps[d, 0], dps[d, 1], 0.5, 7, d, r,
                                                   init_state=init[i])
        assert ties == 0
        assert np.array_equal(gc[i], rc) and np.array_equal(gs[i], rs)
    assert gc[0, :31].tolist() == [4 * k for k in range(1, 32)]
    _, _, gs0 = _skip_run(eng, t, np.array([[0.01, 1e-5]]), 2, 128, 0, 0.37, 42)
    for r in range(2):
        _, rs, _ = oracle.forest_fire_skip_rep(128, 0, 0.01, 1e-5, 0.37, 42, 0, r)
        assert np.array_equal(gs0[r], rs)


def test_forest_fire_skip_workload_full(eng, torch_mod):
    """The 128x128, 1,000-step, 1,024-replication workload with skip-sampled
    events, in the bench's launch: every replication's 1,000 counts and its
    scalar bit-exact against the oracle.  Where floating point decides a gap
    (the oracle floors E / mu in FP64, the kernel in integers) the two may
    differ only when E / mu lies within a few ulps of an integer; the oracle
    flags such draws, and this workload has none."""
    t = torch_mod
    w = mrip_inputs.workload("ff128")
    n = w["n_reps"]
    counts = t.empty(n * w["n_steps"], dtype=t.int32, device="cuda")
    scalar = t.empty(n, dtype=t.float64, device="cuda")
    eng.mrip_forest_fire_skip_simulate(dev(t, w["dps"]), n, w["L"], w["n_steps"],
                                       w["density"], w["seed"], None, counts, scalar)
    gc = counts.cpu().numpy().reshape(n, w["n_steps"])
    rc, ties = oracle.forest_fire_skip(w["L"], w["n_steps"], w["dps"], w["density"],
                                       *oracle.all_items(1, n), w["seed"], threads=threads())
    assert int(ties.sum()) == 0
    assert np.array_equal(gc, rc)
    assert np.array_equal(scalar.cpu().numpy(), rc.sum(axis=1) / (w["n_steps"] * w["L"] ** 2))


def test_forest_fire_skip_cv_workload_sampled(eng, torch_mod):
    """256x256, 2,000 steps, 64 design points x 128 replications with
    skip-sampled events (p_grow up to 0.05): every design point's
    replications {0, 1, 127} at full length bit-exact against the oracle
    (192 replications, no near-ties)."""
    t = torch_mod
    w = mrip_inputs.workload("ff256_cv")
    n = w["n_dp"] * w["n_reps"]
    counts = t.empty(n * w["n_steps"], dtype=t.int32, device="cuda")
    eng.mrip_forest_fire_skip_simulate(dev(t, w["dps"]), w["n_reps"], w["L"], w["n_steps"],
                                       w["density"], w["seed"], None, counts)
    gc = counts.cpu().numpy().reshape(n, w["n_steps"])
    dp = np.repeat(np.arange(w["n_dp"]), 3).astype(np.int32)
    rep = np.tile([0, 1, w["n_reps"] - 1], w["n_dp"])
    rc, ties = oracle.forest_fire_skip(w["L"], w["n_steps"], w["dps"], w["density"], dp, rep,
                                       w["seed"], threads=threads())
    assert int(ties.sum()) == 0
    assert np.array_equal(gc[dp * w["n_reps"] + rep], rc)


# ------------------------------------------------------------------ empty batches
def test_every_stage_accepts_an_empty_batch(eng, torch_mod):
    """Zero replications (or design points) is a valid request for every stage
    entry point: it succeeds and leaves the outputs untouched."""
    t = torch_mod
    sentinel = t.full((4,), 7.0, dtype=t.float64, device="cuda")
    eng.mrip_mm1_simulate(dev(t, MM1_DPS), 0, 100, 42, eng.MRIP_MAP_CTA, sentinel)
    eng.mrip_mm1_simulate(dev(t, MM1_DPS), 0, 100, 42, eng.MRIP_MAP_THREAD, sentinel)
    eng.mrip_tandem3_simulate(dev(t, mrip_inputs.tandem_design_points(2, seed=1)), 0, 0, 100, 10, 42,
                              0, eng.MRIP_MAP_WARP_COOP, sentinel)
    counts = t.full((4,), 7, dtype=t.int32, device="cuda")
    eng.mrip_forest_fire_simulate(dev(t, [[0.01, 1e-5]]), 0, 64, 10, 0.5, 42, None, counts)
    eng.mrip_forest_fire_skip_simulate(dev(t, [[0.01, 1e-5]]), 0, 64, 10, 0.5, 42, None, counts)
    tau = t.full((4,), 7, dtype=t.int64, device="cuda")
    eng.mrip_walk_simulate(np.array([16.0]), 0, 42, 1 << 20, eng.MRIP_MAP_PERSISTENT, tau)
    eng.mrip_pi_simulate(0, 1000, 42, tau)
    fa = t.full((4,), 7, dtype=t.int32, device="cuda")
    eng.mrip_area_walk_simulate(0, 100, 42, eng.MRIP_MAP_THREAD, fa, None)
    eng.mrip_stats_reduce(t.empty((0, 5), dtype=t.float64, device="cuda"), sentinel)
    t.cuda.synchronize()
    assert sentinel.cpu().tolist() == [7.0] * 4
    assert counts.cpu().tolist() == [7] * 4 and tau.cpu().tolist() == [7] * 4
    assert fa.cpu().tolist() == [7] * 4
    # design points without replications: (0, 0, 0) each, the empty input may be NULL
    z = t.full((9,), 7.0, dtype=t.float64, device="cuda")
    eng.mrip_stats_reduce(t.empty((3, 0), dtype=t.float64, device="cuda"), z)
    zi = t.full((6,), 7.0, dtype=t.float64, device="cuda")
    eng.mrip_stats_reduce_i64(t.empty((2, 0), dtype=t.int64, device="cuda"), zi)
    assert z.cpu().tolist() == [0.0] * 9 and zi.cpu().tolist() == [0.0] * 6
