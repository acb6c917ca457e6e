"""The bounds-checked debug build on the GPU (compute-sanitizer's stand-in).

The library compiled with -DMRIP_DEBUG checks, inside the kernels, the
data-dependent indices (event positions, the walk's work-item decoding,
minibatch sample indices, map cells, output ranges) and every use of
dynamically sized shared memory against the launch's actual size; a failed
check records (site, index) and skips the access, it never traps.  Here every
model and mapping runs on small ragged shapes through that library: the
outputs must equal the oracle's (bit-exact integers, FP64 within 1e-12) and
no check may have failed.  A deliberately failed check (mrip_debug_selftest,
guarding no access) must arrive at mrip_debug_checks and be cleared by it.
"""
import numpy as np
import pytest

import mrip_inputs
import oracle
from oracle import stats as ostats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1501_01405_gb300 as eng
    from paper_1501_01405_gb300 import build
    L = eng.load_library(build.build(variant="debug"))
    en, first = eng.mrip_debug_checks(L)
    assert en, "the debug variant must report its checks as enabled"
    return eng, torch, L


def _clean(eng, L):
    en, first = eng.mrip_debug_checks(L)
    assert en and first is None, "failed bounds check (site, index) = %r" % (first,)


def _dev(torch, a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def test_failed_check_is_recorded_and_cleared(dbg):
    eng, torch, L = dbg
    _clean(eng, L)
    assert L.mrip_debug_selftest() == 0
    assert eng.mrip_debug_checks(L) == (True, (999, 12345))
    assert eng.mrip_debug_checks(L) == (True, None)


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP", "CTA"])
@pytest.mark.parametrize("n_clients", [77, 13000])
def test_mm1(dbg, mapping, n_clients):
    """13,000 clients: the CTA mapping's stage no longer fits (unstaged replay)
    and the warp mapping's segments are long."""
    eng, torch, L = dbg
    dps = np.array([[0.9, 1.0], [0.02, 9.0]])
    n_reps = 5
    w = torch.empty(2 * n_reps, dtype=torch.float64, device="cuda")
    i = torch.empty_like(w)
    s = torch.empty_like(w)
    with eng.using_library(L):
        eng.mrip_mm1_simulate(_dev(torch, dps, torch.float64), n_reps, n_clients, 42,
                              getattr(eng, "MRIP_MAP_" + mapping), w, i, s, rep0=3)
    ref = oracle.mm1(dps, np.repeat([0, 1], n_reps), np.tile(np.arange(3, 3 + n_reps), 2), n_clients, 42)
    for got, r in zip((w, i, s), ref):
        np.testing.assert_allclose(got.cpu().numpy(), r, rtol=1e-12, atol=0)
    _clean(eng, L)


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_COOP", "CTA"])
def test_tandem(dbg, mapping):
    eng, torch, L = dbg
    dps = mrip_inputs.tandem_design_points(2, seed=9)
    n_reps, n_clients, window = 3, 150, 40
    y = torch.empty(2 * n_reps, dtype=torch.float64, device="cuda")
    f = torch.empty(8 * 2 * n_reps, dtype=torch.float64, device="cuda")
    with eng.using_library(L):
        eng.mrip_tandem3_simulate(_dev(torch, dps, torch.float64), 0, n_reps, n_clients, window, 42, 0,
                                  getattr(eng, "MRIP_MAP_" + mapping), y, f)
    ry, rf = oracle.tandem3(dps, *oracle.all_items(2, n_reps), n_clients, 42, window=window)
    np.testing.assert_allclose(y.cpu().numpy(), ry, rtol=1e-12, atol=0)
    np.testing.assert_allclose(f.view(8, -1).T.cpu().numpy(), rf, rtol=1e-12, atol=0)
    _clean(eng, L)


@pytest.mark.parametrize("skip", [False, True])
@pytest.mark.parametrize("L_side", [32, 64, 128])
def test_forest_fire(dbg, skip, L_side):
    """70 steps: a full 64-step chunk and a ragged one; L = 32 draws the skip
    events with one warp, larger lattices with the shared-round scheme."""
    eng, torch, L = dbg
    dps = np.array([[0.05, 0.001], [0.01, 0.0]])
    n_reps, T = 3, 70
    c = torch.empty(2 * n_reps * T, dtype=torch.int32, device="cuda")
    sc = torch.empty(2 * n_reps, dtype=torch.float64, device="cuda")
    fin = torch.empty(2 * n_reps * L_side * L_side, dtype=torch.uint8, device="cuda")
    fn = eng.mrip_forest_fire_skip_simulate if skip else eng.mrip_forest_fire_simulate
    with eng.using_library(L):
        fn(_dev(torch, dps, torch.float64), n_reps, L_side, T, 0.5, 42, counts=c, scalar=sc, final=fin)
    ofn = oracle.forest_fire_skip_rep if skip else oracle.forest_fire_rep
    got_c = c.view(2, n_reps, T).cpu().numpy()
    got_f = fin.view(2, n_reps, L_side, L_side).cpu().numpy()
    for d in range(2):
        for r in range(n_reps):
            out = ofn(L_side, T, dps[d, 0], dps[d, 1], 0.5, 42, d, r)
            if skip and out[2]:
                continue  # the oracle's FP64 gap was within a few ulps of an integer
            counts, final = out[0], out[1]
            assert np.array_equal(got_c[d, r], counts)
            assert np.array_equal(got_f[d, r], final)
    _clean(eng, L)


@pytest.mark.parametrize("mapping", ["PERSISTENT", "THREAD", "WARP_COOP"])
@pytest.mark.parametrize("noalloc", [False, True])
def test_walk(dbg, mapping, noalloc):
    eng, torch, L = dbg
    radii = np.array([3.0, 16.0, 9.0])
    n_reps = 40
    tau = torch.empty(3 * n_reps, dtype=torch.int64, device="cuda")
    fn = eng.mrip_walk_simulate_noalloc if noalloc else eng.mrip_walk_simulate
    with eng.using_library(L):
        fn(radii, n_reps, 42, 1 << 30, getattr(eng, "MRIP_MAP_" + mapping), tau, chunk=7, rep0=11)
        torch.cuda.synchronize()
    ref = oracle.walk(radii, np.repeat([0, 1, 2], n_reps), np.tile(np.arange(11, 11 + n_reps), 3), 42)
    assert np.array_equal(tau.cpu().numpy(), ref)
    _clean(eng, L)


@pytest.mark.parametrize("mapping", ["THREAD", "WARP_1LANE", "WARP_COOP"])
def test_area_walk(dbg, mapping):
    eng, torch, L = dbg
    n_reps, n_steps = 10, 700
    fa = torch.empty(n_reps, dtype=torch.int32, device="cuda")
    vis = torch.empty(30 * n_reps, dtype=torch.int32, device="cuda")
    with eng.using_library(L):
        eng.mrip_area_walk_simulate(n_reps, n_steps, 42, getattr(eng, "MRIP_MAP_" + mapping), fa, vis)
    rfa, rvis = oracle.area_walk(np.arange(n_reps), n_steps, 42)
    assert np.array_equal(fa.cpu().numpy(), rfa)
    assert np.array_equal(vis.view(30, n_reps).T.cpu().numpy(), rvis)
    _clean(eng, L)


def test_pi_and_statistics(dbg):
    eng, torch, L = dbg
    hits = torch.empty(4, dtype=torch.int64, device="cuda")
    x = mrip_inputs.random_matrix((3, 5001), 2, scale=3.0, loc=-1.0)  # two slices per design point
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    with eng.using_library(L):
        eng.mrip_pi_simulate(4, 10_007, 42, hits)
        eng.mrip_stats_reduce(_dev(torch, x, torch.float64), out)
    assert np.array_equal(hits.cpu().numpy(), oracle.pi_hits(np.arange(4), 10_007, 42))
    got = out.cpu().numpy().reshape(3, 3)
    for d in range(3):
        n, mean, var = ostats.dp_stats(x[d])
        assert got[d, 0] == n
        assert got[d, 1] == pytest.approx(mean, rel=1e-13)
        assert got[d, 2] / (n - 1) == pytest.approx(var, rel=1e-12)
    _clean(eng, L)


def test_training_and_control_variate_pipeline(dbg):
    """The tensor-core training kernel (partial tiles, a validation set) and
    the whole control-variate pipeline of the model handle run through the
    debug library with no failed check; they give the release library's
    results (the same deterministic kernels)."""
    eng, torch, L = dbg
    import oracle.mlp as omlp
    d_in, n = 8, 300
    X = omlp.f32(mrip_inputs.random_matrix((n, d_in), 3))
    y = omlp.f32(np.tanh(X[:, 0]) + 0.2 * mrip_inputs.random_matrix(n, 4))
    theta0 = omlp.init_params(d_in, 5)

    def train():
        dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")  # noqa: E731
        th = dev(theta0)
        info = eng.mrip_mlp_train(d_in, dev(X[:250].T.copy()), dev(y[:250]), th, 64, 3, 7,
                                  xv=dev(X[250:].T.copy()), yv=dev(y[250:]))
        return th.cpu().numpy(), info

    dps = mrip_inputs.tandem_design_points(3, seed=6)

    def cv():
        m = eng.Model(eng.MRIP_TANDEM3, n_clients=200, window=20)
        try:
            return m.run_cv(dps, 60, 42, train_frac=0.3, val_frac=0.2, epochs=3, batch=32, gate=False)
        finally:
            m.close()

    th_rel, info_rel = train()
    plain_rel, cv_rel, _ = cv()
    with eng.using_library(L):
        th_dbg, info_dbg = train()
        plain_dbg, cv_dbg, _ = cv()
    assert info_dbg == info_rel
    np.testing.assert_allclose(th_dbg, th_rel, rtol=1e-6, atol=1e-7)
    for a, b in zip(plain_dbg, plain_rel):
        assert a["mean"] == pytest.approx(b["mean"], rel=1e-12)
    for a, b in zip(cv_dbg, cv_rel):
        assert a["mean"] == pytest.approx(b["mean"], rel=1e-5)
    _clean(eng, L)
