"""GPU parity of the learned control variate: network stages and estimator.

* initialisation bit-exact (FP32) against the oracle;
* forward pass and minibatch gradient against the FP64 oracle evaluated on
  the same BF16-rounded operands (norm-wise relative error <= 1e-3; the GPU
  accumulates in FP32, and an FP32-vs-FP64 difference can flip a BF16
  rounding of an activation);
* one Adam step (FP32 vs FP64, 1e-5);
* the per-design-point estimator on seeded arrays (FP64, 1e-12);
* the whole mrip_run_cv pipeline against the oracle pipeline on small
  tandem and forest-fire workloads: plain intervals and standardisation
  1e-12; given the GPU's trained network, the oracle's validation rho^2,
  control-run count and intervals match (1e-2); the oracle's own training
  reaches the same loss (5 %) and compatible means;
* the gate: an informative early window keeps the control variate with
  control runs sized from rho^2, an uninformative one declines it and
  returns the plain intervals;
* validity: coverage of the control-variate interval over 200 seeds;
* what the network gains: on a workload whose early window is informative
  the control-variate half-width is smaller than the plain one computed on
  the same held-out replications.
"""
import math

import numpy as np
import pytest

import mrip_inputs
import oracle
import oracle.cv as ocv
import oracle.mlp as omlp
import oracle.stats as ostats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1501_01405_gb300 as eng
    eng.lib()
    return eng, torch


def f32dev(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("d_in", [6, 8])
def test_init_bit_exact(env, d_in):
    eng, torch = env
    P = eng.mrip_mlp_param_count(d_in)
    assert P == omlp.n_params(d_in)
    th = torch.empty(P, dtype=torch.float32, device="cuda")
    eng.mrip_mlp_init(d_in, 42, th)
    assert np.array_equal(th.cpu().numpy().astype(np.float64), omlp.init_params(d_in, 42))


def _seeded_net(d_in, seed):
    theta = omlp.init_params(d_in, seed) + mrip_inputs.random_matrix(omlp.n_params(d_in), seed + 1,
                                                                      scale=0.05)
    return omlp.f32(theta)


@pytest.mark.parametrize("d_in,n", [(8, 1000), (6, 77)])
def test_forward(env, d_in, n):
    eng, torch = env
    theta = _seeded_net(d_in, 3)
    X = omlp.f32(mrip_inputs.random_matrix((n, d_in), 4))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    eng.mrip_mlp_forward(f32dev(torch, theta), d_in, f32dev(torch, X.T.copy()), out)
    ref, _ = omlp.forward(theta, X, d_in)
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3
    np.testing.assert_allclose(got, ref, rtol=2e-2, atol=2e-3 * np.abs(ref).max())


@pytest.mark.parametrize("d_in,n,B", [(8, 3000, 1024), (6, 500, 500), (8, 100, 33)])
def test_loss_and_gradient(env, d_in, n, B):
    eng, torch = env
    theta = _seeded_net(d_in, 5)
    X = omlp.f32(mrip_inputs.random_matrix((n, d_in), 6))
    y = omlp.f32(mrip_inputs.random_matrix(n, 7))
    idx = np.random.default_rng(8).choice(n, B, replace=False).astype(np.int64)
    grad = torch.empty(omlp.n_params(d_in), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    eng.mrip_mlp_loss_grad(f32dev(torch, theta), d_in, f32dev(torch, X.T.copy()), f32dev(torch, y),
                           torch.tensor(idx, device="cuda"), B, grad, loss)
    ref_loss, ref_g = omlp.loss_and_grad(theta, X[idx], y[idx], d_in)
    g = grad.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-4)
    assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) < 1e-3
    # every block of parameters on its own (W1, b1, W2, b2, W3, b3)
    for a, b in zip(omlp.unpack(g, d_in), omlp.unpack(ref_g, d_in)):
        assert np.linalg.norm(np.ravel(a) - np.ravel(b)) <= 1e-3 * np.linalg.norm(b) + 1e-7


def test_adam_step(env):
    eng, torch = env
    n = 4801
    theta = omlp.f32(mrip_inputs.random_matrix(n, 1))
    m = omlp.f32(mrip_inputs.random_matrix(n, 2, 0.01))
    v = omlp.f32(np.abs(mrip_inputs.random_matrix(n, 3, 0.01)))
    g = omlp.f32(mrip_inputs.random_matrix(n, 4))
    dt, dm, dv = f32dev(torch, theta), f32dev(torch, m), f32dev(torch, v)
    eng.mrip_adam_step(dt, dm, dv, f32dev(torch, g), 7, 1e-3, 0.9, 0.999, 1e-8)
    # the ABI takes FP32 hyper-parameters: give the oracle the same values
    # (0.999f is 0.99900001287..., so 1 - beta2 differs from 0.001 by 1.3e-5)
    f = lambda x: float(np.float32(x))
    rt, rm, rv = omlp.adam_step(theta, m, v, g, 7, lr=f(1e-3), beta1=f(0.9), beta2=f(0.999),
                                eps=f(1e-8))
    # FP32 against FP64: m and v are sums of two terms that can cancel, so the
    # tolerance is a few FP32 ulps of the terms, not of the result
    scale_m = 0.9 * np.abs(m) + 0.1 * np.abs(g)
    scale_v = 0.999 * v + 0.001 * g * g
    np.testing.assert_allclose(dt.cpu().numpy(), rt, rtol=1e-5, atol=1e-8)
    assert float(np.max(np.abs(dm.cpu().numpy() - rm) / scale_m)) <= 4 * 2.0**-24
    assert float(np.max(np.abs(dv.cpu().numpy() - rv) / scale_v)) <= 4 * 2.0**-24


def test_cv_reduce(env):
    eng, torch = env
    n_dp, n, M = 7, 230, 2301
    Y = np.empty((n_dp, n))
    G = np.empty((n_dp, n))
    GC = np.empty((n_dp, M))
    for d in range(n_dp):
        Y[d], G[d] = mrip_inputs.correlated_pair(n, 0.1 * d, 10 + d)
        GC[d] = mrip_inputs.correlated_pair(M, 0.1 * d, 100 + d)[1]
    out = torch.empty(n_dp * 5, dtype=torch.float64, device="cuda")
    dev = lambda a: torch.tensor(a, device="cuda")
    eng.mrip_cv_reduce(dev(Y), dev(G), dev(GC), out)
    o = out.cpu().numpy().reshape(n_dp, 5)
    for d in range(n_dp):
        r = ocv.cv_estimate(Y[d], G[d], GC[d])
        assert o[d, 0] == pytest.approx(r["beta"], rel=1e-11, abs=1e-14)
        assert o[d, 1] == pytest.approx(r["mean"], rel=1e-12)
        assert o[d, 2] == pytest.approx(r["var"], rel=1e-11)


# the old pipeline semantics: no validation split, no gate, fixed control runs
FIXED = dict(val_frac=0.0, patience=0, gate=False)


def _compare_pipeline(m, kind, dps, n_reps, seed, model_kw, kw, threads):
    """GPU pipeline vs the oracle pipeline.  (1) plain intervals 1e-12;
    (2) the standardisation of the fit set 1e-12; (3) the rest of the
    pipeline -- validation rho^2, control-run count, predictions, control
    runs and estimator -- recomputed by the oracle from the GPU's trained
    network: beta and the interval within 1e-2 (the GPU predicts in FP32 with
    BF16 operands, so g differs from the FP64 oracle's by ~1e-3 relative);
    (4) the oracle's own training for the epochs the GPU ran: last-epoch
    loss within 5 %, means within the combined half-widths."""
    plain, cv, rep = m.run_cv(dps, n_reps, seed, **kw)
    theta, norm = m.cv_network()
    ref_plain, ref_cv, info = ocv.run_cv(kind, dps, n_reps, seed, theta=theta.astype(np.float64),
                                         threads=threads, **model_kw, **kw)
    for g, r in zip(plain, ref_plain):
        assert g["mean"] == pytest.approx(r["mean"], rel=1e-12)
        assert g["half_width"] == pytest.approx(r["half_width"], rel=1e-12)
    xm, xs, ym, ys = info["norm"]
    np.testing.assert_allclose(norm[:-1, 0], xm, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(norm[:-1, 1], xs, rtol=1e-12)
    assert norm[-1, 0] == pytest.approx(ym, rel=1e-12) and norm[-1, 1] == pytest.approx(ys, rel=1e-12)
    if info["val_rho2"] is not None:
        assert rep["val_rho2"] == pytest.approx(info["val_rho2"], abs=2e-3)
    if rep["declined"] == 2:  # the screen (the GPU's network is the screened one)
        n_train = math.ceil(kw["train_frac"] * n_reps)
        assert rep["epochs_run"] < kw["epochs"]
        assert info["val_rho2"] < 0.25 * (1 - (n_reps - n_train) / (1.1 * n_reps)) + 2e-3
    else:
        assert bool(rep["declined"]) == info["declined"]
    assert rep["m_ctrl"] == info["m_ctrl"] or abs(rep["m_ctrl"] - info["m_ctrl"]) <= \
        0.02 * info["m_ctrl"] + 1
    if rep["m_ctrl"] == info["m_ctrl"]:
        for g, r in zip(cv, ref_cv):
            assert g["n"] == r["n"] and g["m"] == r["m"]
            assert abs(g["mean"] - r["mean"]) <= 1e-2 * r["half_width"]
            assert g["half_width"] == pytest.approx(r["half_width"], rel=1e-2)
            assert g["beta"] == pytest.approx(r["beta"], rel=1e-2, abs=1e-3 * abs(r["beta"]) + 1e-12)
    # the oracle trains for as many epochs as the GPU ran (with early stopping
    # the two can stop at different epochs when validation losses nearly tie)
    own_kw = dict(kw, epochs=rep["epochs_run"], patience=0)
    _, own_cv, own = ocv.run_cv(kind, dps, n_reps, seed, threads=threads, **model_kw, **own_kw)
    assert rep["train_loss"] == pytest.approx(own["loss"], rel=0.05)
    if not rep["declined"] and not own["declined"]:
        for g, r in zip(cv, own_cv):
            assert abs(g["mean"] - r["mean"]) <= g["half_width"] + r["half_width"]
    return plain, cv, rep


def test_run_cv_tandem_matches_oracle_pipeline(env):
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(8, seed=3)
    kw = dict(train_frac=0.25, epochs=6, batch=64, lr=3e-3, m_ctrl=300, **FIXED)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=200, window=50)
    _compare_pipeline(m, "tandem3", dps, 48, 7, dict(n_clients=200, window=50), kw,
                      oracle.host_threads())
    m.close()


def test_run_cv_large_minibatch_matches_oracle_pipeline(env):
    """Minibatches of 2,048: each of the training cluster's CTAs takes two tiles
    of 128 samples per step (its gradient accumulates over both)."""
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(16, seed=21)
    kw = dict(train_frac=0.25, epochs=3, batch=2048, lr=3e-3, m_ctrl=60, **FIXED)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=150, window=40)
    _compare_pipeline(m, "tandem3", dps, 600, 9, dict(n_clients=150, window=40), kw,
                      oracle.host_threads())
    m.close()


def test_run_cv_forest_fire_matches_oracle_pipeline(env):
    eng, torch = env
    dps = mrip_inputs.ff_cv_design_points(4)
    kw = dict(train_frac=0.25, epochs=8, batch=32, lr=3e-3, m_ctrl=40, **FIXED)
    m = eng.Model(eng.MRIP_FOREST_FIRE, L=32, n_steps=200, density=0.5, window=40)
    _compare_pipeline(m, "forest_fire", dps, 24, 5, dict(L=32, n_steps=200, window=40), kw,
                      oracle.host_threads())
    m.close()


def test_run_cv_validation_gate_accepts_informative_window(env):
    """120 clients with a 100-client window: the early window explains about
    half of each replication's within-design-point variance (linear R^2
    0.55 by the oracle), well above the break-even rho^2 of 1 - n_held /
    (1.1 n_reps) = 0.27 when a fifth of the replications train the network;
    the control variate is kept, its control runs are sized from the
    validation rho^2 (m_ctrl = 0), and the oracle, given the GPU's network,
    finds the same rho^2 and count."""
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(12, seed=5)
    kw = dict(train_frac=0.2, val_frac=0.25, epochs=40, patience=5, batch=64, lr=3e-3,
              m_ctrl=0, gate=True)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=120, window=100)
    plain, cv, rep = _compare_pipeline(m, "tandem3", dps, 160, 3,
                                       dict(n_clients=120, window=100), kw,
                                       oracle.host_threads())
    assert not rep["declined"] and rep["var_ratio"] < 1.0, rep
    assert rep["n_val"] == math.ceil(0.25 * math.ceil(0.2 * 160))
    assert rep["m_ctrl"] == ocv.control_runs(rep["val_rho2"], 160 - math.ceil(0.2 * 160))
    assert 1 <= rep["best_epoch"] <= rep["epochs_run"] <= 40
    assert np.isfinite(rep["val_loss"])
    for k in ("ms_simulate", "ms_train", "ms_control", "ms_infer", "ms_estimate"):
        assert rep[k] > 0.0, k
    m.close()


def test_run_cv_gate_declines_uninformative_window(env):
    """2,000 clients and a 10-client window: the early window says almost
    nothing about the replication mean, so the validation rho^2 after the
    screen's 64 Adam steps is far below the break-even and the plain
    intervals are returned as the control-variate result, with no further
    training and no control runs."""
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(64, seed=6)
    kw = dict(train_frac=0.2, val_frac=0.25, epochs=10, patience=2, batch=32, lr=1e-3,
              m_ctrl=0, gate=True)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=2000, window=10)
    plain, cv, rep = m.run_cv(dps, 200, 8, **kw)
    assert rep["declined"] and rep["m_ctrl"] == 0 and rep["var_ratio"] >= 1.0
    # 64 x 30 fit samples in minibatches of 32 = 60 steps per epoch, so the
    # screen comes after 2 epochs; with 10 validation replications per design
    # point (576 degrees of freedom) its rho^2 is far below a quarter of the
    # break-even 1 - 160 / 220 = 0.27: declined there, no more training
    assert rep["declined"] == 2 and rep["epochs_run"] == 2
    assert rep["val_rho2"] < 0.25 * (1 - 160 / 220)
    for p, c in zip(plain, cv):
        assert c["mean"] == p["mean"] and c["half_width"] == p["half_width"] and c["m"] == 0
    assert rep["ms_control"] == 0.0 and rep["ms_infer"] == 0.0
    theta, _ = m.cv_network()
    _, _, info = ocv.run_cv("tandem3", dps, 200, 8, n_clients=2000, window=10,
                            theta=theta.astype(np.float64), threads=oracle.host_threads(), **kw)
    assert info["declined"]
    assert rep["val_rho2"] == pytest.approx(info["val_rho2"], abs=2e-3)
    m.close()


def test_cv_interval_coverage(env):
    """200 independent macro-replications (seeds) of a 2-design-point tandem
    study; the truth is the plain mean of 2^15 replications."""
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(2, seed=21)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=150, window=75)
    m.run(dps, 1 << 15, 999)
    truth = [s["mean"] for s in m.stats()]
    hits = np.zeros(2)
    trials = 200
    for k in range(trials):
        _, cv, _ = m.run_cv(dps, 64, 10_000 + k, train_frac=0.25, epochs=3, batch=32, lr=3e-3,
                            m_ctrl=640, **FIXED)
        for d in range(2):
            hits[d] += abs(cv[d]["mean"] - truth[d]) <= cv[d]["half_width"]
    rate = hits.sum() / (2 * trials)
    assert abs(rate - 0.95) < 3.3 * math.sqrt(0.95 * 0.05 / (2 * trials)), rate
    m.close()


def test_network_gain_when_the_window_is_informative(env):
    """Tandem with 150 clients and a 75-client window: the early window
    explains a large share of each replication's mean sojourn, and the
    control-variate half-width is well below the plain half-width of the same
    held-out replications."""
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(16, seed=5)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=150, window=75)
    plain, cv, rep = m.run_cv(dps, 256, 3, train_frac=0.25, epochs=40, batch=256, lr=3e-3,
                              m_ctrl=2000, **FIXED)
    n_held = cv[0]["n"]
    Y = m.outputs(0).reshape(16, 256)[:, 256 - n_held:]
    ratios = [c["half_width"] / ostats.ci(Y[d])["half_width"] for d, c in enumerate(cv)]
    assert np.median(ratios) < 0.9, ratios
    assert max(ratios) < 1.05, ratios
    m.close()
