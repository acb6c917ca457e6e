"""GPU parity of the learned control variate: network stages and estimator.

* initialisation bit-exact (FP32) against the oracle;
* forward pass and minibatch gradient against the FP64 oracle evaluated on
  the same BF16-rounded operands (norm-wise relative error <= 1e-3; the GPU
  accumulates in FP32, and an FP32-vs-FP64 difference can flip a BF16
  rounding of an activation);
* one Adam step (FP32 vs FP64, 1e-5);
* the per-design-point estimator on seeded arrays (FP64, 1e-12);
* the whole mrip_run_cv pipeline against the oracle pipeline on small
  tandem and forest-fire workloads: plain intervals 1e-12, training loss
  within 5 %, control-variate means within their combined half-widths;
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


def _compare_pipeline(plain, cv, loss, ref_plain, ref_cv, ref_loss):
    for g, r in zip(plain, ref_plain):
        assert g["mean"] == pytest.approx(r["mean"], rel=1e-12)
        assert g["half_width"] == pytest.approx(r["half_width"], rel=1e-12)
    assert loss == pytest.approx(ref_loss, rel=0.05)
    for g, r in zip(cv, ref_cv):
        assert g["n"] == r["n"] and g["m"] == r["m"]
        assert abs(g["mean"] - r["mean"]) <= g["half_width"] + r["half_width"]
        assert g["half_width"] == pytest.approx(r["half_width"], rel=0.25)


def test_run_cv_tandem_matches_oracle_pipeline(env):
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(8, seed=3)
    kw = dict(train_frac=0.25, epochs=6, batch=64, lr=3e-3, m_ctrl=300)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=200, window=50)
    plain, cv, loss = m.run_cv(dps, 48, 7, **kw)
    ref_plain, ref_cv, ref_loss = ocv.run_cv("tandem3", dps, 48, 7, n_clients=200, window=50,
                                             threads=oracle.host_threads(), **kw)
    _compare_pipeline(plain, cv, loss, ref_plain, ref_cv, ref_loss)
    m.close()


def test_run_cv_large_minibatch_matches_oracle_pipeline(env):
    """Minibatches of 2,048: each of the training cluster's CTAs takes two tiles
    of 128 samples per step (its gradient accumulates over both)."""
    eng, torch = env
    dps = mrip_inputs.tandem_design_points(16, seed=21)
    kw = dict(train_frac=0.25, epochs=3, batch=2048, lr=3e-3, m_ctrl=60)
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=150, window=40)
    plain, cv, loss = m.run_cv(dps, 600, 9, **kw)
    ref_plain, ref_cv, ref_loss = ocv.run_cv("tandem3", dps, 600, 9, n_clients=150, window=40,
                                             threads=oracle.host_threads(), **kw)
    _compare_pipeline(plain, cv, loss, ref_plain, ref_cv, ref_loss)
    m.close()


def test_run_cv_forest_fire_matches_oracle_pipeline(env):
    eng, torch = env
    dps = mrip_inputs.ff_cv_design_points(4)
    kw = dict(train_frac=0.25, epochs=8, batch=32, lr=3e-3, m_ctrl=40)
    m = eng.Model(eng.MRIP_FOREST_FIRE, L=32, n_steps=200, density=0.5, window=40)
    plain, cv, loss = m.run_cv(dps, 24, 5, **kw)
    ref_plain, ref_cv, ref_loss = ocv.run_cv("forest_fire", dps, 24, 5, L=32, n_steps=200,
                                             window=40, threads=oracle.host_threads(), **kw)
    _compare_pipeline(plain, cv, loss, ref_plain, ref_cv, ref_loss)
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
                            m_ctrl=640)
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
    plain, cv, loss = m.run_cv(dps, 256, 3, train_frac=0.25, epochs=40, batch=256, lr=3e-3,
                               m_ctrl=2000)
    n_held = cv[0]["n"]
    Y = m.outputs(0).reshape(16, 256)[:, 256 - n_held:]
    ratios = [c["half_width"] / ostats.ci(Y[d])["half_width"] for d, c in enumerate(cv)]
    assert np.median(ratios) < 0.9, ratios
    assert max(ratios) < 1.05, ratios
    m.close()
