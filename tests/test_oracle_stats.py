"""Pins for the oracle's statistics, Student-t critical value, network and
control-variate estimator (CPU only).

* t critical values: closed forms for 1, 2 and 4 degrees of freedom, the
  normal limit with its first Cornish-Fisher correction, scipy's independent
  implementation, a CDF round trip, and (when mpmath is importable) a
  40-digit evaluation of the incomplete beta function.
* Two-pass moments: exact values for arithmetic sequences; interval
  coverage on seeded normal samples (paper, Section 1: the CLT interval).
* Network: with the roundings switched off, the analytic gradient equals
  PyTorch autograd and central finite differences; the BF16 rounding equals
  PyTorch's; Adam equals torch.optim.Adam; initialisation bounds and
  moments; the epoch order is a permutation.
* Control variate: perfect and useless controls, invariance under affine
  maps of the control, and interval coverage on seeded correlated pairs.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import mrip_inputs
import oracle
import oracle.cv as ocv
import oracle.mlp as omlp
import oracle.stats as ostats


# ---------------------------------------------------------------- Student t
@pytest.mark.parametrize("conf", [0.9, 0.95, 0.99])
def test_t_closed_forms(conf):
    p = 1.0 - (1.0 - conf) / 2.0
    assert oracle.t_crit(conf, 1) == pytest.approx(math.tan(math.pi * (p - 0.5)), rel=1e-13)
    assert oracle.t_crit(conf, 2) == pytest.approx((2 * p - 1) / math.sqrt(2 * p * (1 - p)),
                                                   rel=1e-14)
    a = 4 * p * (1 - p)
    q = math.cos(math.acos(math.sqrt(a)) / 3.0) / math.sqrt(a)
    assert oracle.t_crit(conf, 4) == pytest.approx(2 * math.sqrt(q - 1), rel=1e-13)


def test_t_normal_limit():
    z = special.ndtri(0.975)
    for nu in (10**5, 2**17 - 1, 10**6):
        # Cornish-Fisher: t = z + (z^3 + z) / (4 nu) + O(nu^-2)
        approx = z + (z**3 + z) / (4 * nu)
        assert abs(oracle.t_crit(0.95, nu) - approx) < 10.0 / nu**2


@pytest.mark.parametrize("nu", [3, 5, 9, 29, 31, 127, 229, 254, 255, 1023, 2**17 - 1])
def test_t_matches_scipy_and_round_trips(nu):
    t = oracle.t_crit(0.95, nu)
    assert t == pytest.approx(stats.t.ppf(0.975, nu), rel=1e-13)
    assert oracle.t_cdf(t, nu) == pytest.approx(0.975, abs=1e-15)
    assert oracle.t_cdf(-t, nu) == pytest.approx(0.025, rel=1e-13)


def test_t_high_precision_reference():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for nu in (7, 256, 2**17 - 1):
        x = mp.mpf(nu) / (nu + mp.mpf(oracle.t_crit(0.95, nu)) ** 2)
        tail = mp.betainc(mp.mpf(nu) / 2, mp.mpf(1) / 2, 0, x, regularized=True) / 2
        # the tail at the oracle's t is (1-conf)/2 to within its slope x ulp(t)
        assert abs(float(tail) - (1 - 0.95) / 2) < 1e-16


# ---------------------------------------------------------------- moments
def test_two_pass_moments_exact():
    for n in (2, 3, 32, 1000):
        x = np.arange(1, n + 1, dtype=np.float64)
        k, mean, var = ostats.dp_stats(x)
        assert k == n and mean == (n + 1) / 2 and var == pytest.approx(n * (n + 1) / 12,
                                                                        rel=1e-15)
    k, mean, var = ostats.dp_stats([3.5])
    assert k == 1 and mean == 3.5 and math.isnan(var)
    # a large mean and a small spread: exact rational arithmetic decides (the
    # deviations from the rounded mean alone would miss by up to ~1e-10 here)
    from fractions import Fraction
    rng = np.random.default_rng(5)
    for loc in (1e9, -3e12):
        x = loc + 1e-2 * rng.standard_normal(777)
        fx = [Fraction(v) for v in x.tolist()]
        em = sum(fx) / len(fx)
        ev = sum((v - em) ** 2 for v in fx) / (len(fx) - 1)
        k, mean, var = ostats.dp_stats(x)
        assert mean == float(em)
        assert var == pytest.approx(float(ev), rel=1e-13)
    c = ostats.ci([1.0, 1.0, 1.0])
    assert c["half_width"] == 0.0 and c["mean"] == 1.0


def test_ci_coverage_normal_samples():
    rng = np.random.default_rng(12)
    trials, n = 2000, 10
    hits = 0
    for _ in range(trials):
        x = 3.0 + 2.0 * rng.standard_normal(n)
        c = ostats.ci(x, 0.95)
        hits += abs(c["mean"] - 3.0) <= c["half_width"]
    # binomial 99.9% band around 0.95
    assert abs(hits / trials - 0.95) < 3.3 * math.sqrt(0.95 * 0.05 / trials)


# ---------------------------------------------------------------- network
def _torch():
    return pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    torch = _torch()
    x = np.concatenate([mrip_inputs.random_matrix(20000, 1, scale=3.0),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1e-30, 3.0e38]])
    ref = torch.tensor(x, dtype=torch.float64).float().bfloat16().double().numpy()
    assert np.array_equal(omlp.bf16(x), ref)


@pytest.mark.parametrize("d_in", [6, 8])
def test_gradient_matches_autograd_without_rounding(d_in):
    torch = _torch()
    B = 37
    theta = omlp.init_params(d_in, 5) + mrip_inputs.random_matrix(omlp.n_params(d_in), 2, 0.05)
    X = mrip_inputs.random_matrix((B, d_in), 3)
    y = mrip_inputs.random_matrix(B, 4)
    loss, g = omlp.loss_and_grad(theta, X, y, d_in, rounding=False)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(np.arange(theta.size), d_in)
    Xt = torch.tensor(X)

    def sl(ix):
        ix = np.asarray(ix)
        return th[int(ix.min()):int(ix.max()) + 1].reshape(ix.shape)
    h1 = torch.relu(Xt @ sl(W1).T + sl(b1))
    h2 = torch.relu(h1 @ sl(W2).T + sl(b2))
    yh = h2 @ sl(W3) + sl(b3)[0]
    lt = ((yh - torch.tensor(y)) ** 2).mean()
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    np.testing.assert_allclose(g, th.grad.numpy(), rtol=1e-10, atol=1e-13)


def test_gradient_matches_finite_differences():
    d_in, B = 8, 16
    theta = omlp.init_params(d_in, 9) + mrip_inputs.random_matrix(omlp.n_params(d_in), 8, 0.05)
    X = mrip_inputs.random_matrix((B, d_in), 10)
    y = mrip_inputs.random_matrix(B, 11)
    _, g = omlp.loss_and_grad(theta, X, y, d_in, rounding=False)
    rng = np.random.default_rng(0)
    for j in rng.choice(theta.size, 60, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        lp, _ = omlp.loss_and_grad(tp, X, y, d_in, rounding=False)
        lm, _ = omlp.loss_and_grad(tm, X, y, d_in, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[j], rel=1e-6, abs=1e-9)


def test_rounded_gradient_close_to_exact():
    d_in, B = 8, 256
    theta = omlp.init_params(d_in, 1)
    X = mrip_inputs.random_matrix((B, d_in), 2)
    y = mrip_inputs.random_matrix(B, 3)
    _, g0 = omlp.loss_and_grad(theta, X, y, d_in, rounding=False)
    _, g1 = omlp.loss_and_grad(theta, X, y, d_in, rounding=True)
    assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) < 2e-2
    assert not np.array_equal(g0, g1)


def test_adam_matches_torch():
    torch = _torch()
    n = 500
    theta = mrip_inputs.random_matrix(n, 1)
    m = np.zeros(n)
    v = np.zeros(n)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = mrip_inputs.random_matrix(n, 100 + t)
        theta, m, v = omlp.adam_step(theta, m, v, g, t)
        p.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_init_bounds_and_moments():
    theta = omlp.init_params(8, 42)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(theta, 8)
    assert np.all(b1 == 0) and np.all(b2 == 0) and b3[0] == 0
    for W, fan in ((W1, 8), (W2, 64), (W3, 64)):
        a = math.sqrt(6.0 / fan)
        assert np.all(np.abs(W) <= a * (1 + 1e-7))
        assert abs(W.mean()) < 5 * a / math.sqrt(3 * W.size)
    assert W2.var() == pytest.approx(2.0 / 64, rel=0.1)
    assert np.array_equal(theta, omlp.f32(theta))
    assert not np.array_equal(theta, omlp.init_params(8, 43))


@pytest.mark.parametrize("n", [1, 2, 7, 832, 1024, 106496])
def test_batch_order_is_a_permutation(n):
    o0 = omlp.batch_order(n, 0, 42)
    assert np.array_equal(np.sort(o0), np.arange(n))
    if n > 3:
        assert not np.array_equal(o0, omlp.batch_order(n, 1, 42))


def test_training_learns_a_smooth_function():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(2048, 8))
    y = 2.0 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2] ** 2 + 3.0
    theta, norm, losses, _ = omlp.train(X, y, 8, 42, epochs=15, batch=256, lr=3e-3)
    assert losses[-1] < 0.05 * losses[0]
    pred = omlp.predict(theta, X, norm, 8) * norm[3] + norm[2]
    assert np.sqrt(np.mean((pred - y) ** 2)) < 0.2 * y.std()


# ---------------------------------------------------------------- CV
def test_cv_perfect_and_useless_controls():
    y, g = mrip_inputs.correlated_pair(200, 0.5, 1)
    gc = mrip_inputs.random_matrix(1000, 2, scale=0.5, loc=1.0)
    r = ocv.cv_estimate(y, y, gc[:6], 0.95)  # the control is Y itself
    assert r["beta"] == pytest.approx(1.0, rel=1e-12)
    assert r["mean"] == pytest.approx(np.mean(gc[:6]), rel=1e-12)
    const = ocv.cv_estimate(y, np.full(200, 2.0), gc)
    assert const["beta"] == 0.0 and const["mean"] == pytest.approx(np.mean(y), rel=1e-14)


def test_cv_affine_invariance():
    y, g = mrip_inputs.correlated_pair(300, 0.8, 3)
    gc = mrip_inputs.correlated_pair(3000, 0.8, 4)[1]
    a = ocv.cv_estimate(y, g, gc)
    b = ocv.cv_estimate(y, -3.0 * g + 7.0, -3.0 * gc + 7.0)
    for k in ("mean", "half_width", "var"):
        assert a[k] == pytest.approx(b[k], rel=1e-10)


def test_cv_coverage_and_variance_reduction():
    trials, n, M, rho = 1000, 50, 500, 0.9
    hits_cv = hits_plain = 0
    ratio = []
    for s in range(trials):
        y, g = mrip_inputs.correlated_pair(n, rho, 1000 + s)
        _, gc = mrip_inputs.correlated_pair(M, rho, 500000 + s)
        r = ocv.cv_estimate(y, g, gc, 0.95)
        p = ostats.ci(y, 0.95)
        hits_cv += abs(r["mean"] - 5.0) <= r["half_width"]
        hits_plain += abs(p["mean"] - 5.0) <= p["half_width"]
        ratio.append(r["half_width"] / p["half_width"])
    band = 3.3 * math.sqrt(0.95 * 0.05 / trials)
    assert abs(hits_cv / trials - 0.95) < band
    assert abs(hits_plain / trials - 0.95) < band
    # half-width ratio -> sqrt(1 - rho^2 + rho^2 n / M)
    expect = math.sqrt(1 - rho**2 + rho**2 * n / M)
    assert np.median(ratio) == pytest.approx(expect, rel=0.1)


def test_training_early_stop_rule():
    """With a validation set the kept parameters are those after the epoch of
    lowest validation loss -- the same as a run stopped there -- and training
    ends `patience` epochs later; the validation loss is the mean squared
    error of the standardised target, computed independently here."""
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, size=(600, 6))
    y = np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2]
    Xv = rng.uniform(-1, 1, size=(200, 6))
    yv = -(np.sin(3 * Xv[:, 0]) + Xv[:, 1] * Xv[:, 2])  # anti-correlated target
    theta, norm, losses, info = omlp.train(X, y, 6, 11, epochs=12, batch=128, lr=3e-3,
                                           X_val=Xv, y_val=yv, patience=2)
    vl, best, run = info["val_losses"], info["best_epoch"], info["epochs_run"]
    assert len(vl) == run and len(losses) == run * 5
    assert best == int(np.argmin(vl)) + 1 and run == best + 2 and run < 12
    assert all(vl[k] >= vl[best - 1] for k in range(best, run))
    ref, _, _, _ = omlp.train(X, y, 6, 11, epochs=best, batch=128, lr=3e-3)
    assert np.array_equal(theta, ref)
    pred = omlp.predict(theta, Xv, norm, 6)
    ystd = (yv - norm[2]) / norm[3]
    assert vl[best - 1] == pytest.approx(np.mean((pred - ystd) ** 2), rel=1e-6)


def test_within_rho2_known_correlation_and_offsets():
    """Pooled within-design-point rho^2: design-point offsets do not enter;
    an exact affine control gives 1, an independent one about 0, and a
    bivariate normal with correlation rho about rho^2."""
    rng = np.random.default_rng(4)
    n_dp, n = 400, 6
    y = rng.standard_normal((n_dp, n))
    g = 0.6 * y + 0.8 * rng.standard_normal((n_dp, n))
    off_y = rng.uniform(-50, 50, size=(n_dp, 1))
    off_g = rng.uniform(-50, 50, size=(n_dp, 1))
    r = ocv.within_rho2(y, g)
    assert r == pytest.approx(ocv.within_rho2(y + off_y, g + off_g), rel=1e-9)
    # sampling error of a pooled correlation on 400 x 5 degrees of freedom
    assert abs(math.sqrt(r) - 0.6) < 4 * (1 - 0.36) / math.sqrt(n_dp * (n - 1))
    assert ocv.within_rho2(y, -2.0 * y + off_g) == pytest.approx(1.0, rel=1e-12)
    assert ocv.within_rho2(y, rng.standard_normal((n_dp, n))) < 0.01
    # a single replication per design point carries no within information
    assert ocv.within_rho2(y[:, :1], g[:, :1]) == 0.0


def test_within_rho2_equal_weights_with_fit_scales():
    """Design points of very different variance: half have a correlated
    control (rho 0.9) and a scale 100 times the others', half an
    uncorrelated one.  Unscaled pooling is dominated by the large ones
    (rho^2 ~ 0.81); scaled by each design point's fit-set deviations every
    design point weighs the same and the estimate is the squared mean
    correlation, (0.9 / 2)^2 ~ 0.2."""
    rng = np.random.default_rng(12)
    n_dp, n_val, n_fit = 600, 4, 40

    def draw(n):
        z1 = rng.standard_normal((n_dp, n))
        z2 = rng.standard_normal((n_dp, n))
        rho = np.where(np.arange(n_dp) % 2 == 0, 0.9, 0.0)[:, None]
        scale = np.where(np.arange(n_dp) % 2 == 0, 100.0, 1.0)[:, None]
        return scale * z1, scale * (rho * z1 + np.sqrt(1 - rho**2) * z2)
    yv, gv = draw(n_val)
    yf, gf = draw(n_fit)
    assert ocv.within_rho2(yv, gv) == pytest.approx(0.81, abs=0.05)
    assert ocv.within_rho2(yv, gv, yf, gf) == pytest.approx(0.45**2, abs=0.05)
    # a constant fit output leaves its design point out
    gf0 = gf.copy()
    gf0[1::2] = 3.0
    assert ocv.within_rho2(yv, gv, yf, gf0) == pytest.approx(0.81, abs=0.05)


def test_control_run_sizing_and_gate():
    # M keeps beta^2 Var(g')/M <= 0.1 (1 - rho^2) s^2 / n: closed values
    assert ocv.control_runs(None, 230) == 2300
    assert ocv.control_runs(0.0, 230) == 2
    assert ocv.control_runs(0.5, 230) == 2300
    assert ocv.control_runs(0.02, 230) == math.ceil(230 * 0.02 / (0.1 * 0.98))
    assert ocv.control_runs(0.9999999, 230) == 23000
    for rho2 in (0.05, 0.3, 0.8):
        M = ocv.control_runs(rho2, 230)
        assert rho2 / M <= 0.1 * (1 - rho2) / 230 * (1 + 1e-12)
    # the gate: no correlation -> training replications are pure loss
    assert ocv.var_ratio(0.0, 256, 230, 2) == pytest.approx(256 / 230)
    # break-even rho^2 with M sized as above: (1 + 0.1) (1 - rho^2) n_reps / n_held = 1
    rho_be = 1 - 230 / (256 * 1.1)
    assert ocv.var_ratio(rho_be + 0.01, 256, 230, ocv.control_runs(rho_be + 0.01, 230)) < 1.0
    assert ocv.var_ratio(rho_be - 0.01, 256, 230, ocv.control_runs(rho_be - 0.01, 230)) > 1.0


def test_training_callback_stops_after_the_requested_epoch():
    """The screen's hook: a callback that asks to stop after epoch 2 ends
    training there; the parameters are those of a 2-epoch run, the callback
    saw epochs 1 and 2 with the parameters then kept, and the standardisation
    it was given is the run's."""
    rng = np.random.default_rng(13)
    X = rng.uniform(-1, 1, size=(500, 8))
    y = X[:, 0] - 2 * X[:, 3] + 0.1 * rng.standard_normal(500)
    seen = []

    def cb(e, th, norm):
        seen.append((e, th.copy(), norm))
        return e == 2
    theta, norm, losses, info = omlp.train(X, y, 8, 5, epochs=9, batch=100, lr=3e-3,
                                           after_epoch=cb)
    assert info["stopped_by_callback"] and info["epochs_run"] == 2 and len(losses) == 10
    assert [s[0] for s in seen] == [1, 2]
    ref, _, _, _ = omlp.train(X, y, 8, 5, epochs=2, batch=100, lr=3e-3)
    assert np.array_equal(theta, ref) and np.array_equal(seen[1][1], ref)
    one, _, _, _ = omlp.train(X, y, 8, 5, epochs=1, batch=100, lr=3e-3)
    assert np.array_equal(seen[0][1], one)
    assert all(np.array_equal(a, b) for a, b in zip(seen[0][2][:2], norm[:2]))
