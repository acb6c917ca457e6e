"""GPU parity of the tensor-core training kernel (mrip_mlp_train), step by step.

mrip_run_cv trains with this kernel (one cluster launch, tcgen05 MMAs), so
it is pinned here directly against the FP64 oracle (oracle/mlp.py), one Adam
step at a time.  The kernel is deterministic, so a run limited to j steps
(max_steps = j) gives the j-th point of the full trajectory; for every j:

* the gradient of step j (d_grad) equals the oracle's loss_and_grad at the
  GPU's own parameters after step j - 1, on the same minibatch (the oracle's
  epoch order) and the same BF16-rounded operands: norm-wise relative error
  <= 1e-3 for each parameter block (W1, b1, W2, b2, W3, b3) -- the bar of the
  SIMT stage test; the GPU accumulates in FP32, and an FP32-vs-FP64
  difference can flip a BF16 rounding of an activation;
* the minibatch loss within 1e-4 relative;
* Adam's moments and parameters after step j equal the Adam update (FP64,
  the same FP32 hyper-parameters) of the GPU's state after step j - 1 with
  the GPU's gradient, within a few FP32 ulps.

Sizes: minibatches of 64 (each CTA of the cluster a partial tile of 8),
1,024 (one tile per CTA) and 2,048 (two tiles per CTA), inputs of 6 and 8
features, a last partial minibatch and the first step of the next epoch.

Validation and early stopping: the per-epoch validation losses equal the
oracle's mean squared error at the GPU's parameters after that epoch, the
kept epoch and the stop follow from them by the rule (lowest loss kept,
stop after `patience` epochs without a lower one), and the returned
parameters equal, bit for bit, those of a run stopped after the kept epoch.
"""
import numpy as np
import pytest

import mrip_inputs
import oracle.mlp as omlp

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))  # noqa: E731  (the ABI takes FP32 hyper-parameters)
LR, B1, B2, EPS = 3e-3, 0.9, 0.999, 1e-8


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1501_01405_gb300 as eng
    eng.lib()
    return eng, torch


def _data(d_in, n, seed):
    X = omlp.f32(mrip_inputs.random_matrix((n, d_in), seed))
    # a smooth target of the inputs plus noise, so the gradient is not tiny
    y = omlp.f32(np.tanh(X[:, 0]) - 0.5 * X[:, 1] * X[:, -1] +
                 0.3 * mrip_inputs.random_matrix(n, seed + 1))
    theta0 = omlp.init_params(d_in, seed + 2)
    return X, y, theta0


def _run(eng, torch, d_in, X, y, theta0, batch, epochs, seed, max_steps, **kw):
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")  # noqa: E731
    P = omlp.n_params(d_in)
    th = dev(theta0)
    n = X.shape[0]
    steps = max_steps if max_steps > 0 else epochs * -(-n // batch)
    out = dict(grad=torch.zeros(P, dtype=torch.float32, device="cuda"),
               m=torch.zeros(P, dtype=torch.float32, device="cuda"),
               v=torch.zeros(P, dtype=torch.float32, device="cuda"),
               losses=torch.full((max(steps, 1),), np.nan, dtype=torch.float32, device="cuda"))
    xv = kw.pop("xv", None)
    yv = kw.pop("yv", None)
    if xv is not None:
        kw["xv"], kw["yv"] = dev(xv.T.copy()), dev(yv)
        out["val_losses"] = torch.full((epochs,), np.nan, dtype=torch.float32, device="cuda")
    info = eng.mrip_mlp_train(d_in, dev(X.T.copy()), dev(y), th, batch, epochs, seed, lr=LR,
                              beta1=B1, beta2=B2, eps=EPS, max_steps=max_steps, **kw, **out)
    res = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    res["theta"] = th.cpu().numpy().astype(np.float64)
    res["info"] = info
    return res


def _minibatch(n, batch, seed, step):
    """Sample indices of Adam step `step` (0-based): the oracle's epoch order."""
    spe = -(-n // batch)
    e, k = divmod(step, spe)
    order = omlp.batch_order(n, e, seed)
    return order[k * batch:min(k * batch + batch, n)]


@pytest.mark.parametrize("d_in,n,batch,steps", [
    (8, 3000, 1024, 4),   # one tile per CTA, a last minibatch of 952, then epoch 2
    (6, 3000, 2048, 3),   # two tiles per CTA, a last minibatch of 952, then epoch 2
    (8, 200, 64, 5),      # partial tiles of 8 per CTA, a last minibatch of 8, then epoch 2
    (6, 1100, 1024, 2),   # a last minibatch of 76: CTAs 7 and 8 get fewer rows or none
])
def test_training_steps_match_oracle(env, d_in, n, batch, steps):
    eng, torch = env
    seed = 31 + d_in
    X, y, theta0 = _data(d_in, n, seed)
    prev = dict(theta=theta0, m=np.zeros_like(theta0), v=np.zeros_like(theta0))
    for j in range(1, steps + 1):
        r = _run(eng, torch, d_in, X, y, theta0, batch, 3, seed, j)
        assert r["info"][2] == j
        idx = _minibatch(n, batch, seed, j - 1)
        ref_loss, ref_g = omlp.loss_and_grad(prev["theta"], X[idx], y[idx], d_in)
        g = r["grad"]
        for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), omlp.unpack(g, d_in),
                              omlp.unpack(ref_g, d_in)):
            err = np.linalg.norm(np.ravel(a) - np.ravel(b))
            assert err <= 1e-3 * np.linalg.norm(b) + 1e-7, (j, name, err, np.linalg.norm(b))
        assert r["losses"][j - 1] == pytest.approx(ref_loss, rel=1e-4)
        # Adam on the GPU's own state and gradient (FP64 reference of the FP32 arithmetic)
        rt, rm, rv = omlp.adam_step(prev["theta"], prev["m"], prev["v"], g, j, lr=F32(LR),
                                    beta1=F32(B1), beta2=F32(B2), eps=F32(EPS))
        scale_m = F32(B1) * np.abs(prev["m"]) + (1 - F32(B1)) * np.abs(g)
        scale_v = F32(B2) * prev["v"] + (1 - F32(B2)) * g * g
        assert np.all(np.abs(r["m"] - rm) <= 4 * 2.0**-24 * scale_m + 1e-30), j
        assert np.all(np.abs(r["v"] - rv) <= 4 * 2.0**-24 * scale_v + 1e-30), j
        np.testing.assert_allclose(r["theta"], rt, rtol=2.0**-22, atol=1e-9)
        prev = dict(theta=r["theta"], m=r["m"], v=r["v"])


def _expected_stop(val, epochs, patience):
    best, best_e, bad = np.inf, 0, 0
    for e in range(1, epochs + 1):
        v = val[e - 1]
        if v < best:
            best, best_e, bad = v, e, 0
        else:
            bad += 1
            if patience > 0 and bad >= patience:
                return e, best_e
    return epochs, best_e


@pytest.mark.parametrize("case", ["anti", "same"])
def test_validation_and_early_stop(env, case):
    """'anti': the validation target is the negated training target, so its
    loss grows once the network has learnt the training target and the run
    stops `patience` epochs after its lowest point; 'same': the validation
    set is drawn like the training set."""
    eng, torch = env
    d_in, n, batch, epochs, patience, seed = 8, 2500, 512, 10, 2, 77
    X, y, theta0 = _data(d_in, n, seed)
    Xv, yv, _ = _data(d_in, 700, seed + 100)
    if case == "anti":
        yv = -yv
    r = _run(eng, torch, d_in, X, y, theta0, batch, epochs, seed, 0, xv=Xv, yv=yv,
             patience=patience)
    epochs_run, best_epoch, steps = r["info"]
    val = r["val_losses"]
    assert np.isfinite(val[:epochs_run]).all() and np.isnan(val[epochs_run:]).all()
    assert (epochs_run, best_epoch) == _expected_stop(val, epochs, patience)
    spe = -(-n // batch)
    assert steps == epochs_run * spe
    if case == "anti":  # the stop fires well before the epoch budget
        assert epochs_run == best_epoch + patience and epochs_run < epochs
    # the kept parameters are the trajectory's after `best_epoch` epochs
    k = _run(eng, torch, d_in, X, y, theta0, batch, epochs, seed, best_epoch * spe)
    assert np.array_equal(r["theta"], k["theta"])
    # each epoch's validation loss is the oracle's MSE at that epoch's parameters
    for e in sorted({1, best_epoch, epochs_run}):
        th = _run(eng, torch, d_in, X, y, theta0, batch, epochs, seed, e * spe)["theta"]
        yhat, _ = omlp.forward(th, Xv, d_in)
        ref = float(np.mean((yhat - yv) ** 2))
        assert val[e - 1] == pytest.approx(ref, rel=1e-4), e


def test_resume_continues_the_trajectory(env):
    """One epoch, then the remaining epochs resumed from its parameters and
    Adam moments (epoch0 = 1), equals one run of all epochs bit for bit."""
    eng, torch = env
    d_in, n, batch, epochs, seed = 8, 2100, 512, 4, 12
    X, y, theta0 = _data(d_in, n, seed)
    full = _run(eng, torch, d_in, X, y, theta0, batch, epochs, seed, 0)
    first = _run(eng, torch, d_in, X, y, theta0, batch, 1, seed, 0)
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")  # noqa: E731
    rest = _run(eng, torch, d_in, X, y, first["theta"], batch, epochs - 1, seed, 0, epoch0=1,
                m_in=dev(first["m"]), v_in=dev(first["v"]))
    for k in ("theta", "m", "v"):
        assert np.array_equal(rest[k], full[k]), k
    spe = -(-n // batch)
    assert np.array_equal(np.concatenate([first["losses"], rest["losses"]]), full["losses"])
    assert rest["info"][2] == (epochs - 1) * spe
