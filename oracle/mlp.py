"""Oracle for the learned control variate's network -- FP64, numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned component; this is the reading used by the engine:

* Network d_in -> 64 -> 64 -> 1, ReLU on both hidden layers, linear output.
* Parameters are FP32 masters.  Every matmul takes BF16 operands (round to
  nearest even from the FP32 value) and accumulates exactly here (FP64) where
  the GPU accumulates in FP32:
    forward  z1 = x~ W1~^T + b1, h1 = relu(z1)
             z2 = h1~ W2~^T + b2, h2 = relu(z2)
             yhat = h2~ . W3~ + b3
    backward dyhat = 2 (yhat - y) / B                    (loss = mean (yhat - y)^2)
             dW3 = sum_b dyhat h2~,  db3 = sum_b dyhat,  dh2 = dyhat W3~
             dz2 = dh2 * [z2 > 0]
             dW2 = dz2~^T h1~,  db2 = sum_b dz2,  dh1 = dz2~ W2~
             dz1 = dh1 * [z1 > 0]
             dW1 = dz1~^T x~,   db1 = sum_b dz1
  where ~ is the BF16 rounding; the rounding is treated as the identity in
  the gradient (straight-through).
* Inputs and target are standardised with the training set's FP64 mean and
  population standard deviation (a zero deviation is replaced by 1); the
  standardised value is rounded to FP32 before its BF16 rounding.
* Initialisation (stream tag 3): weight element e of the concatenation
  W1, W2, W3 (row-major) reads words (2(e mod 2), 2(e mod 2)+1) of block
  (c0 = e div 2, c1 = 0, rep 0, dp 0); w = (2u - 1) sqrt(6 / fan_in), rounded
  to FP32; biases start at 0.
* Minibatch order (stream tag 4): epoch e reads block (c0 = 0, c1 = e,
  rep 0, dp 0) -> (w0, w1); a = 1 + w0 mod (n - 1) stepped up to the first
  value coprime with n, b = w1 mod n; sample i of the epoch is
  pi(i) = (a i + b) mod n and minibatch k is pi(kB), ..., pi(min(kB+B, n)-1).
* Adam (Kingma & Ba, 2015) with bias correction, step count from 1.
"""
import math

import numpy as np

from . import stream_block

HIDDEN = 64
TAG_INIT = 3
TAG_ORDER = 4


def bf16(x):
    """Round to BF16 (nearest even) via FP32; returned as float64 values."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def n_params(d_in):
    return HIDDEN * d_in + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def unpack(theta, d_in):
    """Views (W1, b1, W2, b2, W3, b3) into the flat parameter vector."""
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + HIDDEN * d_in].reshape(HIDDEN, d_in); o += HIDDEN * d_in
    b1 = theta[o:o + HIDDEN]; o += HIDDEN
    W2 = theta[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = theta[o:o + HIDDEN]; o += HIDDEN
    W3 = theta[o:o + HIDDEN]; o += HIDDEN
    b3 = theta[o:o + 1]; o += 1
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2),
                           np.ravel(W3), np.ravel(b3)]).astype(np.float64)


def init_params(d_in, seed):
    """He-uniform weights from stream tag 3, zero biases; FP32 values."""
    fans = [(HIDDEN * d_in, d_in), (HIDDEN * HIDDEN, HIDDEN), (HIDDEN, HIDDEN)]
    n_w = sum(c for c, _ in fans)
    e = np.arange(n_w, dtype=np.uint64)
    blocks = stream_block(seed, TAG_INIT, 0, 0, np.zeros(n_w // 2 + 1, np.uint64),
                          np.arange(n_w // 2 + 1, dtype=np.uint64))
    from . import u53_expo
    par = (e % 2).astype(np.int64)
    blk = blocks[(e // 2).astype(np.int64)]
    lo = blk[np.arange(n_w), 2 * par]
    hi = blk[np.arange(n_w), 2 * par + 1]
    u, _ = u53_expo(lo, hi, 1.0)
    scale = np.concatenate([np.full(c, math.sqrt(6.0 / fan)) for c, fan in fans])
    w = f32((2.0 * u - 1.0) * scale)
    o1 = HIDDEN * d_in
    o2 = o1 + HIDDEN * HIDDEN
    return pack(w[:o1], np.zeros(HIDDEN), w[o1:o2], np.zeros(HIDDEN), w[o2:], np.zeros(1))


def batch_order(n, epoch, seed):
    """Sample order of one epoch: pi(i) = (a i + b) mod n."""
    if n <= 1:
        return np.zeros(max(n, 0), dtype=np.int64)
    blk = stream_block(seed, TAG_ORDER, 0, 0, [epoch], [0])[0]
    a = 1 + int(blk[0]) % (n - 1)
    while math.gcd(a, n) != 1:
        a += 1
        if a >= n:
            a = 1
    b = int(blk[1]) % n
    i = np.arange(n, dtype=np.int64)
    return (a * i + b) % n


def standardizer(X):
    """(mean, std) per column, FP64, population std, zero std -> 1."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    n = X.shape[0]
    mean = np.array([math.fsum(X[:, j].tolist()) / n for j in range(X.shape[1])])
    var = np.array([math.fsum(((X[:, j] - mean[j]) ** 2).tolist()) / n
                    for j in range(X.shape[1])])
    std = np.sqrt(var)
    std[std == 0.0] = 1.0
    return mean, std


def apply_std(X, mean, std):
    """Standardised value rounded to FP32 (the network's input precision)."""
    return f32((np.asarray(X, dtype=np.float64) - mean) / std)


def _identity(x):
    return np.asarray(x, dtype=np.float64)


def forward(theta, X, d_in, rounding=True):
    """Forward pass; returns (yhat, cache).  rounding=False drops every BF16
    and FP32 rounding (the exact-arithmetic network, used to pin the
    formulas against autograd and finite differences)."""
    rb = bf16 if rounding else _identity
    rf = f32 if rounding else _identity
    W1, b1, W2, b2, W3, b3 = unpack(theta, d_in)
    x = rb(X)
    z1 = x @ rb(W1).T + rf(b1)
    h1 = np.maximum(z1, 0.0)
    h1t = rb(h1)
    z2 = h1t @ rb(W2).T + rf(b2)
    h2 = np.maximum(z2, 0.0)
    h2t = rb(h2)
    yhat = h2t @ rb(W3) + rf(b3)[0]
    return yhat, (x, z1, h1t, z2, h2t)


def loss_and_grad(theta, X, y, d_in, rounding=True):
    """Mean squared error of a minibatch and its gradient (flat vector)."""
    rb = bf16 if rounding else _identity
    W1, b1, W2, b2, W3, b3 = unpack(theta, d_in)
    B = X.shape[0]
    yhat, (x, z1, h1t, z2, h2t) = forward(theta, X, d_in, rounding)
    r = yhat - np.asarray(y, dtype=np.float64)
    loss = math.fsum((r * r).tolist()) / B
    dy = 2.0 * r / B
    dW3 = dy @ h2t
    db3 = np.array([math.fsum(dy.tolist())])
    dh2 = np.outer(dy, rb(W3))
    dz2 = dh2 * (z2 > 0.0)
    dz2t = rb(dz2)
    dW2 = dz2t.T @ h1t
    db2 = dz2.sum(axis=0)
    dh1 = dz2t @ rb(W2)
    dz1 = dh1 * (z1 > 0.0)
    dz1t = rb(dz1)
    dW1 = dz1t.T @ x
    db1 = dz1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def train(X, y, d_in, seed, epochs, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999,
          eps=1e-8, master_fp32=True, X_val=None, y_val=None, patience=0, after_epoch=None):
    """Full training run in FP64 (masters rounded to FP32 after each step when
    master_fp32).  With a validation set (X_val, y_val; standardised with the
    training set's moments) the mean squared error over it is taken after
    every epoch; the parameters of the epoch with the lowest value are kept,
    and training stops after `patience` epochs without a lower value
    (0: never).  after_epoch(e, theta, norm), called after epoch e (1-based)
    with the parameters kept so far, may return True to stop.  Returns
    (theta, (x_mean, x_std, y_mean, y_std), losses, info) with
    info = {val_losses, epochs_run, best_epoch, stopped_by_callback}."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    xm, xs = standardizer(X)
    ym, ys = standardizer(y)
    Xs = apply_std(X, xm, xs)
    ysd = apply_std(y[:, None], ym, ys)[:, 0]
    have_val = X_val is not None and len(X_val) > 0
    if have_val:
        Xv = apply_std(np.asarray(X_val, dtype=np.float64), xm, xs)
        yv = apply_std(np.asarray(y_val, dtype=np.float64).reshape(-1, 1), ym, ys)[:, 0]
    theta = init_params(d_in, seed)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    n = X.shape[0]
    t = 0
    losses, val_losses = [], []
    best, best_theta, best_epoch, bad, epochs_run = math.inf, theta, 0, 0, 0
    stopped = False
    norm = (xm, xs, ym[0], ys[0])
    for e in range(epochs):
        order = batch_order(n, e, seed)
        for k in range(0, n, batch):
            idx = order[k:k + batch]
            loss, g = loss_and_grad(theta, Xs[idx], ysd[idx], d_in)
            t += 1
            theta, m, v = adam_step(theta, m, v, g, t, lr, beta1, beta2, eps)
            if master_fp32:
                theta = f32(theta)
            losses.append(loss)
        epochs_run = e + 1
        if have_val:
            yhat, _ = forward(theta, Xv, d_in)
            vl = math.fsum(((yhat - yv) ** 2).tolist()) / len(yv)
            val_losses.append(vl)
            if vl < best:
                best, best_theta, best_epoch, bad = vl, theta, e + 1, 0
            else:
                bad += 1
                if patience > 0 and bad >= patience:
                    break
        if after_epoch is not None and after_epoch(e + 1, best_theta if have_val else theta, norm):
            stopped = True
            break
    if have_val:
        theta = best_theta
    else:
        best_epoch = epochs_run
    info = dict(val_losses=np.array(val_losses), epochs_run=epochs_run, best_epoch=best_epoch,
                stopped_by_callback=stopped)
    return theta, norm, np.array(losses), info


def predict(theta, X, norm, d_in):
    """Network output (standardised units) for raw features X."""
    xm, xs = norm[0], norm[1]
    yhat, _ = forward(theta, apply_std(X, xm, xs), d_in)
    return yhat
