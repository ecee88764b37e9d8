"""FP64 reference of the learned smoothing-length seed -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` may
use this module; it shares no code with the CUDA library.

The paper solves for h_i by Newton-Raphson on the constant kernel mass
(Sec. 2.3.3) and says nothing about where the iteration starts.  The learned
form adds a small network that proposes the start: it predicts a correction
to the continuity-equation estimate of the next h and is trained on the
smoothing lengths the Newton iteration itself converges to.  The paper has no
counterpart for the network; its definition here is:

features of particle i at the end of step n (dt = new step, dt_old = last):
    phi0 = dt * divv_i / 3            continuity estimate of ln(h_{n+1}/h_n)
    phi1 = nngb_i / N_ngb - 1         integer neighbour count against the target
    phi2 = ln(h_n / seed_n)           how far the last seed was off
    phi3 = ln(dt / dt_old)            step-size change (0 on the first step)
network input  x = (100 phi0, 4 phi1, 100 phi2, 10 phi3)
network        y = W3 . relu(W2 relu(W1 x + b1) + b2) + b3     (4 -> 32 -> 32 -> 1)
seed           h_seed = h_n * clamp(exp(phi0 + y / 100), 1/2, 2), with y taken
               as 0 where |phi0| and |phi2| are both below the Newton
               tolerance (the estimate is already converged there) or where
               |y| / 100 is below the dead zone sqrt(training loss) / 100
training target y* = 100 (ln(h_{n+1} / h_n) - phi0), loss = mean (y - y*)^2,
optimiser Adam (Kingma & Ba 2015) with bias correction.

Parameters are one flat vector of NPARAM floats in the order
W1 (32 x 4, row = hidden unit), b1 (32), W2 (32 x 32), b2 (32), W3 (32), b3 (1).

The inference path of the GPU rounds x, the weights and the hidden
activations to bfloat16 and accumulates in FP32; ``infer_bf16`` restates
that rounding (round to nearest even) with the sums taken in FP64.
"""
from __future__ import annotations

import numpy as np

NIN = 4
NHID = 32
NPARAM = NHID * NIN + NHID + NHID * NHID + NHID + NHID + 1   # 1249
X_SCALE = np.array([100.0, 4.0, 100.0, 10.0])
Y_SCALE = 100.0


def unpack(w):
    """Views (W1, b1, W2, b2, W3, b3) of a flat parameter vector."""
    w = np.asarray(w, dtype=np.float64)
    assert w.shape == (NPARAM,)
    o = 0
    W1 = w[o:o + NHID * NIN].reshape(NHID, NIN); o += NHID * NIN
    b1 = w[o:o + NHID]; o += NHID
    W2 = w[o:o + NHID * NHID].reshape(NHID, NHID); o += NHID * NHID
    b2 = w[o:o + NHID]; o += NHID
    W3 = w[o:o + NHID]; o += NHID
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2),
                           np.ravel(W3), np.atleast_1d(b3)]).astype(np.float64)


def features(dt, divv, nngb, n_ngb, h, seed, dt_old):
    """Network inputs x (N x 4) from the quantities defined above."""
    divv = np.asarray(divv, dtype=np.float64)
    phi0 = dt * divv / 3.0
    phi1 = np.asarray(nngb, dtype=np.float64) / n_ngb - 1.0
    phi2 = np.log(np.asarray(h, dtype=np.float64) / np.asarray(seed, dtype=np.float64))
    phi3 = np.full_like(phi0, np.log(dt / dt_old) if dt_old > 0 else 0.0)
    return np.stack([phi0, phi1, phi2, phi3], axis=1) * X_SCALE


def forward(w, X):
    """Network output y for inputs X (N x 4), FP64."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    a1 = np.maximum(X @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    return a2 @ W3 + b3


def loss_and_grad(w, X, y):
    """Mean squared error over the samples and its gradient (chain rule,
    layer by layer from the output back to the input)."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    out = a2 @ W3 + b3
    r = out - y
    loss = float(np.mean(r * r))
    d_out = 2.0 * r / n                       # dL/d out
    gW3 = a2.T @ d_out
    gb3 = d_out.sum()
    d_z2 = np.outer(d_out, W3) * (z2 > 0.0)   # dL/d z2
    gW2 = d_z2.T @ a1
    gb2 = d_z2.sum(axis=0)
    d_z1 = (d_z2 @ W2) * (z1 > 0.0)           # dL/d z1
    gW1 = d_z1.T @ X
    gb1 = d_z1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64.  Non-finite inputs are not expected here."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    out = (r << np.uint64(16)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def infer_bf16(w, X):
    """The GPU inference arithmetic: inputs, weights and both hidden layers'
    activations rounded to bfloat16, biases and sums kept wider."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    b1 = np.float32(b1).astype(np.float64)
    b2 = np.float32(b2).astype(np.float64)
    b3 = float(np.float32(b3))
    xb = bf16(X)
    a1 = bf16(np.float32(np.maximum(xb @ bf16(W1).T + b1, 0.0)))
    a2 = bf16(np.float32(np.maximum(a1 @ bf16(W2).T + b2, 0.0)))
    return a2 @ bf16(W3) + b3


def seed(h, X, y, tol=1e-6, dead=0.0):
    """h_seed from the previous h, the inputs X and the network output y
    (tol = the Newton tolerance on |dh|/h, dead = the dead zone in ln h)."""
    X = np.asarray(X)
    y = np.asarray(y, dtype=np.float64)
    phi0 = X[:, 0] / X_SCALE[0]
    rest = (np.abs(phi0) < tol) & (np.abs(X[:, 2] / X_SCALE[2]) < tol)
    y = np.where(rest | (np.abs(y / Y_SCALE) < dead), 0.0, y)
    f = np.exp(phi0 + y / Y_SCALE)
    return np.asarray(h) * np.clip(f, 0.5, 2.0)


def target(h_new, h, X):
    """Training target y* = 100 (ln(h_{n+1}/h_n) - phi0)."""
    phi0 = np.asarray(X)[:, 0] / X_SCALE[0]
    return Y_SCALE * (np.log(np.asarray(h_new) / np.asarray(h)) - phi0)


def train(w, X, y, iters, lr, batch=None, rng=None):
    """Plain Adam training loop (full batch unless `batch` is given)."""
    w = np.array(w, dtype=np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    losses = []
    for t in range(1, iters + 1):
        if batch is None:
            Xb, yb = X, y
        else:
            idx = rng.integers(0, len(y), size=batch)
            Xb, yb = X[idx], y[idx]
        loss, g = loss_and_grad(w, Xb, yb)
        losses.append(loss)
        w, m, v = adam_step(w, g, m, v, t, lr)
    return w, losses
