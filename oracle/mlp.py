"""Rank-predictor MLP, CPU oracle (numpy float64).  TEST INFRASTRUCTURE ONLY.

The network maps the 8 geometry features of an admissible block to
log2(rank + 1) of its ACA factorisation:
    h1 = relu(x W1 + b1)      W1: 8 x H,  b1: H
    h2 = relu(h1 W2 + b2)     W2: H x H,  b2: H
    y  = h2 . w3 + b3         w3: H,      b3: scalar
loss = (1/B) sum_i (y_i - t_i)^2.  Parameters travel as one flat vector in the
order W1 (row-major), b1, W2 (row-major), b2, w3, b3.

forward/backward are the plain chain rule, written out layer by layer.
"""
from __future__ import annotations

import numpy as np

NFEAT = 8


def nparams(hidden: int = 64) -> int:
    return NFEAT * hidden + hidden + hidden * hidden + hidden + hidden + 1


def unpack(theta, hidden: int = 64):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + NFEAT * hidden].reshape(NFEAT, hidden); o += NFEAT * hidden
    b1 = theta[o:o + hidden]; o += hidden
    W2 = theta[o:o + hidden * hidden].reshape(hidden, hidden); o += hidden * hidden
    b2 = theta[o:o + hidden]; o += hidden
    w3 = theta[o:o + hidden]; o += hidden
    b3 = theta[o]; o += 1
    assert o == nparams(hidden)
    return W1, b1, W2, b2, w3, b3


def forward(theta, X, hidden: int = 64):
    W1, b1, W2, b2, w3, b3 = unpack(theta, hidden)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, t, hidden: int = 64):
    """Mean squared error over the batch and its gradient (flat, same layout)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, hidden)
    y, (X, z1, h1, z2, h2) = forward(theta, X, hidden)
    t = np.asarray(t, dtype=np.float64)
    B = len(t)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B                    # dL/dy
    dw3 = h2.T @ dy
    db3 = dy.sum()
    dh2 = np.outer(dy, w3)
    dz2 = dh2 * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    dW1 = X.T @ dz1
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return loss, g


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2014); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
