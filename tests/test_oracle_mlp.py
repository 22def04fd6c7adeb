"""Pins of the rank-predictor MLP oracle (no GPU): gradients against central
finite differences, a one-neuron network whose loss and gradient are written
out by hand, and the Adam step against its defining recursion on a scalar."""
import numpy as np
import pytest

from oracle import mlp
from paper_2204_05536_gb300 import inputs


def test_gradient_matches_finite_differences():
    H = 6
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(mlp.nparams(H)) * 0.5
    X = rng.standard_normal((11, 8))
    t = rng.standard_normal(11)
    loss, g = mlp.loss_and_grad(theta, X, t, H)
    h = 1e-6
    for i in rng.choice(len(theta), 60, replace=False):
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, t, H)[0] - mlp.loss_and_grad(theta - e, X, t, H)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_one_neuron_closed_form():
    # H = 1: y = w3 relu(x.W1 + b1) ... with W2 = 1, b2 = 0 and a positive path
    H = 1
    x = np.array([[1.0, 2.0, 0, 0, 0, 0, 0, -1.0]])
    W1 = np.array([0.5, 0.25, 0, 0, 0, 0, 0, 0.1])
    theta = np.concatenate([W1, [0.2], [1.0], [0.0], [3.0], [0.5]])
    t = np.array([1.0])
    z1 = 0.5 + 0.5 - 0.1 + 0.2       # 1.1
    y = 3.0 * z1 + 0.5                # 3.8
    loss, g = mlp.loss_and_grad(theta, x, t, H)
    assert loss == pytest.approx((y - 1.0) ** 2)
    dy = 2 * (y - 1.0)
    # dL/dw3 = dy * h2 = dy * z1; dL/db3 = dy; dL/dW1 = dy * w3 * W2 * x
    np.testing.assert_allclose(g[-2], dy * z1)
    np.testing.assert_allclose(g[-1], dy)
    np.testing.assert_allclose(g[:8], dy * 3.0 * 1.0 * x[0])


def test_adam_scalar_recursion():
    theta, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    g = np.array([0.5])
    th1, m1, v1 = mlp.adam_step(theta, g, m, v, 1, 0.1)
    # first step: mhat = g, vhat = g^2, so the move is lr * g / (|g| + eps)
    np.testing.assert_allclose(th1, 1.0 - 0.1 * 0.5 / (0.5 + 1e-8))
    assert m1[0] == pytest.approx(0.05) and v1[0] == pytest.approx(0.001 * 0.25)


def test_init_layout():
    th = inputs.mlp_init(64, seed=1)
    assert th.dtype == np.float32 and len(th) == mlp.nparams(64) == 4801
    W1, b1, W2, b2, w3, b3 = mlp.unpack(th)
    assert np.all(b1 == 0) and np.all(b2 == 0) and b3 == 0
