"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the
benchmark.  Holds none of the method's arithmetic: point clouds and right-hand
sides only.

Recipes (the paper measures on synthetic point sets only; Sec. 5.1 uses a
sqrt(N) x sqrt(N) Chebyshev grid on [-1,1]^2):
  uniform(n, seed)          i.i.d. uniform points in [-1,1]^2
  jittered_grid(m, seed)    m x m grid of spacing h = 2/m, each point moved by
                            U(-h/4, h/4) per coordinate inside its own cell
  chebyshev_grid(m)         tensor grid of the m Chebyshev points cos((2i+1)pi/2m)
  rhs(n, nrhs, seed)        standard normal, n x nrhs
"""
from __future__ import annotations

import numpy as np


def uniform(n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, 2))


def jittered_grid(m: int, seed: int = 0) -> tuple[np.ndarray, float]:
    """Points of an m x m grid on [-1,1]^2 with spacing h = 2/m, centred in
    their cells and jittered by U(-h/4, h/4); returns (points, h)."""
    rng = np.random.default_rng(seed)
    h = 2.0 / m
    i = np.arange(m)
    gx, gy = np.meshgrid(i, i, indexing="xy")
    base = np.stack([-1.0 + h * (gx.ravel() + 0.5), -1.0 + h * (gy.ravel() + 0.5)], axis=1)
    return base + rng.uniform(-0.25 * h, 0.25 * h, base.shape), h


def chebyshev_grid(m: int) -> np.ndarray:
    c = np.cos((2.0 * np.arange(m) + 1.0) * np.pi / (2.0 * m))
    gx, gy = np.meshgrid(c, c, indexing="xy")
    return np.stack([gx.ravel(), gy.ravel()], axis=1)


def rhs(n: int, nrhs: int = 1, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, nrhs))
    return x[:, 0].copy() if nrhs == 1 else x


def point_sets(count: int, seed: int = 0, nmin: int = 2048, nmax: int = 65536):
    """Independent point sets of uneven size: n_i log-uniform in [nmin, nmax],
    each uniform in an axis-aligned rectangle with aspect ratio U(1, 4), long
    side 2, random orientation, centre U(-1,1)^2."""
    rng = np.random.default_rng(seed)
    sets = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        rho = rng.uniform(1.0, 4.0)
        long_x = rng.integers(0, 2) == 0
        c = rng.uniform(-1.0, 1.0, 2)
        wx, wy = (2.0, 2.0 / rho) if long_x else (2.0 / rho, 2.0)
        p = rng.uniform(-0.5, 0.5, (n, 2)) * np.array([wx, wy]) + c
        sets.append(p)
    return sets


def mlp_init(hidden: int = 64, seed: int = 0, nfeat: int = 8) -> np.ndarray:
    """He-normal initial parameters of the rank-predictor MLP as one flat
    float32 vector (W1, b1, W2, b2, w3, b3; biases zero)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((nfeat, hidden)) * np.sqrt(2.0 / nfeat)
    W2 = rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    w3 = rng.standard_normal(hidden) * np.sqrt(2.0 / hidden)
    return np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(hidden), w3,
                           [0.0]]).astype(np.float32)
