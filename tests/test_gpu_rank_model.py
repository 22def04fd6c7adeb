"""Learned rank predictor (GPU) against its CPU oracle (oracle/mlp.py), and
what it gains inside the build.

  - forward predictions and the loss gradient of the GPU kernels equal the
    float64 oracle's to binary32 accuracy, on random parameters and data;
  - one Adam step of the GPU trainer equals the oracle's Adam recursion;
  - training is reproducible bit for bit and lowers the loss;
  - a build that uses the trained model produces exactly the factors of the
    build without it, while its ACA workspace (sized from the predicted
    ranks) is smaller.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2204_05536_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_05536_gb300 as p
    p.load()
    return p


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, 8)).astype(np.float32)
    t = (np.sin(X[:, 0] * 3) + X[:, 3] * 2 + 0.5 * X[:, 5]).astype(np.float32)
    return X, t


@pytest.mark.parametrize("hidden", [16, 64])
def test_forward_and_gradient_match_oracle(pkg, hidden):
    theta = inputs.mlp_init(hidden, seed=4)
    X, t = _data(1000, 1)
    m = pkg.RankModel(hidden, theta)
    y_ref, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64), hidden)
    y = m.predict(X)
    np.testing.assert_allclose(y, y_ref, rtol=1e-5, atol=1e-5)
    loss, g = m.loss_grad(X, t)
    loss_ref, g_ref = mlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                        t.astype(np.float64), hidden)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_adam_step_matches_oracle(pkg):
    hidden = 32
    theta = inputs.mlp_init(hidden, seed=7)
    X, t = _data(500, 2)
    m = pkg.RankModel(hidden, theta)
    m.train(X, t, batch=500, epochs=1, lr=1e-2)
    _, g_ref = mlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                 t.astype(np.float64), hidden)
    th_ref, _, _ = mlp.adam_step(theta.astype(np.float64), g_ref, np.zeros_like(g_ref),
                                 np.zeros_like(g_ref), 1, 1e-2)
    np.testing.assert_allclose(m.params(), th_ref, rtol=0, atol=2e-5)


def test_training_reproducible_and_learns(pkg):
    theta = inputs.mlp_init(64, seed=0)
    X, t = _data(20000, 3)
    a = pkg.RankModel(64, theta)
    b = pkg.RankModel(64, theta)
    l0, _ = a.loss_grad(X, t)
    la = a.train(X, t, batch=1024, epochs=5, lr=3e-3)
    lb = b.train(X, t, batch=1024, epochs=5, lr=3e-3)
    assert np.array_equal(a.params(), b.params()) and la == lb
    assert la < 0.1 * l0


def test_predicted_caps_give_identical_factors_and_smaller_workspace(pkg):
    # train on two smaller builds of the same recipe, use on a larger one
    feats, targets = [], []
    for n in (1 << 13, 1 << 14, 1 << 15):
        g = pkg.HODLR2D(inputs.uniform(n, seed=n), pkg.kernel("log"), 64, 1e-8,
                        root=(-1.0, -1.0, 2.0))
        f, r = g.pair_features()
        feats.append(f)
        targets.append(r)
    F = np.concatenate(feats)
    T = np.concatenate(targets)
    perm = np.random.default_rng(0).permutation(len(T))
    model = pkg.RankModel(64, inputs.mlp_init(64, seed=1))
    loss = model.train(F[perm], T[perm], batch=512, epochs=60, lr=3e-3)
    assert loss < 0.05
    n = 1 << 16
    pts = inputs.uniform(n, seed=5)
    plain = pkg.HODLR2D(pts, pkg.kernel("log"), 64, 1e-8, root=(-1.0, -1.0, 2.0))
    learned = pkg.HODLR2D(pts, pkg.kernel("log"), 64, 1e-8, root=(-1.0, -1.0, 2.0),
                          rank_model=model)
    a = plain.export_factors()
    b = learned.export_factors()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])  # bit-identical factors
    sp, sl = plain.stats(), learned.stats()
    assert sl["aca_workspace_values"] < 0.5 * sp["aca_workspace_values"]
    assert sl["aca_fallbacks"] <= 0.05 * sl["npairs"]
