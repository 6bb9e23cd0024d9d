"""Pins of the pair-screening network oracle (CPU only): finite differences of
the loss against the analytic backward pass, the closed form of Adam's first
step, loss reduction on a learnable target, and descriptors of a separable case."""
import numpy as np
import pytest

from oracle import mlp


def random_theta(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(mlp.n_params()) * scale


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((37, 8))
    t = rng.standard_normal(37)
    th = random_theta(2)
    g = mlp.grad(th, x, t)
    h = 1e-6
    idx = rng.choice(mlp.n_params(), 120, replace=False)
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss(th + e, x, t) - mlp.loss(th - e, x, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9


def test_constant_network_closed_form():
    th = np.zeros(mlp.n_params())
    p = mlp.unpack(th)
    p["b3"][:] = 0.7
    th = mlp.pack(p)
    t = np.array([1.0, 2.0, -1.0])
    x = np.zeros((3, 8))
    assert mlp.loss(th, x, t) == pytest.approx(np.mean((0.7 - t) ** 2))
    g = mlp.unpack(mlp.grad(th, x, t))
    assert g["b3"][0] == pytest.approx(2 * (0.7 - t.mean()))
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((20, 8))
    t = rng.standard_normal(20)
    th = random_theta(4)
    g = mlp.grad(th, x, t)
    th2 = th.copy()
    mlp.Adam(lr=1e-3).run(th2, x, t, epochs=1)
    # m_hat = g, v_hat = g^2 after one step -> update = -lr * g / (|g| + eps)
    assert np.allclose(th2 - th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_training_reduces_loss():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((200, 8))
    t = np.tanh(x[:, 0] - 0.5 * x[:, 3]) + 0.1 * x[:, 5]
    th = random_theta(6, 0.2)
    hist = mlp.Adam(lr=3e-3).run(th, x, t, epochs=400)
    assert hist[-1] < 0.05 * hist[0]


def test_features_of_separable_orbitals():
    M = 10
    pos = np.arange(M, dtype=float) * 3.0
    r_ops = np.stack([np.diag(pos), np.zeros((M, M)), np.zeros((M, M))])
    C = np.zeros((M, 3))
    for k, p in enumerate([1, 4, 8]):
        C[p, k] = 1.0
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    sigma = [np.array([2.0, 1.0, 0.0])] * 6
    f = mlp.pair_features(C, r_ops, pairs, sigma, [2] * 6, M)
    assert f[1, 0] == pytest.approx(9.0) and f[2, 0] == pytest.approx(21.0)
    assert np.allclose(f[:, 2], 0.0) and np.allclose(f[:, 3], 0.0)
    assert f[0, 4] == pytest.approx(np.log(2.0)) and f[0, 7] == pytest.approx(0.5 * np.log(5.0))


def test_planted_mistake_missing_tanh_derivative():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((10, 8))
    t = rng.standard_normal(10)
    th = random_theta(8)
    p = mlp.unpack(th)
    y, (x0, h1, h2) = mlp.forward(th, x)
    dy = 2 * (y - t) / 10
    wrong_W2 = ((dy[:, None] * p["W3"])).T @ h1          # tanh' dropped
    right = mlp.unpack(mlp.grad(th, x, t))["W2"]
    assert np.abs(wrong_W2 - right).max() > 1e-3
