"""Pins of the float64 MLP reference (oracle/mlp.py) against facts that do
not come from its own code: central finite differences of the loss, the
collapsed linear model when every ReLU is active, Adam's first-step
property, and convergence on a convex quadratic."""
import numpy as np

import graphgen as gg
from oracle import mlp as M


def _net(F, H, seed, positive=False):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.5, size=M.n_params(F, H))
    if positive:
        theta = np.abs(theta) + 0.05
    return theta


def test_gradient_matches_central_differences():
    F, H, N = 5, 7, 9
    rng = np.random.default_rng(1)
    theta = _net(F, H, 2)
    X = rng.normal(size=(N, F))
    t = rng.normal(size=N)
    y, c = M.forward(theta, X, F, H)
    g = M.backward(c, y, t, F, H)
    h = 1e-6
    num = np.zeros_like(theta)
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num[i] = (M.loss(M.forward(tp, X, F, H)[0], t) - M.loss(M.forward(tm, X, F, H)[0], t)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-7)


def test_all_relus_active_collapses_to_a_linear_model():
    F, H, N = 6, 8, 11
    rng = np.random.default_rng(3)
    theta = _net(F, H, 4, positive=True)
    X = np.abs(rng.normal(size=(N, F)))
    p = M.unpack(theta, F, H)
    a = p["W1"] @ p["W2"] @ p["w3"]
    c0 = p["b1"] @ p["W2"] @ p["w3"] + p["b2"] @ p["w3"] + p["b3"][0]
    y, cache = M.forward(theta, X, F, H)
    assert np.allclose(y, X @ a + c0)
    # chain rule on the collapsed model: dL/dW1 = X^T dy (W2 w3)^T, dL/db3 = sum dy
    t = rng.normal(size=N)
    dy = 2.0 * (y - t) / N
    g = M.unpack(M.backward(cache, y, t, F, H), F, H)
    assert np.allclose(g["W1"], np.outer(X.T @ dy, p["W2"] @ p["w3"]))
    assert np.allclose(g["b3"][0], dy.sum())
    assert np.allclose(g["b1"], dy.sum() * (p["W2"] @ p["w3"]))


def test_adam_first_step_has_magnitude_lr():
    # with zero initial moments the bias-corrected first step is
    # -lr * g / (|g| + eps): magnitude lr in every coordinate with g != 0
    rng = np.random.default_rng(5)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    g[7] = 0.0
    th1, m, v = M.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    step = theta - th1
    mask = g != 0
    assert np.allclose(np.abs(step[mask]), 0.01, rtol=1e-6)
    assert np.all(np.sign(step[mask]) == np.sign(g[mask]))
    assert step[7] == 0.0


def test_adam_minimises_a_quadratic():
    theta = np.array([10.0, -4.0])
    m = v = np.zeros(2)
    for s in range(1, 5001):
        grad = 2.0 * (theta - np.array([3.0, 1.5]))
        theta, m, v = M.adam_step(theta, grad, m, v, s, lr=0.05)
    assert np.allclose(theta, [3.0, 1.5], atol=1e-3)


def test_training_fits_a_smooth_target():
    F, H, N = 4, 16, 64
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, size=(N, F))
    t = X @ np.array([1.0, -2.0, 0.5, 0.0]) + 0.3
    theta0 = gg.mlp_init(F, H, 9).astype(np.float64)
    theta, losses = M.train(theta0, X, t, F, H, steps=400, lr=0.01)
    assert losses[-1] < 0.02 * losses[0]


def test_seeded_init_shape_and_bounds():
    F, H = 64, 128
    p = gg.mlp_init(F, H, 1)
    assert p.dtype == np.float32 and p.shape == (M.n_params(F, H),)
    u = M.unpack(p, F, H)
    assert np.all(np.abs(u["W1"]) <= np.sqrt(6 / F)) and np.all(np.abs(u["W2"]) <= np.sqrt(6 / H))
    assert not u["b1"].any() and not u["b2"].any() and u["b3"][0] == 0
    assert np.array_equal(p, gg.mlp_init(F, H, 1)) and not np.array_equal(p, gg.mlp_init(F, H, 2))
