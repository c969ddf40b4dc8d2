"""Float64 reference of the cost-model MLP (forward, MSE gradient, Adam).

TEST INFRASTRUCTURE ONLY: used by the tests to check the engine's MLP
kernels; nothing in the engine imports it. Plain numpy in float64, written
from the definitions, with no blocking or fusion.

Network (three fully connected layers, ReLU between them):
    H1 = relu(X W1 + b1)      X: (N, F), W1: (F, H)
    H2 = relu(H1 W2 + b2)     W2: (H, H)
    y  = H2 w3 + b3           w3: (H,), b3: scalar
Loss: mean squared error  L = (1/N) sum_n (y_n - t_n)^2.
Optimiser: Adam (Kingma and Ba, ICLR 2015, Algorithm 1) with bias-corrected
first and second moment estimates.

Packed parameter layout (shared interface with the engine, float32 there):
    [W1 row-major (F*H), b1 (H), W2 row-major (H*H), b2 (H), w3 (H), b3 (1)]
"""
from __future__ import annotations

import numpy as np


def n_params(F: int, H: int) -> int:
    return F * H + H + H * H + H + H + 1


def unpack(theta, F: int, H: int) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (n_params(F, H),)
    o = 0
    out = {}
    for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = theta[o:o + size].reshape(shape)
        o += size
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1) for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def forward(theta, X, F: int, H: int):
    """Returns (y, cache) for inputs X of shape (N, F)."""
    p = unpack(theta, F, H)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"] + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, p=p)


def loss(y, t) -> float:
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def backward(cache, y, t, F: int, H: int) -> np.ndarray:
    """Gradient of the mean squared error with respect to the packed parameters."""
    N = len(y)
    p = cache["p"]
    dy = 2.0 * (np.asarray(y, np.float64) - np.asarray(t, np.float64)) / N      # dL/dy, (N,)
    g = {}
    g["w3"] = cache["H2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dZ2 = np.outer(dy, p["w3"]) * (cache["Z2"] > 0)                           # (N, H)
    g["W2"] = cache["H1"].T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"].T) * (cache["Z1"] > 0)                               # (N, H)
    g["W1"] = cache["X"].T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return pack(g)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step counts from 1). Returns new (theta, m, v)."""
    theta = np.asarray(theta, np.float64)
    grad = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def train(theta, X, t, F: int, H: int, steps: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam for `steps` updates; returns (theta, losses before each update)."""
    m = np.zeros_like(theta, dtype=np.float64)
    v = np.zeros_like(theta, dtype=np.float64)
    theta = np.asarray(theta, np.float64).copy()
    losses = []
    for s in range(1, steps + 1):
        y, c = forward(theta, X, F, H)
        losses.append(loss(y, t))
        theta, m, v = adam_step(theta, backward(c, y, t, F, H), m, v, s, lr, beta1, beta2, eps)
    return theta, losses
