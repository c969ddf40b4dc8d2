"""The cost-model MLP kernels (forward, MSE gradient, Adam, training) against
the float64 reference, through the C ABI. Tolerances follow FP32: sums of
at most F + H = 160 products per unit and of N <= 1000 rows per gradient
entry, so a relative error of 1e-4 of the largest magnitude bounds them."""
import numpy as np
import pytest

import graphgen as gg
from oracle import mlp as M

pytestmark = pytest.mark.gpu

F, H = 32, 128


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine
    return Engine(0)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, F)).astype(np.float32)
    t = (np.sin(3 * X[:, 1]) + X[:, 2] * X[:, 5] * 4 + X[:, 7]).astype(np.float32)
    return X, t


def _params(seed):
    p = gg.mlp_init(F, H, seed)
    rng = np.random.default_rng(seed)
    return (p + rng.normal(0, 0.02, size=p.shape)).astype(np.float32)   # nonzero biases too


@pytest.mark.parametrize("n", [1, 31, 77, 1000])
def test_forward_matches_reference(eng, n):
    p = _params(1)
    X, _ = _data(n, 2)
    m = eng.model(F, H, p)
    y = m.forward(X)
    ref, _ = M.forward(p.astype(np.float64), X.astype(np.float64), F, H)
    assert np.allclose(y, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    assert np.array_equal(m.params(), p)
    m.free()


@pytest.mark.parametrize("n", [5, 64, 333])
def test_gradient_matches_reference(eng, n):
    p = _params(3)
    X, t = _data(n, 4)
    m = eng.model(F, H, p)
    g, loss = m.gradient(X, t)
    y, cache = M.forward(p.astype(np.float64), X.astype(np.float64), F, H)
    gref = M.backward(cache, y, t.astype(np.float64), F, H)
    assert np.isclose(loss, M.loss(y, t), rtol=1e-4)
    scale = np.abs(gref).max()
    assert np.allclose(g, gref, rtol=1e-4, atol=1e-4 * scale)
    # per block: the bias gradients are exact sums of the unit gradients
    gu, ru = M.unpack(g, F, H), M.unpack(gref, F, H)
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        assert np.allclose(gu[k], ru[k], rtol=1e-4, atol=1e-4 * scale), k
    m.free()


def test_adam_step_matches_reference(eng):
    p = _params(5)
    X, t = _data(200, 6)
    m = eng.model(F, H, p)
    g, _ = m.gradient(X, t)
    m.adam_step(1e-3)
    th1, mm, vv = M.adam_step(p.astype(np.float64), g.astype(np.float64), 0, 0, 1, 1e-3)
    assert np.allclose(m.params(), th1, rtol=1e-5, atol=1e-6)
    g2, _ = m.gradient(X, t)
    m.adam_step(1e-3)
    th2, _, _ = M.adam_step(th1, g2.astype(np.float64), mm, vv, 2, 1e-3)
    assert np.allclose(m.params(), th2, rtol=1e-5, atol=1e-6)
    m.free()


def test_training_follows_reference(eng):
    p = _params(7)
    X, t = _data(300, 8)
    m = eng.model(F, H, p)
    losses = m.train(X, t, 30, 3e-3)
    _, ref = M.train(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), F, H, 30, 3e-3)
    assert np.allclose(losses, ref, rtol=2e-2)
    assert losses[-1] < 0.5 * losses[0]
    m.free()


def test_model_argument_errors(eng):
    from paper_2604_10601_gb300 import sgm
    with pytest.raises(sgm.SgmError):
        eng.model(F, 100, np.zeros(M.n_params(F, 100), np.float32))
    with pytest.raises(sgm.SgmError):
        eng.model(0, H, np.zeros(10, np.float32))
