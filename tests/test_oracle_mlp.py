"""Pins for the oracle's learned-guess network (forward, backward, Adam).

* the gradient matches central differences of the loss (every parameter
  block);
* a network with zero hidden weights outputs its last bias, and a linear
  probe through tanh reproduces tanh of the input;
* BF16 rounding is round-to-nearest-even on the upper 16 bits;
* one Adam step from zero moments moves every parameter by lr * sign(g)
  (for |g| >> eps), the textbook first-step property.
"""
import numpy as np
import pytest

from oracle import mlp


def _params(seed=0, scale=0.2):
    rng = np.random.default_rng(seed)
    theta = rng.normal(size=mlp.NPARAM) * scale
    return mlp.unpack(theta), theta


def test_gradient_central_differences():
    p, theta = _params(1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, mlp.IN))
    t = rng.normal(size=(7, mlp.OUT))
    loss, g = mlp.loss_and_grad(p, x, t)
    gflat = mlp.pack(g)
    idx = rng.choice(mlp.NPARAM, size=40, replace=False)
    # include the first entries of every block
    k = 0
    for name, shape in mlp.SIZES:
        idx = np.append(idx, k)
        k += int(np.prod(shape))
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        lp, _ = mlp.loss_and_grad(mlp.unpack(tp), x, t)
        lm, _ = mlp.loss_and_grad(mlp.unpack(tm), x, t)
        fd = (lp - lm) / (2 * h)
        assert gflat[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_forward_special_cases():
    p, _ = _params(3)
    for name in ("W1", "W2", "W3"):
        p[name] = np.zeros_like(p[name])
    x = np.random.default_rng(4).normal(size=(5, mlp.IN))
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, p["b3"][None, :])
    # h1 = tanh(x0), h2 = tanh(tanh(x0)), y0 = h2 picked by W3
    p = {k: np.zeros_like(v) for k, v in mlp.unpack(np.zeros(mlp.NPARAM)).items()}
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0, 0] = 1.0
    y, _ = mlp.forward(p, x)
    assert np.allclose(y[:, 0], np.tanh(np.tanh(x[:, 0])))
    assert np.allclose(y[:, 1], 0.0)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.1415926], dtype=np.float32)
    r = mlp.round_bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie -> even
    assert r[2] == 1.0 + 2 ** -7          # representable
    assert r[3] == 1.0 + 2 ** -6          # tie -> even (upward)
    assert r[4] == -2.5
    assert abs(r[5] - 3.140625) < 1e-12


def test_adam_first_step():
    rng = np.random.default_rng(5)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(new, theta - 1e-3 * np.sign(g), atol=1e-9)


def test_features():
    prev = np.array([[2.0 + 1j, -4.0], [1.0, 0.5j], [0, 0], [1j, 1]])
    x, scale = mlp.features(prev, 0.5 + 2.0j, 0.25)
    assert scale == 4.0
    assert np.allclose(x[0, :2], [0.5, 0.25]) and np.allclose(x[1, :2], [-1.0, 0.0])
    assert np.allclose(x[:, 8], 0.125) and np.allclose(x[:, 9], 0.5)
