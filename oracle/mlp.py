"""Learned initial-guess network (oracle): forward, loss gradient, Adam step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper extrapolates the next frequency's solution from the previous ones
by least squares (Sec. 4.2). The learned guess adds one more candidate column
to that least-squares fit: a pointwise network that maps, for every unknown,
the four previous solution values (normalised by the largest magnitude of the
latest one) and the sampling frequency to the next value.

  x (10) -> tanh(W1 x + b1) (256) -> tanh(W2 h1 + b2) (256) -> W3 h2 + b3 (2)

Parameters are kept in one flat float vector:
  W1 (256 x 10, row-major), b1 (256), W2 (256 x 256), b2 (256), W3 (2 x 256), b3 (2).
The GPU path multiplies by the BF16-rounded weight matrices with FP32
accumulation; ``round_bf16`` gives the same rounding so the oracle can use the
identical weights in float64.
Loss: mean over the batch of the squared error summed over the two outputs.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 10, 256, 2
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def round_bf16(a):
    """Round float32 values to bfloat16 (round to nearest even) and back to float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def compute_weights(theta):
    """Parameters as used in the products: matrices BF16-rounded, biases as given."""
    p = unpack(np.asarray(theta, dtype=np.float32).astype(np.float64))
    for name in ("W1", "W2", "W3"):
        p[name] = round_bf16(p[name])
    return p


def forward(p, x):
    """Returns y and the cached activations."""
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, h1, h2)


def loss_and_grad(p, x, t):
    """Mean squared error and its gradient with respect to every parameter."""
    y, (x, h1, h2) = forward(p, x)
    B = x.shape[0]
    d3 = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B
    loss = float(np.sum((y - t) ** 2) / B)
    g = {"W3": d3.T @ h2, "b3": d3.sum(axis=0)}
    d2 = (d3 @ p["W3"]) * (1.0 - h2 ** 2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (1.0 - h1 ** 2)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return loss, g


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of the flat parameter vector; t counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(prev, s, dt):
    """Inputs of the network for every unknown.

    prev: (4, N) complex, the solutions at k-1, k-2, k-3, k-4; s: complex s_k;
    dt: time step. Returns (x (N, 10), scale) with scale = max |a_{k-1}|.
    """
    prev = np.asarray(prev, dtype=np.complex128)
    scale = float(np.max(np.abs(prev[0])))
    scale = scale if scale > 0 else 1.0
    q = prev / scale
    N = prev.shape[1]
    x = np.zeros((N, IN))
    for j in range(4):
        x[:, 2 * j] = q[j].real
        x[:, 2 * j + 1] = q[j].imag
    x[:, 8] = s.real * dt
    x[:, 9] = s.imag * dt
    return x, scale
