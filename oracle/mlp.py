"""FP64 reference of the learned cost model (forward, loss, gradient, Adam).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests and the CPU legs
of bench.py use it; the CUDA path (paper_1501_07350_gb300/csrc/mlp.cu) shares
no code with it.

Network: x (d) -> tanh(x W1 + b1) (H) -> tanh(h1 W2 + b2) (H) -> h2 W3 + b3.
Parameters as one flat vector: W1[d][H], b1[H], W2[H][H], b2[H], W3[H], b3.
Loss: mean over samples of (yhat - y)^2.  Gradient by the chain rule, written
out layer by layer.  Adam as in Kingma & Ba, "Adam: A Method for Stochastic
Optimization" (ICLR 2015), Algorithm 1.
"""
from __future__ import annotations

import numpy as np


def num_params(d: int, H: int) -> int:
    return d * H + H + H * H + H + H + 1


def unpack(p, d: int, H: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + d * H].reshape(d, H); o += d * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def forward(p, X, d: int, H: int):
    W1, b1, W2, b2, W3, b3 = unpack(p, d, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    return h2 @ W3 + b3, (X, h1, h2)


def loss(p, X, y, d: int, H: int) -> float:
    yhat, _ = forward(p, X, d, H)
    return float(np.mean((yhat - np.asarray(y, dtype=np.float64)) ** 2))


def loss_grad(p, X, y, d: int, H: int):
    """Loss and its gradient with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(p, d, H)
    yhat, (X, h1, h2) = forward(p, X, d, H)
    n = X.shape[0]
    r = yhat - np.asarray(y, dtype=np.float64)
    L = float(np.mean(r ** 2))
    dy = 2.0 * r / n                       # dL/dyhat
    gW3 = h2.T @ dy
    gb3 = np.sum(dy)
    dh2 = np.outer(dy, W3)                 # dL/dh2
    dz2 = dh2 * (1.0 - h2 ** 2)            # through tanh
    gW2 = h1.T @ dz2
    gb2 = np.sum(dz2, axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (1.0 - h1 ** 2)
    gW1 = X.T @ dz1
    gb1 = np.sum(dz1, axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return L, g


def adam_step(p, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train(p, X, y, d: int, H: int, steps: int, lr: float):
    """Full-batch Adam; returns (params, loss before each step)."""
    p = np.asarray(p, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(1, steps + 1):
        L, g = loss_grad(p, X, y, d, H)
        losses.append(L)
        p, m, v = adam_step(p, g, m, v, t, lr)
    return p, np.array(losses)


def init_params(d: int, H: int, uniform01) -> np.ndarray:
    """Glorot-uniform weights and zero biases from a stream of U[0,1) draws."""
    u = np.asarray(uniform01, dtype=np.float64)
    p = np.zeros(num_params(d, H))
    o = 0
    k = 0
    for fan_in, fan_out in ((d, H), (H, H)):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        cnt = fan_in * fan_out
        p[o:o + cnt] = (2.0 * u[k:k + cnt] - 1.0) * a
        o += cnt + fan_out
        k += cnt
    a = np.sqrt(6.0 / (H + 1))
    p[o:o + H] = (2.0 * u[k:k + H] - 1.0) * a
    return p
