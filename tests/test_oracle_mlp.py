"""Pins of the FP64 cost-model oracle (oracle/mlp.py) against the mathematics.

- the gradient equals central finite differences of the loss (every
  parameter, tiny network);
- with all weights zero the network is the constant b3: the loss and its
  gradient have closed forms;
- Adam's first step from zero moments moves every parameter by about
  -lr * sign(g) (bias correction makes m_hat = g, v_hat = g^2);
- full-batch training lowers the loss on a learnable target.
"""
import numpy as np

from oracle import mlp
from paper_1501_07350_gb300 import synth


def _data(n, d, seed):
    X = synth.uniform_pm1(seed, n * d).reshape(n, d)
    y = np.sin(X @ np.linspace(0.5, 1.5, d)) + 0.1 * X[:, 0] ** 2
    return X, y


def test_gradient_matches_finite_differences():
    d, H, n = 4, 5, 7
    X, y = _data(n, d, 3)
    p = mlp.init_params(d, H, synth.uniform01(9, 1000))
    p[d * H:d * H + H] = 0.1 * synth.uniform_pm1(10, H)           # non-zero biases too
    L, g = mlp.loss_grad(p, X, y, d, H)
    assert abs(L - mlp.loss(p, X, y, d, H)) < 1e-15
    h = 1e-6
    num = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (mlp.loss(p + e, X, y, d, H) - mlp.loss(p - e, X, y, d, H)) / (2 * h)
    assert np.max(np.abs(num - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_zero_weights_closed_form():
    d, H, n = 3, 4, 6
    X, y = _data(n, d, 5)
    p = np.zeros(mlp.num_params(d, H))
    p[-1] = 0.75                                                      # b3
    L, g = mlp.loss_grad(p, X, y, d, H)
    assert abs(L - np.mean((0.75 - y) ** 2)) < 1e-15
    assert abs(g[-1] - 2 * np.mean(0.75 - y)) < 1e-15
    # h1 = h2 = 0 and W3 = 0: every other gradient is zero except dL/dW3 = h2^T dy = 0
    assert np.all(g[:-1] == 0.0)


def test_adam_first_step_is_minus_lr_sign():
    g = np.array([0.3, -2.0, 1e-3, -5e-2])
    p0 = np.zeros(4)
    p1, m, v = mlp.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-5)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_lowers_the_loss():
    d, H, n = 5, 16, 64
    X, y = _data(n, d, 11)
    p = mlp.init_params(d, H, synth.uniform01(12, 2000))
    _, losses = mlp.train(p, X, y, d, H, steps=300, lr=0.01)
    assert losses[-1] < 0.2 * losses[0]
