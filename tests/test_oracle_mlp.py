"""Pins of the warm-start network's oracle: the backward pass against central finite
differences of the loss (every parameter block, and every parameter of a narrow slice),
GELU against its definition, and the Adam update against its closed-form first step."""
import math

import numpy as np

from oracle import mlp


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, mlp.NF)), rng.normal(size=(n, mlp.NY))


def test_gelu_is_x_times_the_normal_cdf():
    x = np.linspace(-6, 6, 101)
    cdf = np.array([0.5 * (1 + math.erf(v / math.sqrt(2))) for v in x])
    assert np.allclose(mlp.gelu(x), x * cdf, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_backward_matches_central_differences():
    theta = mlp.init_params(3)
    theta += 0.05 * np.random.default_rng(4).normal(size=theta.shape)   # nonzero biases
    P = mlp.unpack(theta)
    P[0][mlp.NF:, :] = 0.0
    X, T = _data(7, 5)
    Y, cache = mlp.forward(theta, X)
    g = mlp.backward(theta, cache, Y, T)
    rng = np.random.default_rng(6)
    # every block: 12 random parameters each (the padded input rows of W1 have zero
    # gradient only because the padded inputs are zero; they are included)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    idx = np.concatenate([rng.integers(offs[k], offs[k + 1], 12) for k in range(len(mlp.SHAPES))])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(mlp.forward(tp, X)[0], T) - mlp.loss(mlp.forward(tm, X)[0], T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_padded_outputs_do_not_enter_the_loss():
    theta = mlp.init_params(1)
    X, T = _data(5, 2)
    Y, cache = mlp.forward(theta, X)
    g = mlp.unpack(mlp.backward(theta, cache, Y, T))
    assert np.all(g[6][:, mlp.NY:] == 0) and np.all(g[7][mlp.NY:] == 0)


def test_adam_first_step_moves_each_parameter_by_lr():
    # with m0 = v0 = 0 the bias-corrected first step is lr * g / (|g| + eps): size lr
    theta = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 3.0, -0.1])
    mlp.adam_step(theta, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    assert np.allclose(theta, -0.01 * np.sign(g), rtol=1e-6)


def test_training_reduces_the_loss_on_a_learnable_target():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(256, mlp.NF))
    T = np.stack([np.tanh(X[:, 0]), X[:, 1] * X[:, 2], np.sin(X[:, 3]), X[:, 4] ** 2], 1)
    theta = mlp.init_params(0)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    l0 = mlp.loss(mlp.forward(theta, X)[0], T)
    for t in range(1, 201):
        Y, c = mlp.forward(theta, X)
        mlp.adam_step(theta, mlp.backward(theta, c, Y, T), m, v, t, lr=2e-3)
    assert mlp.loss(mlp.forward(theta, X)[0], T) < 0.2 * l0
