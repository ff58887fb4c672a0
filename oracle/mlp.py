"""The warm-start network: a multilayer perceptron mapping per-contact features to an
initial contact impulse and a normal displacement guess.

TEST INFRASTRUCTURE (see the package docstring). Not from the paper: the paper starts
every frame from lambda = 0. This module is the FP64 definition the GPU kernels are checked
against: forward pass, loss, backward pass (plain reverse-mode differentiation of the
forward, written out layer by layer) and the Adam update.

Architecture: inputs padded to IN = 16 (NF = 11 features), three hidden layers of H = 128
units with GELU(x) = x Phi(x) (the exact Gaussian form), a linear output layer padded to
OUT = 8 (NY = 4 outputs used). Parameters are one flat FP32/FP64 vector in the order
W1 (IN x H, row = input), b1 (H), W2 (H x H), b2, W3 (H x H), b3, W4 (H x OUT), b4 (OUT).
Loss: L = 1/(2N) sum_n sum_{c < NY} (y_nc - t_nc)^2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

NF, IN, H, OUT, NY = 11, 16, 128, 8, 4
SHAPES = [(IN, H), (H,), (H, H), (H,), (H, H), (H,), (H, OUT), (OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    """Flat vector -> [W1, b1, W2, b2, W3, b3, W4, b4] (views)."""
    out, off = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[off:off + n].reshape(s))
        off += n
    return out


def init_params(seed):
    """Deterministic initialisation: weights uniform in +-sqrt(6 / (fan_in + fan_out)),
    biases zero, the padded input rows and output columns zero."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(N_PARAMS)
    P = unpack(theta)
    for k in range(0, 8, 2):
        fi, fo = SHAPES[k]
        P[k][...] = rng.uniform(-1, 1, size=(fi, fo)) * math.sqrt(6.0 / (fi + fo))
    P[0][NF:, :] = 0.0
    P[6][:, NY:] = 0.0
    return theta


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def forward(theta, X):
    """X: N x NF (or N x IN). Returns Y (N x OUT) and the cache for backward."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    if X.shape[1] < IN:
        X = np.concatenate([X, np.zeros((X.shape[0], IN - X.shape[1]))], axis=1)
    Z1 = X @ W1 + b1
    A1 = gelu(Z1)
    Z2 = A1 @ W2 + b2
    A2 = gelu(Z2)
    Z3 = A2 @ W3 + b3
    A3 = gelu(Z3)
    Y = A3 @ W4 + b4
    return Y, (X, Z1, A1, Z2, A2, Z3, A3)


def loss(Y, T):
    N = Y.shape[0]
    D = Y[:, :NY] - np.asarray(T, dtype=np.float64)[:, :NY]
    return 0.5 * float(np.sum(D * D)) / N


def backward(theta, cache, Y, T):
    """Gradient of the loss with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(np.asarray(theta, dtype=np.float64))
    X, Z1, A1, Z2, A2, Z3, A3 = cache
    N = Y.shape[0]
    dY = np.zeros_like(Y)
    dY[:, :NY] = (Y[:, :NY] - np.asarray(T, dtype=np.float64)[:, :NY]) / N
    gW4 = A3.T @ dY
    gb4 = dY.sum(axis=0)
    dZ3 = (dY @ W4.T) * gelu_grad(Z3)
    gW3 = A2.T @ dZ3
    gb3 = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ W3.T) * gelu_grad(Z2)
    gW2 = A1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * gelu_grad(Z1)
    gW1 = X.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in place; t counts from 1."""
    m *= beta1
    m += (1 - beta1) * grad
    v *= beta2
    v += (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta
