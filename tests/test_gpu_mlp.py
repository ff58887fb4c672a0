"""The warm-start network's tensor-core kernels against the FP64 oracle: the forward pass
and the gradient of the loss with the same parameters on the same inputs. The device runs
BF16 weights and activations with FP32 accumulation, so agreement is to BF16 tolerance:
relative L2 error <= 1e-2 and cosine >= 0.999 (the oracle is exact FP64)."""
import numpy as np
import pytest

from oracle import mlp
from paper_2503_15078_b300 import WarmStartNet

pytestmark = pytest.mark.gpu


def _params(seed):
    theta = mlp.init_params(seed)
    theta += 0.02 * np.random.default_rng(seed + 1).normal(size=theta.shape)
    P = mlp.unpack(theta)
    P[0][mlp.NF:, :] = 0.0
    P[6][:, mlp.NY:] = 0.0
    P[7][mlp.NY:] = 0.0
    return theta


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cos(a, b):
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.mark.parametrize("rows", [1, 37, 64, 300])
def test_forward_matches_oracle(rows):
    theta = _params(rows)
    X = np.random.default_rng(rows).normal(size=(rows, mlp.NF))
    net = WarmStartNet(max_batch=1024)
    net.set_params(theta)
    Y = net.forward(X)
    Yo, _ = mlp.forward(theta.astype(np.float32).astype(np.float64), X)
    err = _rel(Y, Yo[:, :mlp.NY])
    print("forward rows=%d relerr %.3e" % (rows, err))
    assert err < 1e-2
    net.close()


@pytest.mark.parametrize("rows", [50, 256, 1000])
def test_gradient_matches_oracle(rows):
    theta = _params(7)
    rng = np.random.default_rng(rows)
    X = rng.normal(size=(rows, mlp.NF))
    T = rng.normal(size=(rows, mlp.NY))
    net = WarmStartNet(max_batch=1024)
    net.set_params(theta)
    g, loss = net.gradient(X, T)
    th = theta.astype(np.float32).astype(np.float64)
    Y, cache = mlp.forward(th, X)
    go = mlp.backward(th, cache, Y, T)
    lo = mlp.loss(Y, T)
    # every parameter block on its own
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    for k in range(len(mlp.SHAPES)):
        a, b = g[offs[k]:offs[k + 1]], go[offs[k]:offs[k + 1]]
        if np.linalg.norm(b) == 0:
            assert np.linalg.norm(a) == 0
            continue
        print("block %d: rel %.3e cos %.6f" % (k, _rel(a, b), _cos(a, b)))
        assert _rel(a, b) < 1e-2 and _cos(a, b) > 0.999, k
    assert abs(loss - lo) < 1e-2 * lo
    net.close()


def test_training_on_the_device_reduces_the_loss():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(4096, mlp.NF))
    T = np.stack([np.tanh(X[:, 0]), X[:, 1] * X[:, 2], np.sin(X[:, 3]), 0.5 * X[:, 4] ** 2], 1)
    net = WarmStartNet(max_batch=1024, seed=1)
    _, l0 = net.gradient(X[:1024], T[:1024])
    losses = net.train(X, T, epochs=20, batch=256, lr=2e-3, seed=3)
    _, l1 = net.gradient(X[:1024], T[:1024])
    print("loss %.4f -> %.4f; per epoch %s" % (l0, l1, np.round(losses, 4)))
    assert l1 < 0.1 * l0
    # the trained parameters, run through the oracle, reproduce the device's forward pass
    theta = net.params().astype(np.float64)
    Yo, _ = mlp.forward(theta, X[:200])
    assert _rel(net.forward(X[:200]), Yo[:, :mlp.NY]) < 2e-2
    net.close()
