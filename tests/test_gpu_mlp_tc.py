"""The warm-start network's inference on the 5th-generation tensor cores (tcgen05.mma with
its FP32 accumulators in tensor memory) against the warp-level mma.sync inference and the
FP64 oracle, on the same parameters and inputs: BF16 weights and activations with FP32
accumulation on both device paths, so agreement is to BF16 tolerance (relative L2 <= 1e-2
against the oracle); the two device paths differ only in the order of their FP32 sums."""
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


@pytest.mark.parametrize("rows", [1, 37, 128, 300])
def test_tcgen05_inference_matches_mma_sync_and_the_oracle(rows):
    theta = _params(rows + 11)
    X = np.random.default_rng(rows).normal(size=(rows, mlp.NF))
    net = WarmStartNet(max_batch=1024)
    net.set_params(theta)
    y_mma = net.forward(X)
    net.set_tensor_cores("tcgen05")
    y_tc = net.forward(X)
    y_tc2 = net.forward(X)
    yo, _ = mlp.forward(theta.astype(np.float32).astype(np.float64), X)
    e_or, e_mma = _rel(y_tc, yo[:, :mlp.NY]), _rel(y_tc, y_mma)
    print(f"rows={rows}: tcgen05 vs oracle {e_or:.3e}, vs mma.sync {e_mma:.3e}")
    assert np.all(np.isfinite(y_tc))
    assert np.array_equal(y_tc, y_tc2)
    assert e_or < 1e-2
    assert e_mma < 1e-2
    net.close()
