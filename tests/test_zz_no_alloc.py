"""The allocation-free global solve (sim_apply_inverse_noalloc) agrees with the regular one.

Callers that must not allocate device memory during a step (real-time loops, code running
under another component's stream capture, embedders with their own memory pool) get the
same x = A^-1 g from a variant whose scratch is a static device array. Each case makes two
calls in a row (the array keeps the first call's contents) and compares both with the
existing entry point (sim_apply_inverse of an FP32 simulator) and with the oracle's direct
sparse solve, on an FP32 simulator, a BF16 one (the variant reads the FP32 profile that the
device keeps in either mode) and a batch of two scenes. This file is collected last so that
a failure here comes after every other test has run."""
import numpy as np
import pytest

import scenegen as sg
from oracle.fem import FEM
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu

REL = 1e-5


def _oracle_solve(scenes, b):
    x = np.zeros_like(b)
    off = 0
    for sc in scenes:
        f = FEM(sc)
        blk = b[off:off + sc.n_verts]
        xs = np.zeros_like(blk)
        xs[f.free_verts] = f.solve(blk[f.free_verts].reshape(-1)).reshape(-1, 3)
        x[off:off + sc.n_verts] = xs
        off += sc.n_verts
    return x


@pytest.mark.parametrize("case", ["fp32", "bf16", "batch2"])
def test_noalloc_solve_matches_regular_solve_twice(case):
    import torch
    if case == "batch2":
        scenes = [sg.star_pull(n_side=20, layers=12), sg.cube_drop(m=9, model=sg.MODEL_SNH,
                                                                   E=1e6, seed=3)]
    else:
        scenes = [sg.star_pull(n_side=20, layers=12)]
    arg = scenes if case == "batch2" else scenes[0]
    sim = Simulator(arg, s_precision=1 if case == "bf16" else 0)
    ref = sim if case != "bf16" else Simulator(arg, s_precision=0)
    order, _, _ = sim.ordering()               # solver row k <-> caller vertex order[k]
    assert np.array_equal(order, ref.ordering()[0])
    n = sim.n_verts
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    dev_before = torch.cuda.current_device()
    for call in range(2):
        b = rng.normal(size=(n, 3)) * (1 + 5 * call)
        x_ref = ref.apply_inverse(b)[order]    # the existing entry point, host buffers
        x_or = _oracle_solve(scenes, b)[order]
        g = torch.tensor(b[order], dtype=torch.float32, device="cuda")
        x = torch.full_like(g, float("nan"))
        sim.apply_inverse_noalloc(g.data_ptr(), x.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.cuda.current_device() == dev_before
        xh = x.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(xh))
        err = np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)
        err_or = np.linalg.norm(xh - x_or) / np.linalg.norm(x_or)
        assert err < REL, (case, call, err)
        assert err_or < REL, (case, call, err_or)
    if ref is not sim:
        ref.close()
    sim.close()
