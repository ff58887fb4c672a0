"""The allocation-free global solve (sim_apply_inverse_noalloc) agrees with the regular one.

Callers that must not allocate device memory during a step (real-time loops, code running
under another component's stream capture, embedders with their own memory pool) get the
same x = A^-1 g from a variant whose scratch is a static device array. This file is
collected last so that a failure here comes after every other test has run."""
import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import Plan, Simulator

pytestmark = pytest.mark.gpu

REL = 1e-5


def test_noalloc_solve_matches_regular_solve_twice():
    import torch
    sc = sg.star_pull(n_side=20, layers=12)
    sim = Simulator(sc)
    order, _, _ = Plan(sc).ordering()          # solver row k <-> caller vertex order[k]
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        b = rng.normal(size=(sc.n_verts, 3)) * (1 + 5 * call)
        x_ref = sim.apply_inverse(b)[order]    # the existing entry point, host buffers
        g = torch.tensor(b[order], dtype=torch.float32, device="cuda")
        x = torch.full_like(g, float("nan"))
        sim.apply_inverse_noalloc(g.data_ptr(), x.data_ptr(), stream)
        torch.cuda.synchronize()
        xh = x.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(xh))
        err = np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)
        assert err < REL, (call, err)
    sim.close()
