"""Device allocator hooks (sim_options.dev_alloc / dev_free): every buffer of the simulator
comes from the caller's allocator (here PyTorch's caching allocator), is returned at
sim_destroy, and the results are those of the default allocator bit for bit."""
import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu


def test_simulator_buffers_come_from_the_callers_allocator():
    import torch
    live, total = {}, [0]

    def dev_alloc(nbytes, ctx):
        p = torch.cuda.caching_allocator_alloc(int(nbytes), device=0)
        live[p] = nbytes
        total[0] += nbytes
        return p

    def dev_free(p, ctx):
        torch.cuda.caching_allocator_delete(p)
        del live[p]

    sc = sg.cube_drop(m=6, height=-0.003, seed=2, mu=0.5)
    ref = Simulator(sc)
    sim = Simulator(sc, dev_alloc=dev_alloc, dev_free=dev_free)
    assert len(live) > 50 and total[0] > 1 << 20
    for s in (ref, sim):
        s.set_state(sc.q0, sc.v0)
        s.step(n_frames=3)
    assert np.array_equal(sim.state()[0], ref.state()[0])
    assert sim.stats()["residuals"] == ref.stats()["residuals"]
    sim.close()
    ref.close()
    assert not live
