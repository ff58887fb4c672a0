"""Delassus reuse across frames (sim_options.delassus_reuse): W~ = Y^T Y and Y depend only on
the list of contact vertices (S~ is constant), so a frame with the previous frame's list
keeps them. The trajectory must be bit for bit the one that builds them every frame; a
settled scene must actually reuse them; a state replay (sim_set_state) must not."""
import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu


# a settling cube keeps its contact vertices over many frames; a pressed two-box stack
# (contacts between the bodies, their triangle corners among the contact vertices) fewer
@pytest.mark.parametrize("maker,min_reused", [
    (lambda: sg.cube_drop(m=6, seed=3, height=0.002, mu=0.5), 5),
    (lambda: sg.box_stack(n_boxes=2, m=4, E=1e6, gap=-0.05, seed=2, incline_deg=0.0), 2),
])
def test_reuse_is_bitwise_and_happens(maker, min_reused):
    sc = maker()
    on, off = Simulator(sc, delassus_reuse=1), Simulator(sc, delassus_reuse=0)
    reused = []
    for f in range(30):
        for s in (on, off):
            s.step()
        reused.append(on.stats()["delassus_reused"])
        assert off.stats()["delassus_reused"] == 0
        qa, va = on.state()
        qb, vb = off.state()
        assert np.array_equal(qa, qb) and np.array_equal(va, vb), f
        assert np.array_equal(on.contacts()["lam"], off.contacts()["lam"]), f
        assert np.array_equal(on.delassus()[0], off.delassus()[0]), f
    st = on.stats()
    assert sum(reused) >= min_reused and st["delassus_reuse_frames"] == sum(reused)
    on.close()
    off.close()


def test_state_replay_builds_the_delassus_operator_again():
    sc = sg.cube_drop(m=6, seed=3, height=-0.002, mu=0.5)
    sim = Simulator(sc)
    for _ in range(3):
        sim.set_state(sc.q0, sc.v0)
        sim.step()
        assert sim.stats()["delassus_reused"] == 0
    sim.step()      # the next frame of the same trajectory may reuse it
    sim.close()
