"""Checkpoint and restore (sim_get_checkpoint / sim_set_checkpoint) in every start mode, the
state accessor's impulses, and loading a trained network (sim_load_warmstart).

A restored simulator must continue bit for bit as the saved one did: the previous-frame
start reads the last frame's contact record (impulses and normal moves per vertex), the
learned start reads it as features, and moving anchors read the time; none of that is in
(q, v), so a plain sim_set_state replay differs."""
import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import SimError, Simulator, WarmStartNet

pytestmark = pytest.mark.gpu


def _net(seed=5):
    net = WarmStartNet(seed=seed)
    theta = net.params()
    net.close()
    return theta


@pytest.mark.parametrize("mode", ["cold", "previous", "learned", "anchor"])
def test_checkpoint_replay_is_bitwise(mode):
    if mode == "anchor":
        sc = sg.hanging_cube(m=5, target_vel=(0.3, 0.0, 0.0), floor=True)
    else:
        sc = sg.cube_drop(m=6, seed=7, height=0.01)
    sim = Simulator(sc)
    if mode == "previous":
        sim.set_warmstart(2)
    elif mode == "learned":
        sim.load_warmstart(_net())
    sim.step(n_frames=6)
    blob = sim.checkpoint()
    q6, v6 = sim.state()
    sim.step(n_frames=4)
    q10, v10, lam10, st10 = sim.full_state()
    # restore into the same simulator and into a fresh one
    sim.restore(blob)
    sim.step(n_frames=4)
    q10b, v10b, lam10b, st10b = sim.full_state()
    assert np.array_equal(q10, q10b) and np.array_equal(v10, v10b)
    assert np.array_equal(lam10, lam10b)
    assert st10["frame"] == st10b["frame"] == 10
    fresh = Simulator(sc)
    if mode == "previous":
        fresh.set_warmstart(2)
    elif mode == "learned":
        fresh.load_warmstart(_net())
    fresh.restore(blob)
    fresh.step(n_frames=4)
    assert np.array_equal(fresh.state()[0], q10)
    # the restored contact record is what the warm starts read: the first restored frame's
    # features (7..9: the previous frame's impulse) equal the original continuation's; a
    # plain state replay forgets the record (zero features) and the anchors' time
    if mode in ("previous", "learned"):
        sim.restore(blob)
        sim.step()
        X_ck, _ = sim.warmstart_samples()
        fresh.restore(blob)
        fresh.step()
        assert np.array_equal(fresh.warmstart_samples()[0], X_ck)
        assert np.abs(X_ck[:, 7:10]).max() > 0
        sim.set_state(q6, v6)
        sim.step()
        X_st, _ = sim.warmstart_samples()
        assert np.all(X_st[:, 7:10] == 0)
    if mode == "anchor":
        sim.set_state(q6, v6)
        sim.step(n_frames=4)
        assert not np.array_equal(sim.state()[0], q10)
    fresh.close()
    sim.close()


def test_state_accessor_returns_the_contact_impulses():
    sc = sg.cube_drop(m=6, seed=2, height=-0.003)
    sim = Simulator(sc)
    sim.step()
    q, v, lam, st = sim.full_state()
    ct = sim.contacts()
    assert len(lam) == len(ct["lam"]) == st["n_contacts"] > 3
    assert np.array_equal(lam, ct["lam"])
    assert np.array_equal(q, sim.state()[0])
    assert st["residuals"] == sim.stats()["residuals"]
    sim.close()


def test_checkpoint_of_another_scene_is_rejected():
    a = Simulator(sg.cube_drop(m=6, seed=1))
    b = Simulator(sg.cube_drop(m=6, seed=1, E=2e5))
    with pytest.raises(SimError) as e:
        b.restore(a.checkpoint())
    assert e.value.status == -1
    with pytest.raises(SimError):
        a.restore(a.checkpoint()[:-8])
    a.close()
    b.close()


def test_load_warmstart_equals_set_warmstart_with_the_same_network():
    sc = sg.cube_drop(m=6, seed=4, height=0.005)
    net = WarmStartNet(seed=9)
    a, b = Simulator(sc), Simulator(sc)
    a.set_warmstart(1, net)
    b.load_warmstart(net.params())
    net.close()                         # the simulators keep their own copies
    for s in (a, b):
        s.step(n_frames=8)
    assert np.array_equal(a.state()[0], b.state()[0])
    with pytest.raises(SimError):
        b.load_warmstart(np.zeros(10, np.float32))
    a.close()
    b.close()
