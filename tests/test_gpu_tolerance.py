"""Frames that iterate to a residual tolerance (sim_options.residual_tol, sim_step with
n_iters <= 0): the stopping decision is taken on the device by a CUDA graph while-node. The
result must be the fixed-count frame with the count the tolerance picks, bit for bit."""
import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import SimError, Simulator

pytestmark = pytest.mark.gpu


def _contact_state(sc, frames=60):
    sim = Simulator(sc)
    for _ in range(frames):
        sim.step()
        if sim.stats()["n_contacts"] > 8:
            break
    q, v = sim.state()
    sim.close()
    return q, v


@pytest.mark.parametrize("seed,tol", [(100, 1e-4), (101, 1e-3), (102, 1e-5)])
def test_tolerance_frame_equals_the_fixed_frame_it_stops_at(seed, tol):
    sc = sg.warmstart_scenes([seed], frames=60)[0]
    q, v = _contact_state(sc)
    fixed = Simulator(sc)
    fixed.set_state(q, v)
    fixed.step(n_iters=40)
    r = np.asarray(fixed.stats()["residuals"])
    hit = [k for k in range(1, len(r)) if r[k] <= tol]
    k_star = hit[0] if hit else 40
    fixed.set_state(q, v)
    fixed.step(n_iters=k_star)
    q_fix, v_fix = fixed.state()
    r_fix = np.asarray(fixed.stats()["residuals"])
    adapt = Simulator(sc, residual_tol=tol, max_iters=40)
    adapt.set_state(q, v)
    adapt.step()
    st = adapt.stats()
    assert st["n_iters"] == k_star
    assert np.array_equal(np.asarray(st["residuals"]), r_fix)
    q_a, v_a = adapt.state()
    assert np.array_equal(q_a, q_fix) and np.array_equal(v_a, v_fix)
    ph = adapt.phase_times()
    assert ph["iterations"] > 0 and ph["local"] == 0.0
    assert adapt.scene_residuals().shape == (1, k_star + 1)
    fixed.close()
    adapt.close()


def test_tolerance_frame_stops_at_max_iters():
    sc = sg.warmstart_scenes([103], frames=60)[0]
    q, v = _contact_state(sc)
    fixed = Simulator(sc)
    fixed.set_state(q, v)
    fixed.step(n_iters=7)
    adapt = Simulator(sc, residual_tol=1e-300, max_iters=7)
    adapt.set_state(q, v)
    adapt.step()
    assert adapt.stats()["n_iters"] == 7
    assert np.array_equal(adapt.state()[0], fixed.state()[0])
    # a fixed count still works on the same handle (its own graph)
    adapt.set_state(q, v)
    adapt.step(n_iters=7)
    assert np.array_equal(adapt.state()[0], fixed.state()[0])
    fixed.close()
    adapt.close()


def test_tolerance_frame_without_contact_makes_one_update():
    sc = sg.cube_drop(m=5, height=1.0)
    adapt = Simulator(sc, residual_tol=1e-4)
    fixed = Simulator(sc)
    adapt.step()
    fixed.step(n_iters=1)
    assert adapt.stats()["n_iters"] == 1
    assert np.array_equal(adapt.state()[0], fixed.state()[0])
    adapt.close()
    fixed.close()


def test_tolerance_frames_in_a_batch_and_a_trajectory():
    # several frames in a row over a two-scene batch: every frame stops when the worst
    # scene's residual reaches the tolerance
    scenes = sg.warmstart_scenes([104, 105], frames=60)
    sim = Simulator(scenes, residual_tol=1e-4, max_iters=40)
    counts = []
    for _ in range(40):
        sim.step()
        st = sim.stats()
        counts.append(st["n_iters"])
        if st["n_contacts"]:
            r = st["residuals"]
            assert len(r) == st["n_iters"] + 1
            assert r[-1] <= 1e-4 or st["n_iters"] == 40
            assert all(x > 1e-4 for x in r[1:-1])
    assert max(counts) > 1
    sim.close()


def test_frames_without_phase_marks_are_the_same_frames():
    # the production graph (event nodes only around the once-per-frame phases) computes
    # the instrumented graph's frame bit for bit, reports the iterations as one phase, and
    # is faster (each event node costs a few microseconds)
    sc = sg.warmstart_scenes([101], frames=60)[0]
    q, v = _contact_state(sc)
    sim = Simulator(sc)
    out = {}
    for marks in (True, False, True, False):
        sim.set_phase_marks(marks)
        times = []
        for _ in range(6):
            sim.set_state(q, v)
            sim.step(n_iters=8)
            ph = sim.phase_times()
            times.append(sum(ph.values()))
        out[marks] = (sim.state()[0], sim.stats()["residuals"], ph, min(times))
    assert np.array_equal(out[True][0], out[False][0])
    assert out[True][1] == out[False][1]
    assert out[False][2]["iterations"] > 0 and out[False][2]["local"] == 0.0
    assert out[True][2]["iterations"] == 0.0 and out[True][2]["local"] > 0
    assert out[False][3] < out[True][3]
    sim.close()
