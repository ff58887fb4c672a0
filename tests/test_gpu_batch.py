"""Batches of independent scenes in one simulator: every scene's frame must be the frame
the oracle computes for that scene alone (the same 1e-5 FP32 parity as single scenes), and
the per-scene contacts, residuals and Delassus blocks must be the scene's own."""
import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle, OracleOptions
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu

REL = 1e-5


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _mixed_scenes():
    return [
        sg.cube_drop(m=6, model=sg.MODEL_ARAP, height=-0.003, seed=2, mu=0.5),
        sg.cube_drop(m=5, model=sg.MODEL_SNH, E=2e5, height=-0.002, seed=3, mu=0.3, tilt_deg=20),
        sg.cube_drop(m=3, model=sg.MODEL_SNH, E=1e6, height=-0.001, seed=6, mu=0.0),
        sg.cube_drop(m=7, model=sg.MODEL_COROT, height=-0.004, seed=4, mu=0.8, tilt_deg=10),
        sg.cube_drop(m=4, model=sg.MODEL_ARAP, height=0.3, seed=5),   # in the air: no contact
    ]


def test_batch_frame_matches_the_oracle_scene_by_scene():
    scenes = _mixed_scenes()
    sim = Simulator(scenes)
    sim.step(n_iters=5)
    q, _ = sim.state()
    ct = sim.contacts()
    res_gpu = sim.scene_residuals()
    off = sim.scene_offsets
    n_with_contact = 0
    for k, sc in enumerate(scenes):
        qo, vo, info = Oracle(sc).frame(sc.q0, sc.v0, OracleOptions(n_iters=5, n_cr=sc.n_cr))
        qg = q[off[k]:off[k + 1]]
        assert _relerr(qg, qo) < REL, (k, _relerr(qg, qo))
        mine = (ct["vertex"] >= off[k]) & (ct["vertex"] < off[k + 1])
        keys_g = list(zip((ct["vertex"][mine] - off[k]).tolist(), ct["obstacle"][mine].tolist()))
        # obstacles are numbered over the batch: scene k's obstacles follow the earlier ones
        o_off = sum(len(s.obstacles) for s in scenes[:k])
        keys_o = [(c["vertex"], c["obstacle"] + o_off) for c in info["contacts"]]
        assert keys_g == keys_o, k
        if keys_o:
            n_with_contact += 1
            assert abs(res_gpu[k, -1] - info["residuals"][-1]) < 1e-4 + 0.05 * info["residuals"][-1]
        else:
            assert np.all(res_gpu[k] == 0)
    assert n_with_contact >= 3
    sim.close()


def test_batch_matches_single_scene_simulators_over_frames():
    scenes = _mixed_scenes()
    batch = Simulator(scenes)
    batch.step(n_frames=4)
    qb, vb = batch.state()
    for k, sc in enumerate(scenes):
        one = Simulator(sc)
        one.step(n_frames=4)
        q1, v1 = one.state()
        one.close()
        sl = slice(batch.scene_offsets[k], batch.scene_offsets[k + 1])
        # independent scenes: only the summation order of the products differs
        assert _relerr(qb[sl] - sc.q0, q1 - sc.q0) < 1e-3, k
    batch.close()


def test_batch_delassus_is_block_diagonal():
    scenes = _mixed_scenes()
    sim = Simulator(scenes)
    sim.step(n_iters=1)
    W, cv = sim.delassus()
    off = sim.scene_offsets
    scene_of = np.searchsorted(off, cv, side="right") - 1
    for k, sc in enumerate(scenes):
        one = Simulator(sc)
        one.step(n_iters=1)
        W1, cv1 = one.delassus()
        one.close()
        mine = scene_of == k
        assert np.array_equal(cv[mine] - off[k], cv1)
        if len(cv1):
            blk = W[np.ix_(mine, mine)]
            assert np.abs(blk - W1).max() <= 1e-5 * np.abs(W1).max()
    cross = scene_of[:, None] != scene_of[None, :]
    assert np.all(W[cross] == 0)
    sim.close()


def test_sixty_four_uneven_scenes_run_in_one_simulator():
    # the 64-scene workload (cubes of 8^3 to 20^3 vertices, mixed materials, tilted planes)
    scenes = sg.batch(n_scenes=64, seed=0)
    sim = Simulator(scenes, s_precision=1)
    sim.step(n_frames=3)
    q, v = sim.state()
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(v))
    st = sim.stats()
    assert st["kernels_per_frame"] > 0
    # the smallest scenes against the oracle after one frame from the initial state
    sim2 = Simulator(scenes, s_precision=1)
    sim2.step()
    q2, _ = sim2.state()
    sizes = [sc.n_verts for sc in scenes]
    for k in np.argsort(sizes)[:3]:
        sc = scenes[k]
        qo, _, _ = Oracle(sc).frame(sc.q0, sc.v0, OracleOptions(n_iters=5, n_cr=sc.n_cr))
        sl = slice(sim2.scene_offsets[k], sim2.scene_offsets[k + 1])
        # BF16 S~ with the last-iteration correction: measured error, bounded loosely
        assert _relerr(q2[sl] - sc.q0, qo - sc.q0) < 5e-2, k
    sim.close()
    sim2.close()


def test_sharded_batch_equals_the_whole_batch_scene_by_scene():
    # a batch split over two ranks by nnz(S~) (paper_2503_15078_b300.shard), each part
    # simulated on its own as one rank would (here one after the other on the one GPU): every
    # scene's trajectory equals the whole batch's up to the rounding of its reordered sums,
    # and its contact list is the same
    from paper_2503_15078_b300 import shard
    scenes = sg.batch(n_scenes=10, seed=5, m_lo=4, m_hi=10)
    for sc in scenes:   # start 0.2 mm inside the (tilted) plane
        sc.q0 = sc.q0 - 0.0502 * np.asarray(sc.obstacles[0].axis)
    whole = Simulator(scenes)
    whole.step(n_frames=3)
    qw, _ = whole.state()
    cw = whole.contacts()
    off = whole.scene_offsets
    costs = shard.scene_costs(scenes)
    parts = shard.partition(costs, 2)
    assert all(parts) and sorted(parts[0] + parts[1]) == list(range(len(scenes)))
    n_contact_scenes = 0
    for part in parts:
        sim = Simulator([scenes[i] for i in part])
        sim.step(n_frames=3)
        qp, _ = sim.state()
        cp = sim.contacts()
        for k, i in enumerate(part):
            a, b = sim.scene_offsets[k], sim.scene_offsets[k + 1]
            ref = qw[off[i]:off[i + 1]]
            assert _relerr(qp[a:b] - scenes[i].q0, ref - scenes[i].q0) < 1e-5, i
            mine_p = (cp["vertex"] >= a) & (cp["vertex"] < b)
            mine_w = (cw["vertex"] >= off[i]) & (cw["vertex"] < off[i + 1])
            assert np.array_equal(cp["vertex"][mine_p] - a, cw["vertex"][mine_w] - off[i])
            n_contact_scenes += int(mine_w.sum() > 0)
        sim.close()
    assert n_contact_scenes >= 5
    whole.close()
