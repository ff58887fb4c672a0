"""The portfolio start (not from the paper): copies of a scene in one batch, copy 0 cold and
the others warm-started, every copy continuing from the best one after each frame."""
import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import SimError, Simulator

pytestmark = pytest.mark.gpu


def test_portfolio_rejects_groups_that_are_not_copies():
    a, b = sg.warmstart_scenes([100, 101], frames=10)
    sim = Simulator([a, a])
    with pytest.raises(SimError):
        sim.set_portfolio(3)
    with pytest.raises(SimError):
        sim.set_portfolio(0)
    sim.set_portfolio(2)
    sim.set_portfolio(1)
    sim.close()
    sim = Simulator([a, b])
    with pytest.raises(SimError):
        sim.set_portfolio(2)
    sim.close()


def _contact_state(sc, frames=40):
    sim = Simulator(sc)
    for _ in range(frames):
        sim.step()
        if sim.stats()["n_contacts"] > 8:
            break
    q, v = sim.state()
    sim.close()
    return q, v


def test_cold_portfolio_equals_the_single_scene():
    sc = sg.warmstart_scenes([102], frames=60)[0]
    q, v = _contact_state(sc)
    one = Simulator(sc, n_iters=10)
    one.set_state(q, v)
    pf = Simulator([sc, sc], n_iters=10)
    pf.set_portfolio(2)
    pf.set_state(np.concatenate([q, q]), np.concatenate([v, v]))
    for _ in range(5):
        one.step()
        pf.step()
    q1, _ = one.state()
    qp, _ = pf.state()
    n = len(q)
    assert np.abs(qp[:n] - qp[n:]).max() == 0.0
    # the batch sums in another order than the single scene: FP32 rounding only. Over five
    # contact frames that rounding is amplified by the constraint solve's conditioning, so
    # the bound is the larger of 1e-5 of the positions and twice what the same five frames
    # move in the oracle when its conjugate residual runs in float32
    import oracle.contact as OC
    from oracle import Oracle
    from oracle.integrator import OracleOptions
    cr64 = OC.conjugate_residual

    def cr32(apply, b, n_iter):
        return cr64(lambda x: apply(x.astype(np.float64)).astype(np.float32),
                    b.astype(np.float32), n_iter).astype(np.float64)

    o, opts = Oracle(sc), OracleOptions(n_iters=10)
    runs = []
    for cr in (cr64, cr32):
        OC.conjugate_residual = cr
        try:
            qo, vo = q.copy(), v.copy()
            for _ in range(5):
                qo, vo, _ = o.frame(qo, vo, opts)
        finally:
            OC.conjugate_residual = cr64
        runs.append(qo)
    dev32 = np.abs(runs[1] - runs[0]).max()
    diff = np.abs(qp[:n] - q1).max()
    print(f"\ncold portfolio vs single scene {diff:.2e}, oracle float32 deviation {dev32:.2e}")
    assert diff < max(1e-5 * np.abs(q1).max(), 2 * dev32)
    one.close()
    pf.close()


def _two_frames(sc, q, v, portfolio_second, mode):
    """Frame 1 cold as a portfolio (the copies leave it identical), frame 2 with the given
    start, as a portfolio or with both copies independent."""
    sim = Simulator([sc, sc], n_iters=6)
    sim.set_portfolio(2)
    sim.set_state(np.concatenate([q, q]), np.concatenate([v, v]))
    sim.step()
    if not portfolio_second:
        sim.set_portfolio(1)
    sim.set_warmstart(mode)
    sim.step()
    out = sim.state()[0], sim.scene_residuals()
    sim.close()
    return out


def test_portfolio_continues_from_the_better_copy():
    # the same batch layout with the portfolio switched off for the second frame gives each
    # start's own result bit for bit; with it on, copy 0 matches the cold run, copy 1 the
    # previous-frame run, and both copies end in the state of the one with the lower final
    # residual
    sc = sg.warmstart_scenes([103], frames=60)[0]
    q, v = _contact_state(sc)
    n = len(q)
    q_cold, r_cold = _two_frames(sc, q, v, False, 0)
    q_prev, r_prev = _two_frames(sc, q, v, False, 2)
    q_pf, r_pf = _two_frames(sc, q, v, True, 2)
    assert np.array_equal(r_pf[0], r_cold[0]) and np.array_equal(r_pf[1], r_prev[1])
    assert np.array_equal(q_pf[:n], q_pf[n:])
    winner = q_cold[:n] if r_pf[0, -1] <= r_pf[1, -1] else q_prev[n:]
    assert np.array_equal(q_pf[:n], winner)
    assert r_pf[0, -1] != r_pf[1, -1]


def test_warm_copy_starts_like_a_single_scene():
    # after a synchronised frame the warm copy must see the previous frame's impulses at its
    # own obstacles: its start (residual at k = 0) matches a single scene's warm start, not
    # the cold start
    sc = sg.warmstart_scenes([100], frames=60)[0]
    q, v = _contact_state(sc)
    one = Simulator(sc, n_iters=6)
    one.set_state(q, v)
    one.step()
    one.set_warmstart(2)
    one.step()
    r_one = one.scene_residuals()[0]
    pf = Simulator([sc, sc], n_iters=6)
    pf.set_portfolio(2)
    pf.set_state(np.concatenate([q, q]), np.concatenate([v, v]))
    pf.step()
    pf.set_warmstart(2)
    pf.step()
    r_pf = pf.scene_residuals()
    assert abs(r_pf[1, 0] - r_one[0]) <= 1e-3 * r_one[0]
    assert abs(r_pf[1, 0] - r_pf[0, 0]) > 1e-2 * r_pf[0, 0]
    one.close()
    pf.close()
