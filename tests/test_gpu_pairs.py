"""Two-vertex bilateral rows (App. A.1) on the GPU against the FP64 oracle: a frame of two
cubes tied across a gap resting on a floor (pair rows beside frictional contacts, hard and
compliant), the momentum of free tied cubes (the pair impulses are internal), and a
shrinking offset (a cable pulled in) frame by frame from the oracle's states."""
import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle, OracleOptions
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cr32():
    import oracle.contact as OC
    cr64 = OC.conjugate_residual

    def cr32(apply, b, n_iter):
        return cr64(lambda x: apply(x.astype(np.float64)).astype(np.float32),
                    b.astype(np.float32), n_iter).astype(np.float64)
    return OC, cr64, cr32


@pytest.mark.parametrize("compliance", [0.0, 1e-4])
def test_tied_cubes_frame_matches_oracle(compliance):
    # the cubes start 0.2 mm inside the floor, so the frame has floor contacts beside the
    # four pair rows; where the oracle's own FP32 rounding of its constraint solve moves the
    # frame by more than 1e-6 the device is held to 10x that (the rule of the drop tests)
    sc = sg.tied_cubes(m=4, compliance=compliance, height=-0.0002)
    o = Oracle(sc)
    opts = OracleOptions(n_iters=5, n_cr=sc.n_cr)
    q, v, info = o.frame(sc.q0, sc.v0, opts)
    OC, cr64, cr32 = _cr32()
    OC.conjugate_residual = cr32
    try:
        q32, _, info32 = o.frame(sc.q0, sc.v0, opts)
    finally:
        OC.conjugate_residual = cr64
    dev32 = _relerr(q32 - sc.q0, q - sc.q0)
    sim = Simulator(sc)
    sim.set_state(sc.q0, sc.v0)
    sim.step(n_iters=5)
    qg, _ = sim.state()
    ct = sim.contacts()
    # the same rows: (vertex, obstacle id) pairs in the same order
    ref = [(c["vertex"], c["obstacle"]) for c in info["contacts"]]
    got = list(zip(ct["vertex"].tolist(), ct["obstacle"].tolist()))
    assert got == ref and len(ref) > len(sc.anchors)
    err = _relerr(qg - sc.q0, q - sc.q0)
    print(f"\ntied cubes (e = {compliance}): {len(ref)} rows, displacement error {err:.2e}, "
          f"oracle float32 deviation {dev32:.2e}")
    assert err < max(1e-5, 10 * dev32)
    # the pair rows' impulses: how the load of cube B splits over four rows and the floor
    # contacts is what FP32 moves (the oracle's own float32 run: 5.4e-2 for hard rows,
    # 6e-3 for compliant ones), so they are held to 10x the oracle's float32 deviation
    rows = [j for j, c in enumerate(info["contacts"]) if c.get("anchor")]
    lo, lg = np.asarray(info["lam"])[rows], ct["lam"][rows]
    lam_dev32 = _relerr(np.asarray(info32["lam"])[rows], lo)
    print(f"pair impulses error {_relerr(lg, lo):.2e}, oracle float32 deviation {lam_dev32:.2e}")
    assert _relerr(lg, lo) < max(1e-4, 10 * lam_dev32)
    sim.close()


def test_free_tied_cubes_conserve_momentum():
    sc = sg.tied_cubes(m=4, compliance=1e-4, floor=False, gravity=(0.0, 0.0, 0.0), height=0.0)
    n_a = sc.n_verts // 2
    v0 = np.zeros_like(sc.q0)
    v0[:n_a, 0] = 0.4
    v0[:n_a, 2] = 0.1
    o = Oracle(sc)
    m = o.fem.mass
    sim = Simulator(sc)
    sim.set_state(sc.q0, v0)
    p0 = (m[:, None] * v0).sum(0)
    for _ in range(10):
        sim.step(n_iters=5)
    _, vg = sim.state()
    p1 = (m[:, None] * vg).sum(0)
    print(f"\nmomentum change {np.abs(p1 - p0).max() / np.abs(p0).max():.2e} of the initial")
    # internal impulses only: FP32 rounding of the iterates, nothing systematic
    assert np.abs(p1 - p0).max() < 1e-4 * np.abs(p0).max()
    assert vg[n_a:, 0].mean() > 0.05            # cube B was pulled along
    sim.close()


def test_pulled_pair_rows_frame_by_frame():
    # hard rows whose offset shrinks at 0.3 m/s, the cubes on the floor, 6 frames from rest
    # (the simulator's clock, which moves the offset, runs from its last set_state, so each
    # comparison replays from the start). Hard rows beside floor contacts make the frames
    # FP32-sensitive (the oracle's own float32 run moves them by 4e-3 to 9e-3), so each
    # frame is held to 10x the oracle's float32 deviation on the same frames
    sc = sg.tied_cubes(m=4, compliance=0.0, pull=0.3, height=-0.0002)
    o = Oracle(sc)
    OC, cr64, cr32 = _cr32()
    sim = Simulator(sc)
    for f in range(6):
        sim.set_state(sc.q0, sc.v0)
        qo, vo = sc.q0.copy(), sc.v0.copy()
        q3, v3 = qo.copy(), vo.copy()
        for g in range(f + 1):
            opts = OracleOptions(n_iters=5, n_cr=sc.n_cr)
            qo, vo, _ = o.frame(qo, vo, opts, t=g * sc.h)
            OC.conjugate_residual = cr32
            try:
                q3, v3, _ = o.frame(q3, v3, opts, t=g * sc.h)
            finally:
                OC.conjugate_residual = cr64
            sim.step(n_iters=5)
        qg, _ = sim.state()
        dev32 = _relerr(q3 - sc.q0, qo - sc.q0)
        assert _relerr(qg - sc.q0, qo - sc.q0) < max(1e-4, 10 * dev32), f
    # the rows drew the facing corners together
    for an in sc.anchors:
        assert (qg[an.vertex, 0] - qg[an.partner, 0]) - (sc.X[an.vertex, 0] - sc.X[an.partner, 0]) > 0.01
    sim.close()
