"""Two-vertex bilateral rows (App. A.1; the paper's cable constraints) in the FP64 oracle: a
row ties a vertex to a partner vertex, (q_v - q_partner) - offset + e lambda = 0, and its
impulse acts on both with opposite signs. Pinned by what the mathematics fixes: with no
external force the pair impulses are internal, so the two cubes' total momentum is
conserved exactly (a wrong sign of the partner's term would push both cubes the same way);
a hard row holds its offset (a cube hanging from another by its rows alone), and a
shrinking offset draws the cubes together by the prescribed amount."""
import numpy as np

import scenegen as sg
from oracle import Oracle, OracleOptions


def _momentum(sc, o, v):
    m = o.fem.mass
    return (m[:, None] * v).sum(0)


def test_pair_rows_conserve_momentum_without_external_forces():
    sc = sg.tied_cubes(m=3, compliance=1e-4, floor=False, gravity=(0.0, 0.0, 0.0), height=0.0)
    n_a = sc.n_verts // 2
    v0 = np.zeros_like(sc.q0)
    v0[:n_a, 0] = 0.4       # cube A moves away from cube B: the rows pull back
    v0[:n_a, 2] = 0.1
    o = Oracle(sc)
    q, v = sc.q0.copy(), v0.copy()
    p0 = _momentum(sc, o, v0)
    lam_seen = 0.0
    for _ in range(6):
        q, v, info = o.frame(q, v, OracleOptions(n_iters=5, n_cr=sc.n_cr))
        rows = [j for j, ct in enumerate(info["contacts"]) if ct.get("anchor")]
        assert len(rows) == len(sc.anchors) == 4
        lam_seen = max(lam_seen, float(np.abs(np.asarray(info["lam"])[rows]).max()))
    p1 = _momentum(sc, o, v)
    assert lam_seen > 1e-3                       # the rows did act
    assert np.abs(p1 - p0).max() < 1e-10 * np.abs(p0).max()
    # and they slowed the separation: cube B now moves along +x too
    assert v[n_a:, 0].mean() > 0.05


def test_hard_pair_rows_hold_their_offset():
    # cube A hangs from a hard anchor at its top; cube B hangs from cube A by the four hard
    # rows alone (no floor); solved exactly, each row's map equals its offset at the frame's
    # end
    sc = sg.tied_cubes(m=3, compliance=0.0, floor=False, height=0.0)
    top = int(np.argmax(sc.X[: sc.n_verts // 2, 2] - 1e-3 * np.abs(sc.X[: sc.n_verts // 2, 0] - 0.05)))
    sc.anchors.append(sg.Anchor(top, tuple(float(x) for x in sc.X[top]), (0.0, 0.0, 0.0), 0.0))
    o = Oracle(sc)
    q, v = sc.q0.copy(), sc.v0.copy()
    for _ in range(3):
        q, v, info = o.frame(q, v, OracleOptions(n_iters=40, n_cr=60, exact_constraint_solve=True))
    for an in sc.anchors[:4]:
        d = (q[an.vertex] - q[an.partner]) - np.asarray(an.target)
        assert np.abs(d).max() < 1e-6 * sc.bbox_diagonal
    # cube B sagged with cube A but did not fall away from it
    n_a = sc.n_verts // 2
    assert abs(q[n_a:, 2].mean() - q[:n_a, 2].mean()) < 0.2 * 0.1


def test_shrinking_offset_draws_the_cubes_together():
    # the rows' offset shrinks at 0.3 m/s (a cable pulled in): after 6 frames of h = 1/60 the
    # facing corners are 3 cm closer, hard rows, no gravity
    sc = sg.tied_cubes(m=3, compliance=0.0, pull=0.3, floor=False, gravity=(0.0, 0.0, 0.0),
                       height=0.0)
    o = Oracle(sc)
    q, v = sc.q0.copy(), sc.v0.copy()
    frames = 6
    for f in range(frames):
        q, v, _ = o.frame(q, v, OracleOptions(n_iters=30, n_cr=60, exact_constraint_solve=True),
                          t=f * sc.h)
    for an in sc.anchors:
        gap0 = sc.X[an.vertex, 0] - sc.X[an.partner, 0]
        gap1 = q[an.vertex, 0] - q[an.partner, 0]
        assert abs((gap1 - gap0) - 0.3 * frames * sc.h) < 1e-6
