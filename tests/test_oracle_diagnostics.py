"""Pins of the oracle's trajectory diagnostics, Oracle.energy and Oracle.max_penetration,
against closed forms (they gate the free-running trajectory tests), and of the Kronecker
structure of the 3n system: the oracle factors the full 3n x 3n matrix A, so the identity
A = A~ (x) I3, L = L~ (x) I3 and S = S~ (x) I3 (S = L^-1 P, Theorem 1) is checked on it
rather than assumed.
"""
import math

import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle
from oracle.fem import FEM, lame, snh_parameters
from oracle.sparse_inverse import cholesky, etree, postorder, sparse_inverse_columns


# -- energy -------------------------------------------------------------------------------
def test_free_fall_energy_drifts_by_the_implicit_euler_closed_form():
    # An undeformed body in free fall (uniform velocity, far from the ground) stays rigid
    # and moves as v1 = v0 + h g, q1 = q0 + h v1. Kinetic plus gravitational energy then
    # changes by exactly -M h^2 |g|^2 / 2 per frame (implicit Euler's numerical damping):
    # 1/2 M (|v0 + h g|^2 - |v0|^2) - M g . h (v0 + h g) = -1/2 M h^2 |g|^2.
    # A missing 1/2 in the kinetic term or a flipped gravity sign gives M h g.v0 + ... and
    # fails, because v0 has a component along g.
    sc = sg.cube_drop(m=4, edge=0.2, rho=700.0, height=5.0, seed=0)
    v0 = np.tile([0.3, -0.2, 1.5], (sc.n_verts, 1))
    o = Oracle(sc)
    M = 700.0 * 0.2 ** 3
    g = np.asarray(sc.gravity)
    h = sc.h
    q, v = sc.q0.copy(), v0.copy()
    e_prev = o.energy(q, v)
    for _ in range(3):
        q, v, info = o.frame(q, v)
        assert len(info["contacts"]) == 0
        e = o.energy(q, v)
        assert abs((e - e_prev) - (-0.5 * M * h ** 2 * float(g @ g))) < 1e-9 * abs(e_prev)
        e_prev = e


def test_energy_of_a_translating_rest_shape_is_kinetic_plus_height():
    # no deformation: E = 1/2 M |v|^2 + M |g| z_com with M = rho * edge^3, for any lift
    sc = sg.cube_drop(m=3, edge=0.1, rho=1000.0, height=0.0, seed=1)
    o = Oracle(sc)
    M = 1000.0 * 0.1 ** 3
    v = np.tile([1.0, 2.0, -0.5], (sc.n_verts, 1))
    for lift in (0.0, 0.37):
        q = sc.X + np.array([0.2, -0.1, lift])
        z_com = float(np.average(q[:, 2], weights=o.fem.mass))
        expect = 0.5 * M * 5.25 + M * 9.81 * z_com
        assert abs(o.energy(q, v) - expect) < 1e-12 * abs(expect)


def _no_gravity(sc):
    sc.gravity = (0.0, 0.0, 0.0)
    return sc


@pytest.mark.parametrize("model", [sg.MODEL_ARAP, sg.MODEL_COROT, sg.MODEL_SNH])
def test_elastic_energy_is_invariant_under_rigid_motions(model):
    # ARAP and co-rotational vanish on rotations; stable Neo-Hookean keeps its (non-zero)
    # rest value V (lam/2 (1 - alpha)^2 - mu/2 log 4) on every rotation
    sc = _no_gravity(sg.cube_drop(m=4, model=model, E=2e5, nu=0.4, seed=2))
    o = Oracle(sc)
    rng = np.random.default_rng(3)
    R = sg.random_rotation(rng)
    q = sc.X @ R.T + rng.normal(size=3)
    zero = np.zeros_like(q)
    e_rest = o.energy(sc.X, zero)
    if model == sg.MODEL_SNH:
        mu, lam, alpha = snh_parameters(2e5, 0.4)
        vol = float(o.fem.V.sum())
        expect = vol * (0.5 * lam * (1.0 - alpha) ** 2 - 0.5 * mu * math.log(4.0))
        assert abs(e_rest - expect) < 1e-9 * abs(expect)
    else:
        assert abs(e_rest) < 1e-12
    assert abs(o.energy(q, zero) - e_rest) < 1e-9 * max(abs(e_rest), 1e-6)


@pytest.mark.parametrize("model", [sg.MODEL_ARAP, sg.MODEL_COROT, sg.MODEL_SNH])
def test_elastic_energy_of_a_stretched_tet_by_hand(model):
    # F = diag(s, 1, 1) in a regular tetrahedron of edge e (volume e^3 / (6 sqrt 2)):
    # ARAP mu (s-1)^2, co-rotational mu (s-1)^2 + lam/2 (s-1)^2, stable Neo-Hookean
    # mu/2 (s^2 - 1) + lam/2 (s - alpha)^2 - mu/2 log(s^2 + 3)
    E, nu, e, s = 3e5, 0.35, 0.1, 1.07
    sc = _no_gravity(sg.single_tet(edge=e, model=model, E=E, nu=nu))
    o = Oracle(sc)
    q = sc.X * np.array([s, 1.0, 1.0])
    vol = e ** 3 / (6.0 * math.sqrt(2.0))
    mu, lam = lame(E, nu)
    if model == sg.MODEL_ARAP:
        psi = mu * (s - 1) ** 2
    elif model == sg.MODEL_COROT:
        psi = mu * (s - 1) ** 2 + 0.5 * lam * (s - 1) ** 2
    else:
        ms, ls, al = snh_parameters(E, nu)
        psi = 0.5 * ms * (s * s - 1) + 0.5 * ls * (s - al) ** 2 - 0.5 * ms * math.log(s * s + 3)
    got = o.energy(q, np.zeros_like(q))
    assert abs(got - vol * psi) < 1e-10 * abs(vol * psi), (got, vol * psi)


# -- max penetration ----------------------------------------------------------------------
def test_max_penetration_of_hand_placed_vertices():
    sc = sg.cube_drop(m=3, edge=0.1, height=0.5, seed=0)      # ground plane z = 0
    o = Oracle(sc)
    q = sc.X + np.array([0.0, 0.0, 0.5])
    assert o.max_penetration(q) == 0.0                        # all above the plane
    q[5, 2] = -0.0123                                         # one vertex 12.3 mm below
    q[7, 2] = -0.004
    assert abs(o.max_penetration(q) - 0.0123) < 1e-15
    # a cylinder of radius 0.05 along x through (0, 1, 0): a vertex 0.03 from its axis
    # is 0.02 deep, whatever its axial coordinate
    sc.obstacles = sc.obstacles + [sg.Obstacle(sg.OBST_CYLINDER, (0.0, 1.0, 0.0),
                                               (1.0, 0.0, 0.0), radius=0.05)]
    o = Oracle(sc)
    q = sc.X + np.array([0.0, 0.0, 0.5])
    q[2] = (7.0, 1.0 + 0.03 * math.cos(0.4), 0.03 * math.sin(0.4))
    assert abs(o.max_penetration(q) - 0.02) < 1e-14


def test_max_penetration_skips_pinned_vertices():
    sc = sg.cube_drop(m=3, edge=0.1, height=0.5, seed=0)
    sc.pinned = np.array([4], np.int32)
    o = Oracle(sc)
    q = sc.X + np.array([0.0, 0.0, 0.5])
    q[4, 2] = -0.5                                            # pinned: not a penetration
    assert o.max_penetration(q) == 0.0


# -- Kronecker structure of the 3n factor (C3 reading: the GPU stores scalar S~ only) -----
def test_full_factor_is_the_kronecker_product_of_the_per_vertex_factor():
    sc = sg.cube_drop(m=3, model=sg.MODEL_COROT, E=4e5, seed=4)
    sc.pinned = np.array([0, 1], np.int32)                    # Dirichlet rows eliminated
    f = FEM(sc)
    A = f.A_ff.toarray()                                      # the full 3n_f x 3n_f matrix
    n = A.shape[0] // 3
    At = A[0::3, 0::3]
    # A[3i + r, 3j + c] = delta_rc A~_ij, built entry by entry from G (never from A~)
    assert np.abs(A - np.kron(At, np.eye(3))).max() < 1e-12 * np.abs(A).max()
    # a fill-reducing order of A~ (any permutation serves: here a postorder of its etree
    # after a reversal), lifted to the 3n DoFs as P (x) I3
    perm = postorder(etree(At[::-1, ::-1]))
    perm = (n - 1 - np.arange(n))[perm]
    P = np.eye(n)[perm]
    P3 = np.kron(P, np.eye(3))
    L = cholesky(P @ At @ P.T)
    L3 = cholesky(P3 @ A @ P3.T)
    assert np.abs(L3 - np.kron(L, np.eye(3))).max() < 1e-12 * np.abs(L3).max()
    # S = L^-1 P, column by column over ancestors (Alg. 2), equals S~ (x) I3
    S = sparse_inverse_columns(L, etree(P @ At @ P.T)) @ P
    S3 = sparse_inverse_columns(L3, etree(P3 @ A @ P3.T)) @ P3
    assert np.abs(S3 - np.kron(S, np.eye(3))).max() < 1e-12 * np.abs(S3).max()
    assert np.abs(S3.T @ S3 - np.linalg.inv(A)).max() < 1e-10 * np.abs(np.linalg.inv(A)).max()


def test_fb_terms_evaluated_in_fp32_move_on_the_drop_frames():
    # Why the device evaluates the contact terms (Eqs. 52-57) in FP64: the inputs the oracle
    # meets on a 6^3 drop (impact, bounce, rest; 40 frames of 5 iterations), evaluated once
    # more with every operation in float32, move the compliances by far more than the 1e-5
    # parity gate on a sizeable share of the rows: the difference delta + r lambda - rho
    # cancels near the complementarity point, and the sticking / outside-cone branches of
    # E_f flip. (The kernel is latency-bound, so FP32 would not make it faster either.)
    import oracle.contact as C
    from oracle import OracleOptions
    rec_n, rec_f = [], []
    fb_n, fb_f = C.NCP_TERMS["fb"]

    def nt(dn, ln, rn):
        rec_n.append((dn, ln, rn))
        return fb_n(dn, ln, rn)

    def ft(vf, lf, ln, mu, rf, active=None):
        rec_f.append((np.array(vf, float), np.array(lf, float), ln, mu, rf, active))
        return fb_f(vf, lf, ln, mu, rf, active)

    C.NCP_TERMS["fb"] = (nt, ft)
    try:
        sc = sg.cube_drop(m=6, seed=0)
        o = Oracle(sc)
        q, v = sc.q0.copy(), sc.v0.copy()
        for _ in range(40):
            q, v, _ = o.frame(q, v, OracleOptions(n_iters=5, n_cr=sc.n_cr))
    finally:
        C.NCP_TERMS["fb"] = (fb_n, fb_f)
    f32 = np.float32

    def rel(a, b):
        return abs(float(a) - b) / abs(b) if b != 0 else float(a != 0)

    err_n = []
    for dn, ln, rn in rec_n:
        _, _, E64 = fb_n(dn, ln, rn)
        d, l, r = f32(dn), f32(ln), f32(rn)
        rho = np.sqrt(d * d + r * r * l * l)
        E32 = (f32(1) - r * l / rho) * r if rho != 0 else f32(0)
        err_n.append(rel(E32, E64))
    err_f = []
    for vf, lf, ln, mu, rf, act in rec_f:
        if not (act if act is not None else ln > 0) or mu <= 0:
            continue
        E64 = fb_f(vf, lf, ln, mu, rf, act)[1]
        a = np.sqrt((vf.astype(f32) ** 2).sum())
        lmag = np.sqrt((lf.astype(f32) ** 2).sum())
        l32, m32, r32 = f32(ln), f32(mu), f32(rf)
        s = m32 * l32 - lmag
        root = np.sqrt(a * a + r32 * r32 * s * s)
        num, den = root - r32 * s, a + m32 * r32 * l32 - root
        scale = a + m32 * r32 * l32 + r32 * abs(s)
        if num <= f32(C.TINY_REL) * scale:
            E32 = f32(0)
        elif den <= f32(C.TINY_REL) * scale:
            E32 = (a + r32 * (lmag - m32 * l32)) / (m32 * l32)
        else:
            E32 = num / den * r32
        err_f.append(rel(E32, E64))
    err_n, err_f = np.array(err_n), np.array(err_f)
    share_n, share_f = (err_n > 1e-5).mean(), (err_f > 1e-2).mean()
    print(f"\nFP32 contact terms: E_n {len(err_n)} rows, {share_n:.1%} off by > 1e-5; E_f "
          f"{len(err_f)} rows, {share_f:.1%} off by > 1e-2")
    assert len(err_n) > 1000 and len(err_f) > 200
    assert share_n > 0.05 and share_f > 0.02
