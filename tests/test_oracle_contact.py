"""Pins of the oracle's contact layer: geometry, Fischer-Burmeister functions and their
derivatives (App. B.2), the Coulomb reading of phi_f (App. A.2, Eqs. 43-44), and the
conjugate-residual solver."""
import numpy as np
import pytest

import scenegen as sg
from oracle import contact as C


def test_fb_zero_iff_complementary():
    rng = np.random.default_rng(0)
    a = rng.uniform(-2, 2, 4000)
    b = rng.uniform(-2, 2, 4000)
    assert np.all(C.fb(a, b)[(a > 0) & (b > 0)] > 0)
    assert np.all(C.fb(a, b)[(a < 0) | (b < 0)] < 0)
    z = rng.uniform(0, 2, 100)
    assert np.abs(C.fb(z, 0 * z)).max() == 0 and np.abs(C.fb(0 * z, z)).max() == 0


def test_normal_indicator_and_compliance_are_derivatives():
    # omega_n = d phi_n / d delta_n and E_n = d phi_n / d lambda_n (Eq. 16)
    rng = np.random.default_rng(1)
    for _ in range(200):
        d, lam, r = rng.normal(), rng.normal(), rng.uniform(0.1, 3)
        phi, om, E = C.normal_terms(d, lam, r)
        eps = 1e-7
        dphi_dd = (C.normal_terms(d + eps, lam, r)[0] - C.normal_terms(d - eps, lam, r)[0]) / (2 * eps)
        dphi_dl = (C.normal_terms(d, lam + eps, r)[0] - C.normal_terms(d, lam - eps, r)[0]) / (2 * eps)
        assert abs(om - dphi_dd) < 1e-6 and abs(E - dphi_dl) < 1e-6 * max(1, r)
        assert abs(phi - C.fb(d, r * lam)) < 1e-15


def test_friction_reduces_to_coulomb_at_solutions():
    rng = np.random.default_rng(2)
    for _ in range(100):
        lam_n = rng.uniform(0.1, 5)
        mu = rng.uniform(0.05, 1)
        r = rng.uniform(0.01, 2)
        # sliding: lambda_f opposes the velocity at the cone boundary -> phi_f = 0
        v = rng.normal(size=2)
        lam_f = -mu * lam_n * v / np.linalg.norm(v)
        om, E, phi = C.friction_terms(v, lam_f, lam_n, mu, r)
        assert om == 1.0
        assert abs(E - np.linalg.norm(v) / np.linalg.norm(lam_f)) < 1e-9 * E
        assert np.abs(phi).max() < 1e-9 * np.linalg.norm(v)
        # sticking: zero velocity strictly inside the cone -> E_f = 0, phi_f = 0
        lam_f2 = rng.uniform(0, 0.9) * mu * lam_n * np.array([np.cos(1.0), np.sin(1.0)])
        om, E, phi = C.friction_terms(np.zeros(2), lam_f2, lam_n, mu, r)
        assert E == 0.0 and np.abs(phi).max() == 0.0
        # inactive contact: phi_f = lambda_f drives friction to zero
        om, E, phi = C.friction_terms(v, lam_f, -lam_n, mu, r)
        assert om == 0.0 and E == 1.0 and np.allclose(phi, lam_f)


def test_friction_compliance_positive_and_no_fixed_point_outside_cone():
    rng = np.random.default_rng(3)
    for _ in range(500):
        lam_n, mu, r = rng.uniform(0.1, 5), rng.uniform(0.05, 1), rng.uniform(0.01, 2)
        v = rng.normal(size=2) * rng.choice([0.0, 1e-3, 1.0])
        lam_f = rng.normal(size=2) * mu * lam_n * rng.uniform(0, 4)
        om, E, phi = C.friction_terms(v, lam_f, lam_n, mu, r)
        assert E >= 0.0
        if np.linalg.norm(lam_f) > mu * lam_n * (1 + 1e-9):
            assert np.linalg.norm(phi) > 0.0


def test_plane_and_cylinder_geometry():
    pl = sg.Obstacle(sg.OBST_PLANE, (0, 0, 1.0), (0, 0, 1.0))
    phi, n, p = C.closest_point(pl, np.array([0.3, -0.2, 0.75]))
    assert abs(phi + 0.25) < 1e-15 and np.allclose(n, [0, 0, 1]) and np.allclose(p, [0.3, -0.2, 1.0])
    cy = sg.Obstacle(sg.OBST_CYLINDER, (1.0, 0, 0), (0, 0, 1.0), radius=0.5)
    phi, n, p = C.closest_point(cy, np.array([1.0, 0.3, 7.0]))
    assert abs(phi + 0.2) < 1e-15 and np.allclose(n, [0, 1, 0]) and np.allclose(p, [1.0, 0.5, 7.0])
    phi, n, p = C.closest_point(cy, np.array([4.0, 4.0, -1.0]))
    assert abs(phi - (5.0 - 0.5)) < 1e-14 and np.allclose(n, [0.6, 0.8, 0])


def test_tangent_frames_orthonormal_right_handed():
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        f1, f2 = C.tangent_frame(n)
        D = np.stack([n, f1, f2])
        assert np.abs(D @ D.T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(D) - 1.0) < 1e-14


def test_conjugate_residual_exact_in_n_steps_and_monotone():
    rng = np.random.default_rng(5)
    n = 12
    B = rng.normal(size=(n, n))
    K = B @ B.T + n * np.eye(n)
    b = rng.normal(size=n)
    x = C.conjugate_residual(lambda v: K @ v, b, n)
    assert np.abs(x - np.linalg.solve(K, b)).max() < 1e-10 * np.abs(x).max()
    res = [np.linalg.norm(b - K @ C.conjugate_residual(lambda v: K @ v, b, k)) for k in range(n)]
    assert all(res[k + 1] <= res[k] * (1 + 1e-12) for k in range(n - 1))


def test_detection_finds_exactly_the_vertices_below_margin():
    sc = sg.cube_drop(m=4, height=0.004, seed=3)
    pts = sc.q0
    cts = C.detect(sc, pts, np.arange(sc.n_verts))
    below = set(np.nonzero(pts[:, 2] < sc.contact_margin)[0].tolist())
    assert {c["vertex"] for c in cts} == below
    for c in cts:
        assert abs(c["d_n"]) < 1e-15 and np.allclose(c["n"], [0, 0, 1])


def test_minmap_normal_zero_iff_complementary_and_branch_derivatives():
    # min(delta, r lambda) vanishes exactly on 0 <= delta _|_ lambda >= 0 (App. B.1), and on
    # each branch omega_n and E_n are the derivatives in delta_n and lambda_n
    rng = np.random.default_rng(11)
    for _ in range(400):
        d, lam, r = rng.normal(), rng.normal(), rng.uniform(0.1, 3)
        phi, om, E = C.minmap_normal_terms(d, lam, r)
        if d > 0 and lam > 0:
            assert phi > 0
        if d < 0 or lam < 0:
            assert phi < 0
        eps = 1e-7 * min(1.0, abs(d - r * lam))
        dphi_dd = (C.minmap_normal_terms(d + eps, lam, r)[0] -
                   C.minmap_normal_terms(d - eps, lam, r)[0]) / (2 * eps)
        dphi_dl = (C.minmap_normal_terms(d, lam + eps / r, r)[0] -
                   C.minmap_normal_terms(d, lam - eps / r, r)[0]) / (2 * eps / r)
        assert abs(om - dphi_dd) < 1e-6 and abs(E - dphi_dl) < 1e-6 * max(1, r)
        assert om in (0.0, 1.0) and E in (0.0, r) and (om == 1.0) == (E == 0.0)
    z = rng.uniform(0, 2, 50)
    for x in z:
        assert C.minmap_normal_terms(x, 0.0, 1.3)[0] == 0.0
        assert C.minmap_normal_terms(0.0, x, 1.3)[0] == 0.0


def test_minmap_friction_vanishes_exactly_on_coulomb_states():
    rng = np.random.default_rng(12)
    for _ in range(200):
        lam_n = rng.uniform(0.1, 5)
        mu = rng.uniform(0.05, 1)
        r = rng.uniform(0.01, 2)
        v = rng.normal(size=2)
        # slip: lambda_f on the cone boundary, opposite to the velocity
        lam_f = -mu * lam_n * v / np.linalg.norm(v)
        om, E, phi = C.minmap_friction_terms(v, lam_f, lam_n, mu, r)
        assert om == 1.0
        assert abs(E - np.linalg.norm(v) / (mu * lam_n)) < 1e-12 * E
        assert np.abs(phi).max() < 1e-12 * np.linalg.norm(v)
        # stick: zero velocity inside the cone
        lam_f2 = rng.uniform(0, 0.99) * mu * lam_n * np.array([np.cos(0.3), np.sin(0.3)])
        om, E, phi = C.minmap_friction_terms(np.zeros(2), lam_f2, lam_n, mu, r)
        assert E == 0.0 and np.abs(phi).max() == 0.0
        # not solutions: slip along the velocity, or a moving contact inside the cone with
        # the velocity above r (mu lambda_n - |lambda_f|)
        om, E, phi = C.minmap_friction_terms(v, -lam_f, lam_n, mu, r)
        assert np.linalg.norm(phi) > 1.9 * np.linalg.norm(v)
        s = mu * lam_n - np.linalg.norm(lam_f2)
        v2 = v / np.linalg.norm(v) * (r * s * rng.uniform(1.5, 3.0))
        om, E, phi = C.minmap_friction_terms(v2, lam_f2, lam_n, mu, r)
        assert E > 0 and np.linalg.norm(phi) > 0
        # inactive contact: phi_f = lambda_f, the same as the Fischer-Burmeister form
        om, E, phi = C.minmap_friction_terms(v, lam_f, -lam_n, mu, r)
        assert om == 0.0 and E == 1.0 and np.allclose(phi, lam_f)


def test_minmap_and_fb_share_indicators_away_from_the_kink():
    # on the two arms of the complementarity set (an active contact with delta_n -> 0, a
    # separated one with lambda_n -> 0) the FB indicator and compliance tend to the
    # minimum map's branch values
    for d, lam in ((1e-9, 1.0), (1.0, 1e-9), (1e-12, 3.0), (2.0, 1e-12)):
        r = 0.7
        _, om_fb, E_fb = C.normal_terms(d, lam, r)
        _, om_mm, E_mm = C.minmap_normal_terms(d, lam, r)
        assert abs(om_fb - om_mm) < 1e-6 and abs(E_fb - E_mm) < 1e-6


def test_friction_activity_needs_a_resolvable_normal_impulse():
    # App. B.1-B.2 switch friction on for lambda_n > 0; the reading takes that decision with
    # a tolerance r_n lambda_n > ACTIVE_REL L, so a rounding residue of a cancelled impulse
    # is inactive, while any impulse that displaces the contact by more than that is active
    r, L, mu = 2e-3, 0.2, 0.5
    v = np.array([3e-3, -1e-3])
    for lam_n, expect in ((1e-52, False), (4.8e-7 * 1e-3, False), (-1.0, False),
                          (2.0 * C.ACTIVE_REL * L / r, True), (1.0, True)):
        act = C.friction_active(lam_n, r, L)
        assert act == expect
        for terms in (C.friction_terms, C.minmap_friction_terms):
            om, E, phi = terms(v, np.zeros(2), lam_n, mu, 0.01, act)
            assert om == (1.0 if expect else 0.0)
            if not expect:
                assert E == 1.0 and np.all(phi == 0.0)
