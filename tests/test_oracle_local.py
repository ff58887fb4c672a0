"""Pins of the oracle's local step p = argmin w/2 ||p - F||^2 + V psi(p) (Eq. 5).

Each projection is checked against conditions that do not reuse the oracle's sigma-space
reduction: closed forms for ARAP, rotation equivariance, and stationarity of the full
9-dimensional objective with psi evaluated directly from F (finite differences).
"""
import math

import numpy as np
import pytest

import scenegen as sg
from oracle.fem import lame, snh_parameters
from oracle.local import project, svd_signed


def _rot(rng):
    return sg.random_rotation(rng)


def test_signed_svd_reconstructs_and_has_rotations():
    rng = np.random.default_rng(0)
    F = rng.normal(size=(200, 3, 3))
    U, s, Vt = svd_signed(F)
    assert np.abs(np.einsum("tij,tj,tjk->tik", U, s, Vt) - F).max() < 1e-12
    assert np.allclose(np.linalg.det(U), 1) and np.allclose(np.linalg.det(Vt), 1)
    assert np.all(np.sign(s[:, 2]) == np.sign(np.linalg.det(F)))


def test_arap_projection_is_the_rotation_factor():
    rng = np.random.default_rng(1)
    n = 50
    R1 = np.stack([_rot(rng) for _ in range(n)])
    R2 = np.stack([_rot(rng) for _ in range(n)])
    d = rng.uniform(0.5, 2.0, size=(n, 3))
    F = np.einsum("tij,tj,tjk->tik", R1, d, R2)
    one = np.ones(n)
    p = project(F, np.zeros(n, np.int32), one, one, one, one, 0 * one)
    assert np.abs(p - R1 @ R2).max() < 1e-12
    # inverted element: flipping the smallest singular value gives the closest rotation
    d2 = d.copy()
    d2[:, 2] = -0.1
    F2 = np.einsum("tij,tj,tjk->tik", R1, d2, R2)
    p2 = project(F2, np.zeros(n, np.int32), one, one, one, one, 0 * one)
    assert np.allclose(np.linalg.det(p2), 1.0)
    assert np.abs(p2 - R1 @ R2).max() < 1e-12


def _psi_F(model, F, mu, lam, alpha):
    """psi evaluated from F itself (no SVD): the independent reference for stationarity."""
    if model == sg.MODEL_COROT:
        # R from the polar decomposition via the matrix square root of F^T F
        w, Q = np.linalg.eigh(F.T @ F)
        Sroot = Q @ np.diag(np.sqrt(w)) @ Q.T
        R = F @ np.linalg.inv(Sroot)
        if np.linalg.det(R) < 0:
            raise ValueError("use positive det for this reference")
        return mu * np.sum((F - R) ** 2) + 0.5 * lam * (np.trace(R.T @ F) - 3) ** 2
    ic = np.trace(F.T @ F)
    J = np.linalg.det(F)
    return 0.5 * mu * (ic - 3) + 0.5 * lam * (J - alpha) ** 2 - 0.5 * mu * math.log(ic + 1)


@pytest.mark.parametrize("model", [sg.MODEL_COROT, sg.MODEL_SNH])
def test_projection_is_stationary_for_full_objective(model):
    rng = np.random.default_rng(7 + model)
    E, nu, V = 1e5, 0.4, 2e-6
    mu_le, lam_le = lame(E, nu)
    if model == sg.MODEL_SNH:
        mu, lam, alpha = snh_parameters(E, nu)
    else:
        mu, lam, alpha = mu_le, lam_le, 0.0
    w = 2 * mu_le * V
    n = 12
    F = np.stack([_rot(rng) @ np.diag(rng.uniform(0.7, 1.4, 3)) @ _rot(rng) for _ in range(n)])
    ones = np.ones(n)
    p = project(F, np.full(n, model, np.int32), w * ones, V * ones, mu * ones, lam * ones,
                alpha * ones)
    eps = 1e-6
    for t in range(n):
        def obj(P):
            return 0.5 * w * np.sum((P - F[t]) ** 2) + V * _psi_F(model, P, mu, lam, alpha)
        g = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                d = np.zeros((3, 3))
                d[i, j] = eps
                g[i, j] = (obj(p[t] + d) - obj(p[t] - d)) / (2 * eps)
        scale = w * np.abs(F[t]).max()
        assert np.abs(g).max() < 1e-6 * scale, (t, np.abs(g).max() / scale)
        # a minimum, not a saddle: random perturbations do not decrease the objective
        for _ in range(10):
            d = 1e-3 * rng.normal(size=(3, 3))
            assert obj(p[t] + d) >= obj(p[t]) - 1e-12 * abs(obj(p[t]))


@pytest.mark.parametrize("model", [sg.MODEL_ARAP, sg.MODEL_COROT, sg.MODEL_SNH])
def test_projection_rotation_equivariant(model):
    rng = np.random.default_rng(11)
    n = 20
    F = np.stack([np.eye(3) + 0.3 * rng.normal(size=(3, 3)) for _ in range(n)])
    Q = _rot(rng)
    c = np.ones(n)
    args = (np.full(n, model, np.int32), 2e-1 * c, 1e-6 * c, 4e4 * c, 1e5 * c, 1.3 * c)
    p1 = project(F, *args)
    p2 = project(Q[None] @ F, *args)
    assert np.abs(Q[None] @ p1 - p2).max() < 1e-10


@pytest.mark.parametrize("model", [sg.MODEL_ARAP, sg.MODEL_COROT, sg.MODEL_SNH])
def test_rest_shape_projects_to_identity(model):
    E, nu = 1e6, 0.45
    mu_le, lam_le = lame(E, nu)
    mu, lam, alpha = snh_parameters(E, nu) if model == sg.MODEL_SNH else (mu_le, lam_le, 0.0)
    c = np.ones(3)
    rng = np.random.default_rng(3)
    R = np.stack([_rot(rng) for _ in range(3)])
    p = project(R, np.full(3, model, np.int32), 2 * mu_le * 1e-6 * c, 1e-6 * c, mu * c,
                lam * c, alpha * c)
    assert np.abs(p - R).max() < 1e-12
