"""Pins of the oracle's FEM layer (G, masses, A) against facts fixed by the mathematics.

The system matrix is A = M + h^2 sum_i w_i G_i^T G_i (Eq. 6); F_i = G_i q is the
deformation gradient of element i.
"""
import math

import numpy as np
import pytest

import scenegen as sg
from oracle.fem import FEM, gradient_operator, lame, rest_data, snh_parameters


def test_gradient_operator_reproduces_affine_maps():
    # any affine deformation x -> M x + t has F = M in every element, exactly
    sc = sg.cube_drop(m=4)
    rng = np.random.default_rng(0)
    M = rng.normal(size=(3, 3))
    t = rng.normal(size=3)
    q = sc.X @ M.T + t
    G = gradient_operator(sc.X, sc.tets)
    F = (G @ q.reshape(-1)).reshape(-1, 3, 3)
    assert np.abs(F - M[None]).max() < 1e-12


def test_volumes_sum_to_cube_volume_and_mass():
    sc = sg.cube_drop(m=5, edge=0.2, rho=750.0)
    _, _, V = rest_data(sc.X, sc.tets)
    assert abs(V.sum() - 0.2 ** 3) < 1e-15
    fem = FEM(sc)
    assert abs(fem.mass.sum() - 750.0 * 0.2 ** 3) < 1e-12


def test_lame_parameters_textbook_values():
    # E = 1, nu = 0.25 -> mu = 0.4, lambda = 0.4 (mu = E / (2 (1 + nu)))
    mu, lam = lame(1.0, 0.25)
    assert abs(mu - 0.4) < 1e-15 and abs(lam - 0.4) < 1e-15


def test_system_matrix_symmetric_positive_definite():
    fem = FEM(sg.cube_drop(m=4))
    A = fem.A.toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_rigid_translations_see_only_the_mass():
    # sum_a g_a = 0, so G maps a uniform translation to zero: A t = M t
    fem = FEM(sg.cube_drop(m=4))
    for r in range(3):
        t = np.zeros((fem.n, 3))
        t[:, r] = 1.0
        lhs = fem.A @ t.reshape(-1)
        rhs = np.repeat(fem.mass, 3) * t.reshape(-1)
        assert np.abs(lhs - rhs).max() < 1e-10 * fem.mass.max()


def test_regular_tet_affine_modes_are_eigenvectors():
    # For a regular tet centred at the origin with edge e, barycentric gradients are
    # 3 x_a / (4 R^2) with R^2 = 3 e^2 / 8, so G^T G u = (2 / e^2) u on linear fields.
    e = 0.1
    sc = sg.single_tet(edge=e)
    fem = FEM(sc)
    rng = np.random.default_rng(1)
    B = rng.normal(size=(3, 3))
    u = sc.X @ B.T
    GtG = (fem.G.T @ fem.G).toarray()
    assert np.allclose(GtG @ u.reshape(-1), 2.0 / e ** 2 * u.reshape(-1), rtol=1e-12, atol=0)


def test_snh_parameters_rest_stress_free_and_linearise():
    # stable Neo-Hookean: gradient zero at F = I and small-strain energy equals linear
    # elasticity mu_LE ||eps||^2 + lam_LE / 2 tr(eps)^2 (checked by finite differences
    # of the F-space energy, computed here from I_C and det F directly).
    E, nu = 3.0e5, 0.41
    mu, lam, alpha = snh_parameters(E, nu)
    mu_le, lam_le = lame(E, nu)

    def psi(F):
        ic = np.trace(F.T @ F)
        J = np.linalg.det(F)
        return 0.5 * mu * (ic - 3) + 0.5 * lam * (J - alpha) ** 2 - 0.5 * mu * math.log(ic + 1)

    eps = 1e-5
    grad = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            d = np.zeros((3, 3))
            d[i, j] = eps
            grad[i, j] = (psi(np.eye(3) + d) - psi(np.eye(3) - d)) / (2 * eps)
    assert np.abs(grad).max() < 1e-6 * mu
    rng = np.random.default_rng(2)
    S = rng.normal(size=(3, 3))
    S = 0.5 * (S + S.T) * 1e-4
    lin = mu_le * np.sum(S * S) + 0.5 * lam_le * np.trace(S) ** 2
    assert abs(psi(np.eye(3) + S) - psi(np.eye(3)) - lin) < 1e-3 * lin


@pytest.mark.parametrize("model", [sg.MODEL_ARAP, sg.MODEL_COROT, sg.MODEL_SNH])
def test_weights_are_two_mu_volume(model):
    sc = sg.cube_drop(m=3, model=model, E=2e5, nu=0.3)
    fem = FEM(sc)
    mu = 2e5 / (2 * 1.3)
    assert np.allclose(fem.w, 2 * mu * fem.V, rtol=1e-14)
