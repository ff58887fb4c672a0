"""Rest-shape data, the deformation-gradient operator G, lumped masses and the PD system
matrix A = M + h^2 sum_i w_i G_i^T G_i (Sec. 3.3, Eq. 6).

TEST INFRASTRUCTURE (see the package docstring). Plain FP64.

Conventions used throughout the oracle:
  * the 3n position vector is vertex-major: q[3 v + r] is coordinate r of vertex v;
  * F_i = D_s D_m^-1 with D_s = [x1 - x0, x2 - x0, x3 - x0]; F is flattened row-major,
    F[3 r + c];
  * G_i is the explicit 9 x 3n sparse block with F_i = G_i q. It is built entry by entry
    from D_m^-1; the oracle never uses the fact that G acts identically on x, y and z.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from scenegen import MODEL_SNH


def lame(E, nu):
    """Lame parameters (mu, lambda) of linear elasticity from Young's modulus and Poisson's
    ratio."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def snh_parameters(E, nu):
    """Stable Neo-Hookean parameters (Smith, de Goes and Kim 2018): the energy
    mu/2 (I_C - 3) + lam/2 (J - alpha)^2 - mu/2 log(I_C + 1) with mu = 4/3 mu_LE,
    lam = lam_LE + 5/6 mu_LE (so that it linearises to linear elasticity with the given E,
    nu) and alpha = 1 + 3 mu / (4 lam) (so that the rest shape is stress free)."""
    mu_le, lam_le = lame(E, nu)
    mu = 4.0 / 3.0 * mu_le
    lam = lam_le + 5.0 / 6.0 * mu_le
    alpha = 1.0 + 0.75 * mu / lam
    return mu, lam, alpha


def rest_data(X, tets):
    """D_m (T,3,3), its inverse and the rest volumes V_i = det(D_m)/6."""
    Dm = np.stack([X[tets[:, 1]] - X[tets[:, 0]],
                   X[tets[:, 2]] - X[tets[:, 0]],
                   X[tets[:, 3]] - X[tets[:, 0]]], axis=2)        # columns are edges
    V = np.linalg.det(Dm) / 6.0
    if np.any(V <= 0):
        raise ValueError("inverted or degenerate rest tetrahedron")
    return Dm, np.linalg.inv(Dm), V


def gradient_operator(X, tets):
    """Sparse G (9T x 3n) with F_i (row-major) = G[9i:9i+9] q.

    F_rc = sum_a x_{a,r} g_{a,c}, where g_a (a = 1..3) is row a-1 of D_m^-1 and
    g_0 = -(g_1 + g_2 + g_3). Hence G[9i + 3r + c, 3 v_a + r] = g_{a,c}.
    """
    n = X.shape[0]
    T = tets.shape[0]
    _, Dm_inv, _ = rest_data(X, tets)
    g = np.empty((T, 4, 3))
    g[:, 1:, :] = Dm_inv
    g[:, 0, :] = -Dm_inv.sum(axis=1)
    rows, cols, vals = [], [], []
    for a in range(4):
        for r in range(3):
            for c in range(3):
                rows.append(9 * np.arange(T) + 3 * r + c)
                cols.append(3 * tets[:, a] + r)
                vals.append(g[:, a, c])
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(9 * T, 3 * n))
    return G


class FEM:
    """Everything the frame loop needs that depends only on the rest shape and h."""

    def __init__(self, scene):
        self.scene = scene
        X, tets = scene.X, scene.tets
        n, T = X.shape[0], tets.shape[0]
        self.n, self.T = n, T
        self.h = float(scene.h)
        self.Dm, self.Dm_inv, self.V = rest_data(X, tets)
        mats = scene.materials
        mid = scene.tet_material
        E = np.array([mats[m].E for m in mid])
        nu = np.array([mats[m].nu for m in mid])
        self.rho = np.array([mats[m].rho for m in mid])
        self.model = np.array([mats[m].model for m in mid], dtype=np.int32)
        self.mu, self.lam = lame(E, nu)
        smu, slam, salpha = snh_parameters(E, nu)
        snh = self.model == MODEL_SNH
        # per-element energy parameters (mu, lam) as used by psi; alpha for SNH only
        self.emu = np.where(snh, smu, self.mu)
        self.elam = np.where(snh, slam, self.lam)
        self.alpha = np.where(snh, salpha, 0.0)
        # PD weight: w_i = 2 mu V_i for every material (ARAP: the energy mu V ||F - R||^2)
        self.w = 2.0 * self.mu * self.V
        # lumped mass: a quarter of each incident element's mass
        m = np.zeros(n)
        np.add.at(m, tets.ravel(), np.repeat(self.rho * self.V / 4.0, 4))
        if np.any(m <= 0):
            raise ValueError("vertex without mass")
        self.mass = m
        self.G = gradient_operator(X, tets)
        M3 = sp.diags(np.repeat(m, 3))
        Wd = sp.diags(np.repeat(self.w, 9))
        self.A = (M3 + self.h ** 2 * (self.G.T @ Wd @ self.G)).tocsc()
        # Dirichlet elimination of pinned vertices: unknowns are the free DoFs
        pinned = np.zeros(n, dtype=bool)
        pinned[scene.pinned] = True
        self.pinned_mask = pinned
        self.free_verts = np.nonzero(~pinned)[0]
        self.free_dofs = (3 * self.free_verts[:, None] + np.arange(3)).ravel()
        self.pin_dofs = (3 * np.nonzero(pinned)[0][:, None] + np.arange(3)).ravel()
        self.A_ff = self.A[self.free_dofs][:, self.free_dofs].tocsc()
        self.A_fp = self.A[self.free_dofs][:, self.pin_dofs].tocsc()
        self._lu = None

    # -- the plain definition of the global solve ------------------------------------
    def solve(self, rhs):
        """x = A_ff^-1 rhs by a direct sparse LU of the full 3n_f x 3n_f matrix."""
        if self._lu is None:
            import scipy.sparse.linalg as sla
            self._lu = sla.splu(self.A_ff, permc_spec="MMD_AT_PLUS_A",
                                options={"SymmetricMode": True}, diag_pivot_thresh=0.0)
        return self._lu.solve(np.asarray(rhs, dtype=np.float64))

    def deformation_gradients(self, q):
        """F_i = G_i q for all elements, shape (T, 3, 3)."""
        return (self.G @ q.reshape(-1)).reshape(self.T, 3, 3)

    def assemble_rhs(self, s_tilde, p, q_pinned):
        """b = M s~ + h^2 sum_i w_i G_i^T p_i (Eq. 6), restricted to the free DoFs, with the
        pinned vertices' prescribed positions moved to the right-hand side."""
        full = (np.repeat(self.mass, 3) * s_tilde.reshape(-1)
                + self.h ** 2 * (self.G.T @ (np.repeat(self.w, 9) * p.reshape(-1))))
        b = full[self.free_dofs]
        if len(self.pin_dofs):
            b = b - self.A_fp @ q_pinned.reshape(-1)
        return b
