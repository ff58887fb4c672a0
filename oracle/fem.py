"""Rest-shape data, the deformation-gradient operator G, lumped masses and the PD system
matrix A = M + h^2 sum_i w_i G_i^T G_i (Sec. 3.3, Eq. 6), for tetrahedra and for triangle
(membrane) elements, plus the constant Laplace-Beltrami bending term of a triangle sheet.

TEST INFRASTRUCTURE (see the package docstring). Plain FP64.

Conventions used throughout the oracle:
  * the 3n position vector is vertex-major: q[3 v + r] is coordinate r of vertex v;
  * F_i = D_s D_m^-1 with D_s = [x1 - x0, x2 - x0, x3 - x0]; F is flattened row-major,
    F[3 r + c];
  * G_i is the explicit 9 x 3n sparse block with F_i = G_i q. It is built entry by entry
    from D_m^-1; the oracle never uses the fact that G acts identically on x, y and z;
  * a triangle's F is 3 x 2: [x1 - x0, x2 - x0] D_m^-1 with D_m the 2 x 2 rest edges in the
    triangle's own plane (first axis along x1 - x0), flattened row-major F[2 r + c]; its
    "volume" is area x thickness and its weight 2 mu V like a tetrahedron's;
  * bending (Laplace-Beltrami, flat rest shape): E_b = k_b/2 sum over interior vertices
    of |(L x)_i|^2 / A_i with L the cotangent Laplacian (L_ij = -(cot a_ij + cot b_ij)/2) and
    A_i the mixed Voronoi area of the vertex; it is quadratic in x and adds
    h^2 k_b L^T diag(interior / A) L (per coordinate) to A. Its minimisers are the flat
    sheet's rigid and in-plane motions (L annihilates affine fields at interior vertices).
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


def triangle_rest_data(X, tris):
    """Per triangle: the 2 x 2 rest edge matrix D_m in the triangle's plane, its inverse and
    the area."""
    e1 = X[tris[:, 1]] - X[tris[:, 0]]
    e2 = X[tris[:, 2]] - X[tris[:, 0]]
    l1 = np.linalg.norm(e1, axis=1)
    a1 = e1 / l1[:, None]
    nrm = np.cross(e1, e2)
    area = 0.5 * np.linalg.norm(nrm, axis=1)
    if np.any(area <= 0):
        raise ValueError("degenerate rest triangle")
    a2 = np.cross(nrm / (2.0 * area)[:, None], a1)
    Dm = np.zeros((len(tris), 2, 2))
    Dm[:, 0, 0] = l1
    Dm[:, 0, 1] = (e2 * a1).sum(1)
    Dm[:, 1, 1] = (e2 * a2).sum(1)
    return Dm, np.linalg.inv(Dm), area


def triangle_gradient_operator(X, tris):
    """Sparse G (6 Nt x 3n) with F_i (row-major 3 x 2) = G[6i:6i+6] q; g_a (a = 1, 2) is row
    a-1 of D_m^-1 and g_0 = -(g_1 + g_2): G[6i + 2r + c, 3 v_a + r] = g_{a,c}."""
    n, Nt = X.shape[0], tris.shape[0]
    _, Dm_inv, _ = triangle_rest_data(X, tris)
    g = np.empty((Nt, 3, 2))
    g[:, 1:, :] = Dm_inv
    g[:, 0, :] = -Dm_inv.sum(axis=1)
    rows, cols, vals = [], [], []
    for a in range(3):
        for r in range(3):
            for c in range(2):
                rows.append(6 * np.arange(Nt) + 2 * r + c)
                cols.append(3 * tris[:, a] + r)
                vals.append(g[:, a, c])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(6 * Nt, 3 * n))


def bending_matrix(X, tris, k_b):
    """K (n x n) = k_b L^T diag(interior / A) L: the cotangent Laplacian of the rest sheet,
    the per-vertex mixed Voronoi area (Meyer et al. 2003: a non-obtuse triangle gives each
    corner its Voronoi part (|PR|^2 cot Q + |PQ|^2 cot R) / 8, an obtuse one half its area to
    the obtuse corner and a quarter to the others), interior vertices only (a boundary edge
    belongs to one triangle)."""
    n = X.shape[0]
    W = sp.lil_matrix((n, n))
    A = np.zeros(n)
    edges = {}
    for t in tris:
        P = X[t]
        area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        cots = np.zeros(3)
        for k in range(3):
            i, j, o = t[k], t[(k + 1) % 3], t[(k + 2) % 3]
            u, v = X[i] - X[o], X[j] - X[o]
            cot = float(u @ v) / np.linalg.norm(np.cross(u, v))
            cots[(k + 2) % 3] = cot            # the angle at o
            W[i, j] += 0.5 * cot
            W[j, i] += 0.5 * cot
            key = (min(i, j), max(i, j))
            edges[key] = edges.get(key, 0) + 1
        obtuse = [k for k in range(3) if cots[k] < 0]
        for k in range(3):
            if obtuse:
                A[t[k]] += area / 2 if k in obtuse else area / 4
            else:
                kn, kp = (k + 1) % 3, (k + 2) % 3
                A[t[k]] += (np.sum((P[kp] - P[k]) ** 2) * cots[kn]
                            + np.sum((P[kn] - P[k]) ** 2) * cots[kp]) / 8.0
    W = W.tocsr()
    L = sp.diags(np.asarray(W.sum(axis=1)).ravel()) - W
    boundary = np.zeros(n, dtype=bool)
    for (i, j), cnt in edges.items():
        if cnt == 1:
            boundary[[i, j]] = True
    used = A > 0
    dinv = np.where(used & ~boundary, 1.0 / np.where(used, A, 1.0), 0.0)
    return (k_b * (L.T @ sp.diags(dinv) @ L)).tocsr()


class FEM:
    """Everything the frame loop needs that depends only on the rest shape and h."""

    def __init__(self, scene):
        self.scene = scene
        X, tets = scene.X, scene.tets
        tris = getattr(scene, "tris", None)
        tris = np.zeros((0, 3), np.int32) if tris is None else np.asarray(tris).reshape(-1, 3)
        n, T, Nt = X.shape[0], tets.shape[0], tris.shape[0]
        self.n, self.T, self.Nt = n, T, Nt
        self.h = float(scene.h)
        if T:
            self.Dm, self.Dm_inv, self.V = rest_data(X, tets)
        else:
            self.Dm, self.Dm_inv, self.V = np.zeros((0, 3, 3)), np.zeros((0, 3, 3)), np.zeros(0)
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
        # lumped mass: a quarter of each incident tetrahedron's mass, a third of each
        # incident triangle's
        m = np.zeros(n)
        np.add.at(m, tets.ravel(), np.repeat(self.rho * self.V / 4.0, 4))
        # triangles (membranes): area x thickness as volume, the same weights
        tm = np.asarray(getattr(scene, "tri_material", np.zeros(Nt, np.int32)), dtype=np.int32)
        self.t_model = np.array([mats[k].model for k in tm], dtype=np.int32)
        self.t_mu, self.t_lam = lame(np.array([mats[k].E for k in tm]),
                                     np.array([mats[k].nu for k in tm]))
        t_rho = np.array([mats[k].rho for k in tm])
        if Nt:
            _, self.t_Dm_inv, area = triangle_rest_data(X, tris)
            self.t_V = area * float(scene.thickness)
            if np.any(self.t_V <= 0):
                raise ValueError("a triangle sheet needs a positive thickness")
        else:
            self.t_Dm_inv, self.t_V = np.zeros((0, 2, 2)), np.zeros(0)
        self.t_w = 2.0 * self.t_mu * self.t_V
        np.add.at(m, tris.ravel(), np.repeat(t_rho * self.t_V / 3.0, 3))
        if np.any(m <= 0):
            raise ValueError("vertex without mass")
        self.mass = m
        G_tet = gradient_operator(X, tets) if T else sp.csr_matrix((0, 3 * n))
        G_tri = triangle_gradient_operator(X, tris) if Nt else sp.csr_matrix((0, 3 * n))
        self.G_tet, self.G_tri = G_tet, G_tri
        self.G = sp.vstack([G_tet, G_tri]).tocsr()
        self.wvec = np.concatenate([np.repeat(self.w, 9), np.repeat(self.t_w, 6)])
        M3 = sp.diags(np.repeat(m, 3))
        Wd = sp.diags(self.wvec)
        self.K_bend = (bending_matrix(X, tris, float(getattr(scene, "bending", 0.0)))
                       if Nt and getattr(scene, "bending", 0.0) > 0 else sp.csr_matrix((n, n)))
        K3 = sp.kron(self.K_bend, sp.eye(3)).tocsr()
        self.A = (M3 + self.h ** 2 * (self.G.T @ Wd @ self.G + K3)).tocsc()
        # Dirichlet elimination of pinned vertices: unknowns are the free DoFs
        pinned = np.zeros(n, dtype=bool)
        pinned[scene.pinned] = True
        self.pinned_mask = pinned
        self.free_verts = np.nonzero(~pinned)[0]
        self.free_dofs = (3 * self.free_verts[:, None] + np.arange(3)).ravel()
        self.pin_verts = np.nonzero(pinned)[0]          # increasing vertex order
        self.pin_dofs = (3 * self.pin_verts[:, None] + np.arange(3)).ravel()
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
        """F_i = G_i q for all tetrahedra, shape (T, 3, 3)."""
        return (self.G_tet @ q.reshape(-1)).reshape(self.T, 3, 3)

    def triangle_gradients(self, q):
        """F_i = G_i q for all triangles, shape (Nt, 3, 2)."""
        return (self.G_tri @ q.reshape(-1)).reshape(self.Nt, 3, 2)

    def assemble_rhs(self, s_tilde, p, q_pinned):
        """b = M s~ + h^2 sum_i w_i G_i^T p_i (Eq. 6), restricted to the free DoFs, with the
        pinned vertices' prescribed positions q_pinned (rows in increasing vertex order,
        pin_verts) moved to the right-hand side. p holds the tetrahedra's 9 values then the
        triangles' 6 per element (the bending term has no projection: its rest curvature is
        zero)."""
        full = (np.repeat(self.mass, 3) * s_tilde.reshape(-1)
                + self.h ** 2 * (self.G.T @ (self.wvec * p.reshape(-1))))
        b = full[self.free_dofs]
        if len(self.pin_dofs):
            b = b - self.A_fp @ q_pinned.reshape(-1)
        return b
