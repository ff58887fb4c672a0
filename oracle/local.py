"""Per-element local projections p_i = argmin_p w_i/2 ||p - F_i||^2 + V_i psi(p) (Sec. 3.3,
Eq. 5), and the elastic energies psi.

TEST INFRASTRUCTURE (see the package docstring). Plain FP64, vectorised over elements.

For an isotropic psi the minimiser shares the singular vectors of F: with the signed SVD
F = U diag(sigma) V^T (U, V rotations, the smallest singular value negative when
det F < 0), p = U diag(sigma_hat) V^T where sigma_hat minimises the same objective over
diagonal matrices.

  * ARAP (PD): psi is the indicator of SO(3) (Eq. 5 discussion), so sigma_hat = (1, 1, 1).
  * co-rotational: psi = mu ||F - R||^2 + lam/2 tr^2(R^T F - I) is quadratic in sigma, the
    sigma-space problem is linear and solved in closed form.
  * stable Neo-Hookean (Smith, de Goes and Kim 2018): Newton's method with a backtracking
    line search in sigma-space, to a gradient tolerance of 1e-12 (relative).
"""
from __future__ import annotations

import numpy as np

from scenegen import MODEL_ARAP, MODEL_COROT, MODEL_SNH


def svd_signed(F):
    """Batched signed SVD: F = U diag(s) Vt with det U = det Vt = +1; the last (smallest)
    singular value carries the sign of det F."""
    U, s, Vt = np.linalg.svd(F)
    U = U.copy()
    s = s.copy()
    Vt = Vt.copy()
    du = np.linalg.det(U) < 0
    U[du, :, 2] *= -1.0
    s[du, 2] *= -1.0
    dv = np.linalg.det(Vt) < 0
    Vt[dv, 2, :] *= -1.0
    s[dv, 2] *= -1.0
    return U, s, Vt


# -- energies in sigma-space ------------------------------------------------------------
def psi_corot(s, mu, lam):
    return mu * ((s - 1.0) ** 2).sum(-1) + 0.5 * lam * (s.sum(-1) - 3.0) ** 2


def psi_snh(s, mu, lam, alpha):
    ic = (s * s).sum(-1)
    J = s.prod(-1)
    return 0.5 * mu * (ic - 3.0) + 0.5 * lam * (J - alpha) ** 2 - 0.5 * mu * np.log(ic + 1.0)


def _snh_grad_hess(s, mu, lam, alpha):
    """Gradient (.., 3) and Hessian (.., 3, 3) of psi_snh with respect to sigma."""
    ic = (s * s).sum(-1)
    J = s.prod(-1)
    dJ = np.stack([s[..., 1] * s[..., 2], s[..., 0] * s[..., 2], s[..., 0] * s[..., 1]], -1)
    mu_ = mu[..., None]
    lam_ = lam[..., None]
    g = mu_ * s + lam_ * (J - alpha)[..., None] * dJ - mu_ * s / (ic + 1.0)[..., None]
    H = np.zeros(s.shape + (3,))
    eye = np.eye(3)
    d2J = np.zeros(s.shape + (3,))
    d2J[..., 0, 1] = d2J[..., 1, 0] = s[..., 2]
    d2J[..., 0, 2] = d2J[..., 2, 0] = s[..., 1]
    d2J[..., 1, 2] = d2J[..., 2, 1] = s[..., 0]
    H += mu[..., None, None] * eye
    H += lam[..., None, None] * (dJ[..., :, None] * dJ[..., None, :]
                                 + (J - alpha)[..., None, None] * d2J)
    ic1 = (ic + 1.0)[..., None, None]
    H -= mu[..., None, None] * (eye / ic1 - 2.0 * s[..., :, None] * s[..., None, :] / ic1 ** 2)
    return g, H


def sigma_corot(s, w, V, mu, lam):
    """Closed-form minimiser of w/2 ||x - s||^2 + V psi_corot(x).

    Stationarity: (w + 2 mu V) x_i + lam V sum(x) = w s_i + 2 mu V + 3 lam V. Summing over
    i gives sum(x); substituting back gives each x_i.
    """
    a = w + 2.0 * mu * V
    c = lam * V
    rhs = w[:, None] * s + (2.0 * mu * V + 3.0 * lam * V)[:, None]
    S = rhs.sum(-1) / (a + 3.0 * c)
    return (rhs - (c * S)[:, None]) / a[:, None]


def sigma_snh(s, w, V, mu, lam, alpha, tol=1e-12, max_iter=200):
    """Minimiser of f(x) = w/2 ||x - s||^2 + V psi_snh(x), by Newton's method from x = s
    with an Armijo backtracking line search. A Hessian that is not positive definite is
    shifted by a multiple of the identity until it is (its smallest eigenvalue is lifted to
    1e-8 of its scale)."""
    x = s.copy()
    done = np.zeros(len(s), dtype=bool)

    def f(xx, idx):
        return (0.5 * w[idx] * ((xx - s[idx]) ** 2).sum(-1)
                + V[idx] * psi_snh(xx, mu[idx], lam[idx], alpha[idx]))

    for _ in range(max_iter):
        idx = np.nonzero(~done)[0]
        if len(idx) == 0:
            break
        xi = x[idx]
        gp, Hp = _snh_grad_hess(xi, mu[idx], lam[idx], alpha[idx])
        g = w[idx, None] * (xi - s[idx]) + V[idx, None] * gp
        H = w[idx, None, None] * np.eye(3) + V[idx, None, None] * Hp
        scale = w[idx] + V[idx] * (mu[idx] + lam[idx])
        conv = np.linalg.norm(g, axis=-1) <= tol * scale * np.maximum(1.0, np.abs(xi).max(-1))
        done[idx[conv]] = True
        keep = ~conv
        idx, xi, g, H, scale = idx[keep], xi[keep], g[keep], H[keep], scale[keep]
        if len(idx) == 0:
            break
        ev = np.linalg.eigvalsh(H)[:, 0]
        shift = np.where(ev <= 1e-8 * scale, 1e-8 * scale - ev, 0.0)
        H = H + shift[:, None, None] * np.eye(3)
        d = -np.linalg.solve(H, g[..., None])[..., 0]
        f0 = f(xi, idx)
        slope = (g * d).sum(-1)
        t = np.ones(len(idx))
        active = np.ones(len(idx), dtype=bool)
        for _ls in range(60):
            if not active.any():
                break
            cand = xi + t[:, None] * d
            # Armijo test with a rounding allowance, so that near the minimum (where f
            # no longer resolves the decrease) the full Newton step is taken
            ok = f(cand, idx) <= f0 + 1e-4 * t * slope + 8e-16 * np.abs(f0)
            active &= ~ok
            t = np.where(active, 0.5 * t, t)
        x[idx] = xi + t[:, None] * d
        # a step that no longer moves the iterate means the tolerance is below rounding
        stalled = np.abs(t[:, None] * d).max(-1) <= 1e-15 * np.maximum(1.0, np.abs(xi).max(-1))
        done[idx[stalled]] = True
    return x


def project(F, model, w, V, mu, lam, alpha):
    """p_i = argmin w_i/2 ||p - F_i||^2 + V_i psi_i(p) for every element (Eq. 5)."""
    U, s, Vt = svd_signed(F)
    sh = np.ones_like(s)
    c = model == MODEL_COROT
    if c.any():
        sh[c] = sigma_corot(s[c], w[c], V[c], mu[c], lam[c])
    k = model == MODEL_SNH
    if k.any():
        sh[k] = sigma_snh(s[k], w[k], V[k], mu[k], lam[k], alpha[k])
    a = model == MODEL_ARAP
    sh[a] = 1.0
    return np.einsum("tij,tj,tjk->tik", U, sh, Vt)


def elastic_energy(F, model, V, mu, lam, alpha):
    """sum_i V_i psi_i(F_i) with psi the element's own material (ARAP: mu ||F - R||^2)."""
    U, s, Vt = svd_signed(F)
    e = np.zeros(len(F))
    a = model == MODEL_ARAP
    e[a] = mu[a] * ((s[a] - 1.0) ** 2).sum(-1)
    c = model == MODEL_COROT
    e[c] = psi_corot(s[c], mu[c], lam[c])
    k = model == MODEL_SNH
    e[k] = psi_snh(s[k], mu[k], lam[k], alpha[k])
    return float((V * e).sum())


# -- membranes (triangle elements, 3 x 2 deformation gradients) -------------------------
def svd_membrane(F):
    """Thin SVD of 3 x 2 deformation gradients: F = U diag(s) V^T with U (3 x 2, orthonormal
    columns), s >= 0, V a 2 x 2 rotation or reflection (a membrane in 3D cannot invert)."""
    U, s, Vt = np.linalg.svd(F, full_matrices=False)
    return U, s, Vt


def sigma_corot2(s, w, V, mu, lam):
    """Closed-form minimiser of w/2 ||x - s||^2 + V (mu ||x - 1||^2 + lam/2 (sum x - 2)^2)
    over the two singular values: (w + 2 mu V) x_i + lam V sum(x) = w s_i + 2 mu V + 2 lam V,
    summed for sum(x), substituted back for each x_i."""
    a = w + 2.0 * mu * V
    c = lam * V
    rhs = w[:, None] * s + (2.0 * mu * V + 2.0 * lam * V)[:, None]
    S = rhs.sum(-1) / (a + 2.0 * c)
    return (rhs - (c * S)[:, None]) / a[:, None]


def project_membrane(F, model, w, V, mu, lam):
    """p_i = argmin w_i/2 ||p - F_i||^2 + V_i psi_i(p) for 3 x 2 membrane gradients (Eq. 5):
    ARAP the closest matrix with orthonormal columns (U V^T), co-rotational the closed form
    above; the stable Neo-Hookean energy is not defined for membranes here."""
    if np.any(model == MODEL_SNH):
        raise ValueError("membranes are ARAP or co-rotational")
    U, s, Vt = svd_membrane(F)
    sh = np.ones_like(s)
    c = model == MODEL_COROT
    if c.any():
        sh[c] = sigma_corot2(s[c], w[c], V[c], mu[c], lam[c])
    return np.einsum("tij,tj,tjk->tik", U, sh, Vt)


def membrane_energy(F, model, V, mu, lam):
    """sum_i V_i psi_i(F_i): mu ||s - 1||^2 (+ lam/2 (sum s - 2)^2 co-rotational)."""
    _, s, _ = svd_membrane(F)
    e = mu * ((s - 1.0) ** 2).sum(-1)
    c = model == MODEL_COROT
    e[c] += 0.5 * lam[c] * (s[c].sum(-1) - 2.0) ** 2
    return float((V * e).sum())
