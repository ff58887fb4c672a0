"""The frame loop of Alg. 4 (Sec. 6): prediction, detection, Delassus operator and
preconditioner, then local-global iterations constrained by the Fischer-Burmeister
functions, and integration. Two comparison variants of the paper are options: the
minimum-map complementarity functions (App. B.1) and the mass-inverse complementarity
preconditioner r_n = h^2 [H M^-1 H^T]_jj, r_f = h [H M^-1 H^T]_jj (Sec. 5.4).

TEST INFRASTRUCTURE (see the package docstring). Plain FP64.

Readings of the paper used here (the paper leaves these open):
  * q^0 = s~ (the predicted state) and lambda^0 = 0 at the start of every frame;
  * "5 iterations" means exactly n_iters local-global iterations k = 0 .. n_iters - 1;
  * the Schur-complement right-hand side is h^-2 (h - J A^-1 g), the sign of Algs. 3-4
    (eliminating q from Eq. 21 gives this sign; Eq. 22 prints the opposite one);
  * pinned vertices are eliminated (Dirichlet): they are not unknowns and move with the
    scene's handle velocity;
  * the residual used to count iterations (not defined by the paper) is
    R = max_j max(|min(delta_n, r_n lambda_n)|, h |phi_f|) / L, with L the diagonal of the
    rest bounding box. It is one measure for every variant: r from the Delassus diagonal
    and phi_f with the Fischer-Burmeister E_f, whichever complementarity function and
    preconditioner drive the iteration;
  * friction is active when r_n lambda_n > ACTIVE_REL * L (``contact.friction_active``;
    App. B.1-B.2 write lambda_n > 0), decided with the Delassus r_n for every variant;
  * anchors (bilateral constraints, App. A.1-B): each ties a free vertex to a target moving
    at constant velocity (its position at the frame's end time) by the three rows
    e_x, e_y, e_z of phi_b = H_b q - d_b + e lambda_b, always active (Omega = 1), with
    compliance E_b = e entering the Schur system as E_b / h^2 and right-hand side
    -phi_b + J_b q^k like a normal row (Eqs. 19-21); they count in the residual with
    max |phi_b| / L;
  * the Jacobi global step (Sec. 8's comparison of complete and incomplete global solves) is
    for scenes without contact: the Schur complement needs A^-1 itself;
  * ADMM-PD (the paper's implementation follows Overby et al. 2017; Sec. 7): the scaled
    dual variables u_i start at 0 every frame; per iteration z_i = prox of V_i psi_i with
    weight w_i at G_i q + u_i, u_i += G_i q - z_i, and the global step reads z_i - u_i.
    Its fixed point is stationary for the true incremental potential
    |q - s~|_M^2 / (2 h^2) + sum_i V_i psi_i(G_i q), where the plain local step's is
    stationary for the relaxed one (equal for ARAP);
  * the mass-inverse preconditioner, like the Delassus one, uses H (not J = Omega H, which
    depends on r) and gives the two friction rows h times the mean of their diagonal
    entries.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import contact as C
from .fem import FEM
from scenegen import MODEL_ARAP, MODEL_COROT

from .local import elastic_energy, membrane_energy, project, project_membrane


@dataclass
class OracleOptions:
    n_iters: int = 5
    n_cr: int = 10
    exact_constraint_solve: bool = False   # dense solve instead of CR (isolates CR error)
    ncp: str = "fb"                        # "fb" (App. B.2) or "minmap" (App. B.1)
    local: str = "pd"                      # "pd" (Eq. 5) or "admm" (ADMM-PD, Sec. 7)
    global_solver: str = "direct"          # "direct" (A^-1 b) or "jacobi" (the comparison
    jacobi_sweeps: int = 1                 #  of Sec. 8's convergence figure: sweeps from q^k)
    precond: str = "delassus"              # "delassus" (Eq. 28) or "mass" (Sec. 5.4)


class Oracle:
    def __init__(self, scene):
        self.scene = scene
        self.fem = FEM(scene)
        self.h = float(scene.h)
        self.g = np.asarray(scene.gravity, dtype=np.float64)
        self.L_ref = scene.bbox_diagonal
        self.body_data = None
        if getattr(scene, "body_contact", False):
            free = np.zeros(scene.n_verts, dtype=bool)
            free[self.fem.free_verts] = True
            self.body_data = (free, C.mesh_bodies(scene.n_verts, scene.tets),
                              C.surface_triangles(scene.X, scene.tets))

    # -- pieces of Alg. 4 ---------------------------------------------------------------
    def predict(self, q_t, v_t):
        """s~ = q_t + h v_t + h^2 M^-1 f_ext (Eq. 1) with f_ext = M g."""
        return q_t + self.h * v_t + self.h ** 2 * self.g[None, :]

    def pinned_positions(self, q_t):
        """End-of-frame positions of the pinned vertices, in increasing vertex order (the
        order of the columns of A_fp), whatever the order of the scene's pinned list."""
        return (q_t[self.fem.pin_verts] + self.h * np.asarray(self.scene.handle_vel)[None, :])

    def local_step(self, q):
        """p_i = project(G_i q) for every element (Eq. 5): the tetrahedra's (T, 3, 3), then,
        with a triangle sheet, the membranes' 3 x 2 values after them (one flat vector)."""
        f = self.fem
        p = (project(f.deformation_gradients(q), f.model, f.w, f.V, f.emu, f.elam, f.alpha)
             if f.T else np.zeros((0, 3, 3)))
        if not f.Nt:
            return p
        pt = project_membrane(f.triangle_gradients(q), f.t_model, f.t_w, f.t_V, f.t_mu,
                              f.t_lam)
        return np.concatenate([p.reshape(-1), pt.reshape(-1)])

    def jacobi(self, b, x, sweeps):
        """The incomplete global step of the comparison in Sec. 8's convergence figure:
        Jacobi sweeps x <- D^-1 (b - (A - D) x) on A_ff x = b, from the current iterate."""
        A = self.fem.A_ff
        dinv = 1.0 / A.diagonal()
        for _ in range(sweeps):
            x = x + dinv * (b - A @ x)
        return x

    def admm_local_step(self, q, u):
        """ADMM-PD's local step with scaled dual variables u (one 3x3 per element): z_i the
        proximal point of V_i psi_i with weight w_i at G_i q + u_i, then
        u_i <- u_i + G_i q - z_i; the global step reads p_i = z_i - u_i. Returns (p, u).
        ARAP elements use their energy mu ||F - R||^2 (co-rotational with lambda = 0), not
        the SO(3) indicator of the plain local step."""
        f = self.fem
        F = f.deformation_gradients(q)
        arap = f.model == MODEL_ARAP
        model = np.where(arap, MODEL_COROT, f.model)
        lam = np.where(arap, 0.0, f.elam)
        z = project(F + u, model, f.w, f.V, f.emu, lam, f.alpha)
        u = u + F - z
        return z - u, u

    def contact_jacobian(self, contacts):
        """H (3c x 3n_f): rows n_j, f1_j, f2_j at the DoFs of contact j's vertex (Eqs. 36-37);
        a contact with another body has them also at its triangle's corners, times -w_k."""
        f = self.fem
        pos = {int(v): i for i, v in enumerate(f.free_verts)}
        c = len(contacts)
        H = np.zeros((3 * c, 3 * len(f.free_verts)))
        for j, ct in enumerate(contacts):
            D = np.stack([ct["n"], ct["f1"], ct["f2"]])
            k = pos[ct["vertex"]]
            H[3 * j:3 * j + 3, 3 * k:3 * k + 3] += D
            for vk, w in ct.get("corners", ()):
                k = pos[vk]
                H[3 * j:3 * j + 3, 3 * k:3 * k + 3] -= w * D
        return H

    def delassus(self, H):
        """W = H A^-1 H^T (Eq. 27) from direct solves."""
        if H.shape[0] == 0:
            return np.zeros((0, 0))
        X = self.fem.solve(H.T.copy())
        return H @ X

    def preconditioner(self, W, c):
        """r_n = h^2 W_jj on normal rows, r_f = h W_jj on friction rows (Eq. 28); the two
        friction rows share h * mean(W_f1f1, W_f2f2)."""
        d = np.diag(W).reshape(c, 3) if c else np.zeros((0, 3))
        return self.h ** 2 * d[:, 0], self.h * 0.5 * (d[:, 1] + d[:, 2])

    def mass_preconditioner(self, H, c):
        """r_n = h^2 [H M^-1 H^T]_jj on normal rows, r_f = h [H M^-1 H^T]_jj on friction rows
        (the mass-inverse alternative of Sec. 5.4); M is the lumped mass of the free DoFs."""
        if c == 0:
            return np.zeros(0), np.zeros(0)
        minv = 1.0 / np.repeat(self.fem.mass[self.fem.free_verts], 3)
        d = ((H * H) @ minv).reshape(c, 3)
        return self.h ** 2 * d[:, 0], self.h * 0.5 * (d[:, 1] + d[:, 2])

    def contact_state(self, q_f, q_t_f, lam, H, contacts, r_n, r_f, ncp="fb", r_act=None):
        """Gaps, indicators, compliances and NCP values at (q^k, lambda^k) (Alg. 4, "Evaluate
        Omega, J, E, g, h"; Eq. 40 for delta_n and h delta_dot_f) with the Fischer-Burmeister
        (App. B.2) or minimum-map (App. B.1) functions. r_act: the Delassus-diagonal r_n of
        the friction activity test (default r_n)."""
        if r_act is None:
            r_act = r_n
        normal_terms, friction_terms = C.NCP_TERMS[ncp]
        c = len(contacts)
        h = self.h
        Hq = (H @ q_f).reshape(c, 3)
        Hqt = (H @ q_t_f).reshape(c, 3)
        out = dict(omega=np.zeros((c, 3)), E=np.zeros((c, 3)), phi=np.zeros((c, 3)),
                   delta_n=np.zeros(c), vel_f=np.zeros((c, 2)),
                   bilateral=np.array([bool(ct.get("anchor")) for ct in contacts], dtype=bool))
        for j, ct in enumerate(contacts):
            if ct.get("anchor"):
                phi, om, E = C.bilateral_terms(Hq[j] - ct["target"], lam[j], ct["compliance"])
                out["omega"][j], out["E"][j], out["phi"][j] = om, E, phi
                out["delta_n"][j] = Hq[j, 0] - ct["target"][0]
                continue
            dn = Hq[j, 0] - ct["d_n"]
            vf = ((Hq[j, 1:] - Hqt[j, 1:]) - h * ct["d_f"]) / h
            phi_n, om_n, E_n = normal_terms(dn, lam[j, 0], r_n[j])
            act = C.friction_active(lam[j, 0], r_act[j], self.L_ref)
            om_f, E_f, phi_f = friction_terms(vf, lam[j, 1:], lam[j, 0], ct["mu"], r_f[j], act)
            out["omega"][j] = (om_n, om_f, om_f)
            out["E"][j] = (E_n, E_f, E_f)
            out["phi"][j] = (phi_n, phi_f[0], phi_f[1])
            out["delta_n"][j] = dn
            out["vel_f"][j] = vf
        return out

    def residual(self, cs, lam, r_n):
        """max_j max(|min(delta_n, r_n lambda_n)|, h |phi_f|) / L_ref (dimensionless); an
        anchor counts with max_r |phi_r| / L_ref."""
        if len(r_n) == 0:
            return 0.0
        rn = np.abs(np.minimum(cs["delta_n"], r_n * lam[:, 0]))
        rf = self.h * np.linalg.norm(cs["phi"][:, 1:], axis=1)
        res = np.maximum(rn, rf)
        b = cs["bilateral"]
        res[b] = np.abs(cs["phi"][b]).max(axis=1)
        return float(res.max() / self.L_ref)

    # -- one frame --------------------------------------------------------------------
    def frame(self, q_t, v_t, opts: OracleOptions = OracleOptions(), lam0=None, dq0=None,
              t=0.0):
        """Advance (q_t, v_t) by one frame starting at time t (the anchors' targets move with
        time). Returns (q_new, v_new, info)."""
        f = self.fem
        h = self.h
        fv = f.free_verts
        s_tilde = self.predict(q_t, v_t)
        q_pin = self.pinned_positions(q_t)
        contacts = C.detect(self.scene, s_tilde, fv, t + h, self.body_data)
        c = len(contacts)
        if c and opts.global_solver == "jacobi":
            raise ValueError("the Jacobi global step is for scenes without contact")
        H = self.contact_jacobian(contacts)
        W = self.delassus(H)
        r_n, r_f = self.preconditioner(W, c)                 # also the residual's scale
        if opts.precond == "delassus":
            rp_n, rp_f = r_n, r_f
        elif opts.precond == "mass":
            rp_n, rp_f = self.mass_preconditioner(H, c)
        else:
            raise ValueError("precond must be 'delassus' or 'mass'")
        if opts.ncp not in C.NCP_TERMS:
            raise ValueError("ncp must be 'fb' or 'minmap'")
        plain = opts.ncp == "fb" and opts.precond == "delassus"

        def measure(q_f, cs, lam):
            if not plain:
                cs = self.contact_state(q_f, q_t_f, lam, H, contacts, r_n, r_f)
            return self.residual(cs, lam, r_n), cs

        q = s_tilde.copy()
        q[f.pin_verts] = q_pin
        if dq0 is not None:
            q[fv] += dq0[fv]
        lam = np.zeros((c, 3)) if lam0 is None else np.array(lam0, dtype=np.float64)
        q_t_f = q_t[fv].reshape(-1)
        residuals = []
        lam_iters = []                     # lambda at each residual's iterate
        if opts.local not in ("pd", "admm"):
            raise ValueError("local must be 'pd' or 'admm'")
        if opts.local == "admm" and f.Nt:
            raise ValueError("ADMM-PD is for tetrahedra only")
        if opts.global_solver not in ("direct", "jacobi"):
            raise ValueError("global_solver must be 'direct' or 'jacobi'")
        u = np.zeros((f.T, 3, 3))          # ADMM-PD duals, zero at every frame start
        for _k in range(opts.n_iters):
            if opts.local == "admm":
                p, u = self.admm_local_step(q, u)                        # ADMM-PD
            else:
                p = self.local_step(q)                                   # local step
            b = f.assemble_rhs(s_tilde, p, q_pin)                        # RHS (Eq. 6)
            q_f = q[fv].reshape(-1)
            if c:
                cs = self.contact_state(q_f, q_t_f, lam, H, contacts, rp_n, rp_f, opts.ncp, r_n)
                residuals.append(measure(q_f, cs, lam)[0])
                lam_iters.append(lam.copy())
                Om = cs["omega"].reshape(-1)
                J = Om[:, None] * H                                      # J = Omega H (Eq. 25)
                g = b + h ** 2 * (J.T @ lam.reshape(-1))                 # Eq. 19
                # friction rows are velocity-level (h phi_f, E_f / h); an anchor's three
                # rows are position-level like a normal row (App. B, bilateral items)
                lev = np.where(cs["bilateral"][:, None], 1.0, np.array([1.0, h, h])[None, :])
                hv = -(lev * cs["phi"]).reshape(-1) + J @ q_f            # Eq. 19
                Ecal = (cs["E"] / (h * np.where(cs["bilateral"][:, None], h,
                                                np.array([h, 1.0, 1.0])[None, :]))).reshape(-1)
                K = Om[:, None] * W * Om[None, :] + np.diag(Ecal)        # Eq. 26 + E
                rhs = (hv - J @ f.solve(g)) / h ** 2                     # Alg. 4 sign of the RHS
                if opts.exact_constraint_solve:
                    dlam = np.linalg.solve(K, rhs)
                else:
                    dlam = C.conjugate_residual(lambda x: K @ x, rhs, opts.n_cr)
                lam = lam + dlam.reshape(c, 3)                           # Eq. 23a
                omega_last = cs["omega"]
                q_f = f.solve(b + h ** 2 * (J.T @ lam.reshape(-1)))      # Eq. 23b
            elif opts.global_solver == "jacobi":
                q_f = self.jacobi(b, q[fv].reshape(-1), opts.jacobi_sweeps)
            else:
                q_f = f.solve(b)                                         # Eq. 6
            q = q.copy()
            q[fv] = q_f.reshape(-1, 3)
        info = dict(contacts=contacts, lam=lam, W=W, r_n=r_n, r_f=r_f, rp_n=rp_n, rp_f=rp_f,
                    s_tilde=s_tilde, H=H)
        if c and opts.n_iters:
            info["omega_last"] = omega_last
        if c:
            q_f = q[fv].reshape(-1)
            cs = self.contact_state(q_f, q_t_f, lam, H, contacts, rp_n, rp_f, opts.ncp, r_n)
            res, cs = measure(q_f, cs, lam)
            residuals.append(res)
            lam_iters.append(lam.copy())
            info["final_state"] = cs
        info["residuals"] = residuals
        info["lam_iters"] = lam_iters
        v_new = (q - q_t) / h
        return q, v_new, info

    # -- diagnostics --------------------------------------------------------------------
    def energy(self, q, v):
        """Kinetic + elastic (element's own psi) + gravitational energy."""
        f = self.fem
        F = f.deformation_gradients(q)
        kin = 0.5 * float((f.mass[:, None] * v * v).sum())
        ela = elastic_energy(F, f.model, f.V, f.emu, f.elam, f.alpha) if f.T else 0.0
        if f.Nt:
            ela += membrane_energy(f.triangle_gradients(q), f.t_model, f.t_V, f.t_mu, f.t_lam)
            ela += 0.5 * float((q * (f.K_bend @ q)).sum())
        grav = -float((f.mass[:, None] * q * self.g[None, :]).sum())
        return kin + ela + grav

    def max_penetration(self, q):
        worst = 0.0
        for v in self.fem.free_verts:
            for ob in self.scene.obstacles:
                phi, _, _ = C.closest_point(ob, q[v])
                worst = max(worst, -phi)
        return worst
