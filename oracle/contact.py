"""Contacts: detection and linearisation (App. A.1), Fischer-Burmeister complementarity
functions and their derivatives (Eq. 14; App. B.2, Eqs. 52-57), the minimum-map
alternative the paper compares against (App. B.1), split indicators (Eq. 24) and the
conjugate-residual constraint solver (Sec. 6).

TEST INFRASTRUCTURE (see the package docstring). Plain FP64.

Readings of the paper used here (the paper leaves these open):
  * detection runs once per frame on the predicted state s~; a vertex/obstacle pair is a
    contact when the signed distance is below the scene's contact margin; the contact
    frame is frozen for the frame (Sec. 5.3: H depends only on the detection);
  * normal n: the obstacle's outward normal at the closest surface point p^;
    d_n = n . p^ (Eq. 36); tangents: f1 from Gram-Schmidt of the world axis least
    aligned with n (lowest index on ties), f2 = n x f1; d_f = f . u^ with u^ the obstacle
    surface velocity (Eq. 37);
  * friction is isotropic: |lambda_f| and |delta_dot_f| are Euclidean norms over (f1, f2),
    each contact has one scalar friction compliance E_f applied to both rows;
  * phi_f = omega_f delta_dot_f + E_f lambda_f (Eq. 55 with J_f v read as the indicator
    times the relative tangential velocity);
  * degenerate cases: if sqrt(delta_n^2 + r^2 lambda_n^2) is zero, omega_n = 1 and
    E_n = 0. With lambda_n > 0: if the E_f numerator vanishes (relative to its scale) the
    contact sticks, E_f = 0; if the denominator is not positive (the iterate lies beyond
    |lambda_f| = 2 mu lambda_n, where Eq. 57 turns negative) E_f takes the slip value of
    the minimum-map form (Eq. 51), (|delta_dot_f| + r (|lambda_f| - mu lambda_n)) /
    (mu lambda_n), which has no fixed point outside the cone. A contact with mu = 0 is
    treated like an inactive one (omega_f = 0, E_f = 1), so its friction force vanishes;
  * friction is active (App. B.1-B.2: lambda_n > 0) when the normal impulse is resolvable:
    r_n lambda_n > ACTIVE_REL * L, with r_n the Delassus-diagonal scale (Eq. 28) and L the
    residual's length scale. When the Newton step drives a separating contact's lambda_n
    to zero it lands on rounding noise of either sign (1e-40 in FP64, 1e-7 of the cancelled
    impulse in FP32); read literally, a positive residue switches on friction with a
    compliance E_f ~ |delta_dot_f| / (mu lambda_n) that swamps the constraint solve and
    makes the residual jump. The tolerance (1e-6 of the scene's length) lies far above both
    noise levels and far below the residual targets (1e-4).
"""
from __future__ import annotations

import numpy as np

from scenegen import OBST_CYLINDER, OBST_PLANE

TINY_REL = 1e-12
ACTIVE_REL = 1e-6


def tangent_frame(n):
    """f1 by Gram-Schmidt of the world axis least aligned with n, f2 = n x f1."""
    n = np.asarray(n, dtype=np.float64)
    k = int(np.argmin(np.abs(n)))
    e = np.zeros(3)
    e[k] = 1.0
    f1 = e - np.dot(e, n) * n
    f1 /= np.linalg.norm(f1)
    f2 = np.cross(n, f1)
    return f1, f2


def closest_point(obst, x):
    """(signed distance, outward unit normal, closest surface point) of x to an obstacle."""
    p = np.asarray(obst.p, dtype=np.float64)
    a = np.asarray(obst.axis, dtype=np.float64)
    if obst.kind == OBST_PLANE:
        phi = float(np.dot(a, x - p))
        return phi, a.copy(), x - phi * a
    if obst.kind == OBST_CYLINDER:
        d = x - p
        axial = np.dot(d, a)
        radial = d - axial * a
        rho = float(np.linalg.norm(radial))
        if rho == 0.0:
            n, _ = tangent_frame(a)          # on the axis: any perpendicular direction
        else:
            n = radial / rho
        return rho - obst.radius, n, p + axial * a + obst.radius * n
    raise ValueError("unknown obstacle kind")


# -- contact between deformable bodies (App. A.1 with a two-sided contact map) ----------
def mesh_bodies(n_verts, tets):
    """Body id of every vertex: the connected components of the tetrahedra, numbered in
    order of their smallest vertex id (a vertex in no element is a body of its own)."""
    parent = list(range(n_verts))

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for t in np.asarray(tets):
        r0 = root(int(t[0]))
        for v in t[1:]:
            r = root(int(v))
            if r != r0:
                parent[max(r, r0)] = min(r, r0)
                r0 = min(r, r0)
    roots = [root(v) for v in range(n_verts)]
    ids = {}
    for r in roots:               # roots are the components' smallest ids, met in order
        ids.setdefault(r, len(ids))
    return np.array([ids[r] for r in roots], dtype=np.int64)


def surface_triangles(X, tets):
    """The faces of the tetrahedra that belong to one element only, each oriented so that
    its normal (b - a) x (c - a) points away from the element (at the rest shape X) and
    rotated to start at its smallest vertex id; sorted by their sorted vertex triples."""
    count, owner = {}, {}
    for t in np.asarray(tets):
        for k in range(4):
            face = tuple(int(t[i]) for i in range(4) if i != k)
            key = tuple(sorted(face))
            count[key] = count.get(key, 0) + 1
            owner[key] = (face, int(t[k]))
    out = []
    for key in sorted(k for k, c in count.items() if c == 1):
        (a, b, c), d = owner[key]
        if np.dot(np.cross(X[b] - X[a], X[c] - X[a]), X[d] - X[a]) > 0:
            b, c = c, b
        tri = [a, b, c]
        i = int(np.argmin(tri))
        out.append(tri[i:] + tri[:i])
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def closest_point_triangle(x, a, b, c):
    """(closest point of the triangle abc to x, its barycentric weights). Inside the
    triangle's projection the point is the orthogonal projection onto the plane; otherwise
    it lies on the boundary, the nearest of the three edges' clamped projections (edges in
    the order ab, bc, ca; the first wins a tie)."""
    e1, e2, r = b - a, c - a, x - a
    G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    u, v = np.linalg.solve(G, np.array([e1 @ r, e2 @ r]))
    if u >= 0.0 and v >= 0.0 and u + v <= 1.0:
        w = np.array([1.0 - u - v, u, v])
        return w[0] * a + w[1] * b + w[2] * c, w
    best = None
    for i, j in ((0, 1), (1, 2), (2, 0)):
        P, Q = (a, b, c)[i], (a, b, c)[j]
        t = float(np.clip((x - P) @ (Q - P) / ((Q - P) @ (Q - P)), 0.0, 1.0))
        p = P + t * (Q - P)
        dist = float(np.linalg.norm(x - p))
        if best is None or dist < best[0]:
            w = np.zeros(3)
            w[i], w[j] = 1.0 - t, t
            best = (dist, p, w)
    return best[1], best[2]


def detect_bodies(scene, s_tilde, free_mask, bodies, tris, id_base):
    """Contacts between the scene's bodies at the predicted positions, one per vertex at
    most: every free vertex of a surface triangle is matched with the nearest surface
    triangle (Euclidean distance to its closest point p; the lowest index on a tie) of
    another body whose corners are all free. The gap g is signed by the triangle's unit
    normal m at s~ where p lies inside the triangle (g = m . (x - p) = +-|x - p|); where p
    is on its boundary (an edge or a corner) x is taken to be outside the other body,
    g = |x - p| (a single face's plane does not tell inside from outside there). The pair
    is a contact when -2 margin < g < margin. Its normal is n = (x - p) / g, the direction
    of the distance (m itself when x = p): above the triangle's interior that is m, at an
    edge or a corner it does not depend on which of the triangles sharing it was taken. The map is x_v - sum_k w_k x_k (w the closest point's barycentric weights, a
    corner with w_k = 0 dropped), the frame (n, f1, f2), d_n = d_f = 0 (the other body's
    motion is in the map itself). Returns {vertex: contact} with the id id_base + triangle
    index."""
    margin = float(scene.contact_margin)
    surf = np.unique(tris)
    ok_tri = np.all(free_mask[tris], axis=1)
    out = {}
    for v in surf:
        if not free_mask[v]:
            continue
        x = s_tilde[v]
        best = None
        for t in np.nonzero(ok_tri & (bodies[tris[:, 0]] != bodies[v]))[0]:
            a, b, c = (s_tilde[k] for k in tris[t])
            p, w = closest_point_triangle(x, a, b, c)
            d = float(np.linalg.norm(x - p))
            if best is None or d < best[0]:
                best = (d, t, p, w)
        if best is None:
            continue
        d, t, p, w = best
        a, b, c = (s_tilde[k] for k in tris[t])
        m = np.cross(b - a, c - a)
        m /= np.linalg.norm(m)
        inside = bool(np.all(w > 0.0))
        g = float(m @ (x - p)) if inside else d
        if not (-2.0 * margin < g < margin):
            continue
        n = (x - p) / g if d > 0.0 else m
        phi = float(n @ (x - p))
        f1, f2 = tangent_frame(n)
        corners = [(int(tris[t][k]), float(w[k])) for k in range(3) if w[k] != 0.0]
        out[int(v)] = dict(vertex=int(v), obstacle=id_base + int(t), n=n, f1=f1, f2=f2,
                           d_n=0.0, d_f=np.zeros(2), mu=float(scene.body_mu), gap=phi,
                           corners=corners, body=True)
    return out


def detect(scene, s_tilde, free_verts, t_end=0.0, body_data=None):
    """All (vertex, obstacle) pairs with signed distance below the contact margin at the
    predicted positions, ordered by vertex id then obstacle index; then, at its vertex, each
    anchor (a bilateral constraint, App. A.1's b rows) with the id n_obstacles + its index,
    its target at time t_end (the end of the frame) and the world axes as its three rows (an
    anchor with a partner vertex is a two-vertex row: its map is q_v - q_partner, the
    partner a corner of weight 1, and its target an offset);
    then, with body_data = (free mask, bodies, surface triangles), the vertex's contact with
    another body (detect_bodies) with the id n_obstacles + n_anchors + triangle index."""
    body_ct = {}
    if body_data is not None:
        n_ids = len(scene.obstacles) + len(getattr(scene, "anchors", []))
        body_ct = detect_bodies(scene, s_tilde, *body_data, n_ids)
    out = []
    anchor_of = {int(a.vertex): i for i, a in enumerate(getattr(scene, "anchors", []))}
    n_obs = len(scene.obstacles)
    for v in free_verts:
        for oi, ob in enumerate(scene.obstacles):
            phi, n, ph = closest_point(ob, s_tilde[v])
            if phi < scene.contact_margin:
                f1, f2 = tangent_frame(n)
                u = np.asarray(ob.vel, dtype=np.float64)
                out.append(dict(vertex=int(v), obstacle=oi, n=n, f1=f1, f2=f2,
                                d_n=float(np.dot(n, ph)),
                                d_f=np.array([np.dot(f1, u), np.dot(f2, u)]),
                                mu=float(ob.mu), gap=phi))
        a = anchor_of.get(int(v))
        if a is not None:
            an = scene.anchors[a]
            target = np.asarray(an.target, float) + t_end * np.asarray(an.vel, float)
            eye = np.eye(3)
            row = dict(vertex=int(v), obstacle=n_obs + a, n=eye[0], f1=eye[1], f2=eye[2],
                       anchor=True, target=target, compliance=float(an.compliance),
                       d_n=float(target[0]), d_f=np.zeros(2), mu=0.0, gap=0.0)
            partner = int(getattr(an, "partner", -1))
            if partner >= 0:
                row["corners"] = [(partner, 1.0)]
            out.append(row)
        if int(v) in body_ct:
            out.append(body_ct[int(v)])
    return out


def bilateral_terms(delta, lam, e):
    """The three rows of an anchor (App. B, bilateral constraints: J_b q - d_b + E_b lambda_b
    = 0): phi = delta + e lambda, indicator 1 and compliance e on every row."""
    phi = np.asarray(delta, float) + e * np.asarray(lam, float)
    return phi, np.ones(3), np.full(3, float(e))


# -- Fischer-Burmeister (App. B.2) ------------------------------------------------------
def fb(a, b):
    """phi_FB(a, b) = a + b - sqrt(a^2 + b^2) (Eq. 14)."""
    return a + b - np.sqrt(a * a + b * b)


def normal_terms(delta_n, lam_n, r_n):
    """phi_n (Eq. 52), the split indicator omega_n (Eqs. 53, 24) and the compliance E_n
    (Eq. 54) of one normal row."""
    rho = np.sqrt(delta_n * delta_n + r_n * r_n * lam_n * lam_n)
    phi = delta_n + r_n * lam_n - rho
    if rho == 0.0:
        return phi, 1.0, 0.0
    omega = 1.0 - delta_n / rho
    E = (1.0 - r_n * lam_n / rho) * r_n
    return phi, omega, E


def friction_active(lam_n, r_n, L):
    """Whether a contact's friction rows are active: r_n lambda_n > ACTIVE_REL * L."""
    return r_n * lam_n > ACTIVE_REL * L


def friction_terms(vel_f, lam_f, lam_n, mu, r_f, active=None):
    """omega_f (Eqs. 56, 24), the scalar compliance E_f (Eq. 57) and phi_f (Eq. 55) of one
    contact's two friction rows. vel_f is the tangential relative velocity delta_dot_f;
    active: the friction_active decision (default lambda_n > 0)."""
    if active is None:
        active = lam_n > 0.0
    if not active or mu <= 0.0:
        return 0.0, 1.0, np.array(lam_f, dtype=np.float64)
    a = float(np.linalg.norm(vel_f))
    lf = float(np.linalg.norm(lam_f))
    s = mu * lam_n - lf
    root = np.sqrt(a * a + r_f * r_f * s * s)
    num = root - r_f * s
    den = a + mu * r_f * lam_n - root
    scale = a + mu * r_f * lam_n + r_f * abs(s)
    if num <= TINY_REL * scale:
        E = 0.0                                   # sticking: no tangential velocity allowed
    elif den <= TINY_REL * scale:
        E = (a + r_f * (lf - mu * lam_n)) / (mu * lam_n)   # far outside the cone: Eq. 51
    else:
        E = num / den * r_f
    return 1.0, E, vel_f + E * np.asarray(lam_f)


# -- minimum map (App. B.1) ---------------------------------------------------------
def minmap_normal_terms(delta_n, lam_n, r_n):
    """phi_n = min(delta_n, r_n lambda_n) with its indicator and compliance (App. B.1): on
    the gap branch (delta_n <= r_n lambda_n, ties included) phi_n = delta_n, omega_n = 1,
    E_n = 0; on the impulse branch phi_n = r_n lambda_n, omega_n = 0, E_n = r_n."""
    if delta_n <= r_n * lam_n:
        return delta_n, 1.0, 0.0
    return r_n * lam_n, 0.0, r_n


def minmap_friction_terms(vel_f, lam_f, lam_n, mu, r_f, active=None):
    """omega_f, the scalar compliance E_f and phi_f = omega_f delta_dot_f + E_f lambda_f of
    the minimum-map friction rows (App. B.1). Inactive contacts (lambda_n <= 0, or mu = 0)
    as in the Fischer-Burmeister form. Active ones, with s = mu lambda_n - |lambda_f|: stick
    (E_f = 0) while |delta_dot_f| <= r_f s, else the slip compliance
    (|delta_dot_f| - r_f s) / (mu lambda_n). active: as in friction_terms."""
    if active is None:
        active = lam_n > 0.0
    if not active or mu <= 0.0:
        return 0.0, 1.0, np.array(lam_f, dtype=np.float64)
    a = float(np.linalg.norm(vel_f))
    s = mu * lam_n - float(np.linalg.norm(lam_f))
    if a <= r_f * s:
        E = 0.0
    else:
        E = (a - r_f * s) / (mu * lam_n)
    return 1.0, E, vel_f + E * np.asarray(lam_f)


NCP_TERMS = {"fb": (normal_terms, friction_terms),
             "minmap": (minmap_normal_terms, minmap_friction_terms)}


# -- conjugate residual --------------------------------------------------------------
def conjugate_residual(apply, b, n_iter):
    """Unpreconditioned conjugate residual for a symmetric operator, x0 = 0, exactly
    n_iter iterations (stopping early only if the residual or search direction vanishes)."""
    x = np.zeros_like(b)
    r = b.copy()
    if not np.any(r):
        return x
    Ar = apply(r)
    p = r.copy()
    Ap = Ar.copy()
    rAr = float(r @ Ar)
    for _ in range(n_iter):
        ApAp = float(Ap @ Ap)
        if ApAp == 0.0:
            break
        alpha = rAr / ApAp
        x += alpha * p
        r -= alpha * Ap
        if not np.any(r):
            break
        Ar = apply(r)
        rAr_new = float(r @ Ar)
        beta = rAr_new / rAr if rAr != 0.0 else 0.0
        rAr = rAr_new
        p = r + beta * p
        Ap = Ar + beta * Ap
    return x
