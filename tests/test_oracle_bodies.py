"""Pins of the oracle's contact between deformable bodies: a vertex against the nearest
surface triangle of another body, the map x_v - sum_k w_k x_k (App. A.1's contact map with
the other body's motion inside it)."""
import numpy as np

import scenegen as sg
from oracle import Oracle, OracleOptions
from oracle import contact as C


def test_closest_point_on_a_triangle_against_brute_force():
    rng = np.random.default_rng(3)
    s = np.linspace(0.0, 1.0, 401)
    U, V = np.meshgrid(s, s)
    keep = U + V <= 1.0
    U, V = U[keep], V[keep]
    for _ in range(40):
        a, b, c = rng.normal(size=(3, 3))
        x = rng.normal(size=3) * 1.5
        p, w = C.closest_point_triangle(x, a, b, c)
        assert abs(w.sum() - 1.0) < 1e-12 and w.min() >= 0.0
        assert np.abs(w[0] * a + w[1] * b + w[2] * c - p).max() < 1e-12
        pts = a[None] + U[:, None] * (b - a)[None] + V[:, None] * (c - a)[None]
        d_brute = np.linalg.norm(pts - x[None], axis=1).min()
        d = np.linalg.norm(x - p)
        assert d <= d_brute + 1e-12
        assert d_brute - d < 3e-3 * np.linalg.norm(np.cross(b - a, c - a)) ** 0.5
    # the regions: above the interior, past a vertex, past an edge
    a, b, c = np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    p, w = C.closest_point_triangle(np.array([0.2, 0.3, 0.7]), a, b, c)
    assert np.allclose(p, [0.2, 0.3, 0.0]) and np.allclose(w, [0.5, 0.2, 0.3])
    p, w = C.closest_point_triangle(np.array([-1.0, -2.0, 0.5]), a, b, c)
    assert np.allclose(p, a) and np.allclose(w, [1.0, 0, 0])
    p, w = C.closest_point_triangle(np.array([0.5, -1.0, 0.0]), a, b, c)
    assert np.allclose(p, [0.5, 0, 0]) and w[2] == 0.0


def test_surface_of_a_lattice_box_is_closed_and_outward():
    m, edge = 4, 0.3
    X, tets = sg.lattice_tets(m, m, m, edge / (m - 1))
    tris = C.surface_triangles(X, tets)
    assert len(tris) == 12 * (m - 1) ** 2
    a, b, c = X[tris[:, 0]], X[tris[:, 1]], X[tris[:, 2]]
    an = 0.5 * np.cross(b - a, c - a)                       # area-weighted normals
    assert np.abs(an.sum(0)).max() < 1e-14                  # a closed surface
    # divergence theorem with the field x: (1/3) sum_t area n . centroid = volume > 0
    vol = (an * (a + b + c) / 3.0).sum() / 3.0
    assert abs(vol - edge ** 3) < 1e-14
    assert np.all(tris[:, 0] < tris[:, 1]) and np.all(tris[:, 0] < tris[:, 2])


def test_bodies_are_the_connected_components():
    sc = sg.box_stack(n_boxes=3, m=3)
    b = C.mesh_bodies(sc.n_verts, sc.tets)
    assert list(b) == [0] * 27 + [1] * 27 + [2] * 27


def test_facing_vertices_of_stacked_boxes_are_in_contact():
    # aligned boxes, flat ground: the upper box's bottom face and the lower box's top face
    # touch across the stack gap (closed form: each vertex's gap is the stack gap)
    for gap, expect in ((0.25, 2 * 16), (0.6, 0)):
        sc = sg.box_stack(n_boxes=2, m=4, offset=0.0, incline_deg=0.0, gap=gap)
        o = Oracle(sc)
        cts = [c for c in sg_contacts(o, sc) if c.get("body")]
        assert len(cts) == expect
        for c in cts:
            assert abs(c["gap"] - gap * sc.spacing) < 1e-12
            assert abs(abs(c["n"][2]) - 1.0) < 1e-12


def sg_contacts(o, sc):
    s = o.predict(sc.q0, np.zeros_like(sc.q0))
    return C.detect(sc, s, o.fem.free_verts, o.h, o.body_data)


def _forces_on(o, info, verts):
    """Sum over the given vertices of the contact force H^T (omega lambda)."""
    H = o.contact_jacobian(info["contacts"])
    lam = (info["omega_last"] * info["lam"]).reshape(-1)
    F = (H.T @ lam).reshape(-1, 3)
    pos = {int(v): i for i, v in enumerate(o.fem.free_verts)}
    return sum(F[pos[int(v)]] for v in verts)


def test_contact_between_bodies_conserves_momentum():
    # two boxes driven into each other without gravity or ground: the contact forces are
    # internal, so the total momentum is unchanged, and each body's momentum changes by the
    # force the map puts on its own vertices (the -w_k share on a triangle's corners)
    sc = sg.box_stack(n_boxes=2, m=3, incline_deg=0.0, gap=0.1, seed=2)
    sc.obstacles = []
    sc.gravity = (0.0, 0.0, 0.0)
    v0 = np.zeros_like(sc.X)
    v0[:27, 2], v0[27:, 2] = 1.0, -1.0
    o = Oracle(sc)
    q, v, info = o.frame(sc.q0, v0, OracleOptions(n_iters=8))
    m = o.fem.mass[:, None]
    assert info["lam"][:, 0].max() > 1.0
    p0 = np.abs(m * v0).sum()
    assert np.abs((m * v).sum(0) - (m * v0).sum(0)).max() < 1e-9 * p0
    s_tilde = info["s_tilde"]
    for verts in (np.arange(27), np.arange(27, 54)):
        lhs = (m[verts] * (q[verts] - s_tilde[verts])).sum(0)
        rhs = sc.h ** 2 * _forces_on(o, info, verts)
        assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(rhs).max()


def test_resting_stack_carries_the_weights():
    # two boxes on flat ground come to rest: the ground's normal impulses carry both boxes,
    # the contacts between the boxes carry the upper one
    sc = sg.box_stack(n_boxes=2, m=3, incline_deg=0.0, gap=0.1, offset=0.1, seed=4, E=1e6)
    o = Oracle(sc)
    q, v = sc.q0.copy(), np.zeros_like(sc.q0)
    for _ in range(60):
        q, v, info = o.frame(q, v, OracleOptions(n_iters=25))
    mass = o.fem.mass
    g = 9.81
    ground = [j for j, c in enumerate(info["contacts"]) if not c.get("body")]
    assert abs(info["lam"][ground, 0].sum() - mass.sum() * g) < 1e-4 * mass.sum() * g
    up = _forces_on(o, info, np.arange(27, 54))
    assert abs(up[2] - mass[27:].sum() * g) < 1e-4 * mass[27:].sum() * g
    assert np.abs(v).max() < 1e-3


def test_stack_on_an_incline_sticks_or_slides_by_coulombs_law():
    # two boxes on a 20 degree incline: with mu = 0.8 > tan 20 the stack holds; with
    # mu = 0.2 < tan 20 on the ground (and 0.8 between the boxes) it slides as one body with
    # the acceleration g (sin - mu cos) of a block on a slope
    th = np.radians(20.0)
    down = np.array([np.cos(th), 0.0, -np.sin(th)])     # down the slope (plane turned about y)
    for mu_ground, moving in ((0.8, False), (0.2, True)):
        sc = sg.box_stack(n_boxes=2, m=3, incline_deg=20.0, gap=0.1, offset=0.1, seed=5,
                          E=1e6, mu=0.8)
        sc.obstacles[0].mu = mu_ground
        o = Oracle(sc)
        q, v = sc.q0.copy(), np.zeros_like(sc.q0)
        for _ in range(30):
            q, v, info = o.frame(q, v, OracleOptions(n_iters=25))
        m = o.fem.mass
        vs = (m[:, None] * v).sum(0) @ down / m.sum()
        if moving:
            a = 9.81 * (np.sin(th) - mu_ground * np.cos(th))
            assert abs(vs - a * 30 * sc.h) < 0.1 * a * 30 * sc.h, vs
            v_rel = v[27:] @ down - v[:27] @ down
            assert np.abs(v_rel).max() < 0.02 * abs(vs)
        else:
            assert abs(vs) < 1e-3, vs
