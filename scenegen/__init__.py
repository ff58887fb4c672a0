"""Seeded synthetic scenes: tetrahedral lattices, material tables, obstacles, initial states.

This module is shared by the FP64 oracle tests and by the CUDA path's tests and benchmark.
It holds geometry and parameters only (vertex lattices, the Kuhn six-tetrahedron split of a
cell, star-shaped masks, seeded rotations and obstacle layouts). None of the simulator's
arithmetic (masses, gradients, projections, factorisations, contact laws) lives here.

Scene workloads (the paper's meshes are not available, so these stand in for them):

* ``cube_drop``   - an m x m x m vertex cube dropped onto a ground plane (the paper's
  single-body drop tests; Sec. 7).
* ``star_pull``   - an extruded five-point star pulled by a pinned cap through a seeded
  4 x 4 array of fixed cylinders; shaped like the "crossing gingerbread man" teaser scene
  (58.5k DoFs, up to 800 contacts; teaser caption and Tab. 3).
* ``slope_box``   - a stiff box resting on an inclined plane (stick-slip test, Sec. 7.4,
  Fig. 8): the analytic threshold is mu* = tan(theta).
* ``single_tet``  - one regular tetrahedron, for closed-form checks.
* ``batch``       - dozens of cubes of uneven size with mixed materials on tilted planes.
* ``tied_cubes``  - two cubes tied across a gap by two-vertex bilateral rows (App. A.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MODEL_ARAP = 0      # projective-dynamics as-rigid-as-possible (SO(3) indicator)
MODEL_COROT = 1     # co-rotational
MODEL_SNH = 2       # stable Neo-Hookean

OBST_PLANE = 0
OBST_CYLINDER = 1

GRAVITY_EARTH = (0.0, 0.0, -9.81)


@dataclass
class Material:
    model: int
    E: float
    nu: float
    rho: float


@dataclass
class Anchor:
    """A bilateral constraint tying a free vertex to a target point: the three rows
    e_x, e_y, e_z of (q_v - target) + compliance * lambda = 0. The target starts at
    ``target`` and moves at ``vel``; compliance (m/N) 0 makes the constraint hard. With
    ``partner`` >= 0 the rows tie the vertex to that vertex instead (App. A.1's two-vertex
    bilateral rows): (q_v - q_partner) - target + compliance * lambda = 0, the target then
    an offset."""
    vertex: int
    target: tuple
    vel: tuple = (0.0, 0.0, 0.0)
    compliance: float = 0.0
    partner: int = -1


@dataclass
class Obstacle:
    """A static analytic obstacle.

    PLANE: ``p`` is a point on the plane, ``axis`` its unit outward normal.
    CYLINDER: infinite cylinder; ``p`` a point on the axis, ``axis`` the unit axis
    direction, ``radius`` its radius. ``mu`` is the Coulomb friction coefficient and
    ``vel`` the obstacle's surface velocity (zero for fixed obstacles).
    """
    kind: int
    p: tuple
    axis: tuple
    radius: float = 0.0
    mu: float = 0.0
    vel: tuple = (0.0, 0.0, 0.0)


@dataclass
class Scene:
    """A complete simulation input. Units are SI. Arrays are float64 / int32."""
    name: str
    X: np.ndarray                  # (n, 3) rest positions
    tets: np.ndarray               # (T, 4) vertex ids, positively oriented at rest
    tet_material: np.ndarray       # (T,) index into materials
    materials: List[Material]
    obstacles: List[Obstacle]
    h: float
    gravity: tuple = GRAVITY_EARTH
    pinned: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    handle_vel: tuple = (0.0, 0.0, 0.0)   # velocity of every pinned vertex
    anchors: List["Anchor"] = field(default_factory=list)   # bilateral vertex targets
    # triangle (membrane) elements: (Nt, 3) vertex ids, their materials, the sheet's
    # thickness (m) and its bending stiffness k_b (N m, Laplace-Beltrami, flat rest)
    tris: Optional[np.ndarray] = None
    tri_material: Optional[np.ndarray] = None
    thickness: float = 0.0
    bending: float = 0.0
    q0: Optional[np.ndarray] = None       # (n, 3) initial positions (default: X)
    v0: Optional[np.ndarray] = None       # (n, 3) initial velocities (default: 0)
    contact_margin: float = 0.0           # a contact exists when the gap is below this
    # contact between the scene's separate bodies (connected components of its tetrahedra):
    # a vertex against the nearest surface triangle of another body, friction body_mu
    body_contact: bool = False
    body_mu: float = 0.0
    n_iters: int = 5                      # local-global iterations per frame
    n_cr: int = 10                        # conjugate-residual iterations per solve
    n_frames: int = 1
    spacing: float = 0.0                  # lattice spacing (informational)

    def __post_init__(self):
        self.X = np.ascontiguousarray(self.X, dtype=np.float64)
        self.tets = np.ascontiguousarray(self.tets, dtype=np.int32).reshape(-1, 4)
        self.tet_material = np.ascontiguousarray(self.tet_material, dtype=np.int32)
        self.tris = np.ascontiguousarray(np.zeros((0, 3)) if self.tris is None else self.tris,
                                         dtype=np.int32).reshape(-1, 3)
        if self.tri_material is None:
            self.tri_material = np.zeros(len(self.tris), np.int32)
        self.tri_material = np.ascontiguousarray(self.tri_material, dtype=np.int32)
        self.pinned = np.ascontiguousarray(self.pinned, dtype=np.int32)
        if self.q0 is None:
            self.q0 = self.X.copy()
        if self.v0 is None:
            self.v0 = np.zeros_like(self.X)
        self.q0 = np.ascontiguousarray(self.q0, dtype=np.float64)
        self.v0 = np.ascontiguousarray(self.v0, dtype=np.float64)

    @property
    def n_verts(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def bbox_diagonal(self) -> float:
        return float(np.linalg.norm(self.X.max(0) - self.X.min(0)))


# --------------------------------------------------------------------------------------
# lattices
# --------------------------------------------------------------------------------------
# corner c of a unit cell has offsets (c & 1, (c >> 1) & 1, (c >> 2) & 1); the six Kuhn
# tetrahedra all share the main diagonal 0 -> 7, so neighbouring cells conform.
_CELL_OFFSETS = [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]
_KUHN = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]


def lattice_tets(nx: int, ny: int, nz: int, spacing: float, keep=None,
                 origin=(0.0, 0.0, 0.0)):
    """Tetrahedralise the cells of an nx x ny x nz vertex lattice.

    ``keep(i, j, k)`` (cell indices) selects cells; unused vertices are dropped. Returns
    (X, tets) with every tetrahedron positively oriented.
    """
    vid = -np.ones((nx, ny, nz), dtype=np.int64)
    cells = []
    for i in range(nx - 1):
        for j in range(ny - 1):
            for k in range(nz - 1):
                if keep is None or keep(i, j, k):
                    cells.append((i, j, k))
    if not cells:
        raise ValueError("empty lattice")
    cells = np.array(cells, dtype=np.int64)
    corner_ijk = cells[:, None, :] + np.array(_CELL_OFFSETS)[None, :, :]      # (C, 8, 3)
    used = np.zeros((nx, ny, nz), dtype=bool)
    used[corner_ijk[..., 0], corner_ijk[..., 1], corner_ijk[..., 2]] = True
    ijk = np.argwhere(used)                                                   # lexicographic
    vid[ijk[:, 0], ijk[:, 1], ijk[:, 2]] = np.arange(len(ijk))
    X = np.asarray(origin, dtype=np.float64) + spacing * ijk.astype(np.float64)
    corner_ids = vid[corner_ijk[..., 0], corner_ijk[..., 1], corner_ijk[..., 2]]  # (C, 8)
    tets = corner_ids[:, np.array(_KUHN)].reshape(-1, 4)
    # orient positively
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    neg = np.linalg.det(d) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return X, tets.astype(np.int32)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix from a seeded generator (unit quaternion)."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _rot_y(deg: float) -> np.ndarray:
    t = math.radians(deg)
    return np.array([[math.cos(t), 0, math.sin(t)], [0, 1, 0], [-math.sin(t), 0, math.cos(t)]])


def _star_polygon(r_out: float, r_in: float, points: int = 5):
    """Vertices of a star polygon with one tip on the +x axis."""
    ang = np.arange(2 * points) * math.pi / points
    rad = np.where(np.arange(2 * points) % 2 == 0, r_out, r_in)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)


def _inside_polygon(px: float, py: float, poly: np.ndarray) -> bool:
    inside = False
    n = len(poly)
    for a in range(n):
        x1, y1 = poly[a]
        x2, y2 = poly[(a + 1) % n]
        if (y1 > py) != (y2 > py):
            xc = x1 + (py - y1) * (x2 - x1) / (y2 - y1)
            if px < xc:
                inside = not inside
    return inside


# --------------------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------------------
def single_tet(edge: float = 0.1, model: int = MODEL_ARAP, E: float = 1e5, nu: float = 0.4,
               rho: float = 1000.0, h: float = 1.0 / 60.0) -> Scene:
    """One regular tetrahedron centred at the origin, no gravity, no obstacles."""
    a = edge / math.sqrt(8.0)
    X = np.array([[a, a, a], [a, -a, -a], [-a, a, -a], [-a, -a, a]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    if np.linalg.det(d[0]) < 0:
        tets = np.array([[0, 2, 1, 3]], dtype=np.int32)
    return Scene("single_tet", X, tets, np.zeros(1, np.int32), [Material(model, E, nu, rho)],
                 [], h, gravity=(0.0, 0.0, 0.0), contact_margin=0.5 * edge, spacing=edge)


def cube_drop(m: int = 6, edge: float = 0.1, model: int = MODEL_ARAP, E: float = 1e5,
              nu: float = 0.4, rho: float = 1000.0, height: float = 0.2, mu: float = 0.5,
              seed: int = 0, h: float = 1.0 / 60.0, n_frames: int = 100,
              tilt_deg: float = 0.0) -> Scene:
    """An m^3-vertex cube (edge ``edge``) with a seeded random rotation, its lowest point
    ``height`` above a ground plane through the origin tilted by ``tilt_deg`` about y."""
    rng = np.random.default_rng(seed)
    sp = edge / (m - 1)
    X, tets = lattice_tets(m, m, m, sp, origin=(-edge / 2, -edge / 2, -edge / 2))
    R = random_rotation(rng)
    q0 = X @ R.T
    n_plane = _rot_y(tilt_deg) @ np.array([0.0, 0.0, 1.0])
    lift = height - (q0 @ n_plane).min()
    q0 = q0 + lift * n_plane
    obst = [Obstacle(OBST_PLANE, (0.0, 0.0, 0.0), tuple(n_plane), mu=mu)]
    return Scene(f"cube{m}", X, tets, np.zeros(len(tets), np.int32), [Material(model, E, nu, rho)],
                 obst, h, q0=q0, contact_margin=0.5 * sp, n_frames=n_frames, spacing=sp)


def slope_box(mu: float, theta_deg: float = 10.0, m: int = 4, edge: float = 0.1,
              E: float = 1e8, nu: float = 0.3, rho: float = 1000.0, model: int = MODEL_ARAP,
              h: float = 1.0 / 60.0, n_iters: int = 10, n_cr: int = 24) -> Scene:
    """A stiff m^3-vertex box whose bottom face rests on a plane inclined by ``theta_deg``
    (about the y axis). Gravity is -z. The analytic stick/slip threshold is tan(theta)."""
    sp = edge / (m - 1)
    X, tets = lattice_tets(m, m, m, sp, origin=(-edge / 2, -edge / 2, 0.0))
    R = _rot_y(theta_deg)
    q0 = X @ R.T
    n_plane = R @ np.array([0.0, 0.0, 1.0])
    obst = [Obstacle(OBST_PLANE, (0.0, 0.0, 0.0), tuple(n_plane), mu=mu)]
    return Scene("slope_box", X, tets, np.zeros(len(tets), np.int32),
                 [Material(model, E, nu, rho)], obst, h, q0=q0, contact_margin=0.5 * sp,
                 n_iters=n_iters, n_cr=n_cr, spacing=sp)


def star_pull(n_side: int = 42, layers: int = 27, spacing: float = 0.01, seed: int = 0,
              E: float = 1e6, nu: float = 0.45, rho: float = 1000.0, model: int = MODEL_SNH,
              mu: float = 0.3, pull_speed: float = 0.5, cap_depth: float = 0.05,
              h: float = 1.0 / 60.0, n_frames: int = 300, start_gap: float = 0.3,
              inner_ratio: float = 0.5) -> Scene:
    """Extruded five-point star pulled through a seeded 4 x 4 array of fixed cylinders.

    Cross-section: a star polygon (inner/outer radius ratio ``inner_ratio``) inscribed in
    an n_side x n_side vertex lattice; extruded along z over ``layers`` vertex layers.
    The vertices within ``cap_depth`` of the leading (+x) tip are pinned and move at
    ``pull_speed`` along +x. Cylinders have axes along z; four columns at an x pitch of
    0.5 m starting ``start_gap`` ahead of the tip; y centres at -0.45, -0.15, 0.15, 0.45 m
    plus U(-0.03, 0.03); radii U(0.02, 0.06) m. No gravity.
    """
    rng = np.random.default_rng(seed)
    r_out = (n_side - 1) * spacing / 2.0
    poly = _star_polygon(r_out, inner_ratio * r_out)
    c0 = (n_side - 1) / 2.0

    def keep(i, j, k):
        return _inside_polygon((i + 0.5 - c0) * spacing, (j + 0.5 - c0) * spacing, poly)

    X, tets = lattice_tets(n_side, n_side, layers, spacing, keep=keep,
                           origin=(-c0 * spacing, -c0 * spacing, 0.0))
    xmax = X[:, 0].max()
    pinned = np.nonzero(X[:, 0] >= xmax - cap_depth - 1e-9)[0].astype(np.int32)
    zc = 0.5 * (layers - 1) * spacing
    obst = []
    for col in range(4):
        x = xmax + start_gap + 0.5 * col
        for yc in (-0.45, -0.15, 0.15, 0.45):
            y = yc + rng.uniform(-0.03, 0.03)
            r = rng.uniform(0.02, 0.06)
            obst.append(Obstacle(OBST_CYLINDER, (x, y, zc), (0.0, 0.0, 1.0), radius=r, mu=mu))
    return Scene(f"star{n_side}x{layers}", X, tets, np.zeros(len(tets), np.int32),
                 [Material(model, E, nu, rho)], obst, h, gravity=(0.0, 0.0, 0.0),
                 pinned=pinned, handle_vel=(pull_speed, 0.0, 0.0),
                 contact_margin=0.5 * spacing, n_frames=n_frames, spacing=spacing)


def star_placed(scene: Scene, placement: float = 0.094):
    """A contact state of a star_pull scene (pure geometry, no simulation): the rest shape
    translated along +x so that its leading face lies ``placement`` metres beyond the axes of
    the first cylinder row, every vertex moving at the pull speed. At 0.094 m on the 43 x 43
    x 27 star (59,778 DoFs) the tips are inside the first row's cylinders: 837 contacts at
    837 distinct vertices on the predicted positions (0.1025 m on the 42 x 42 x 27 star:
    810). Returns (q, v)."""
    q = scene.q0.copy()
    x_front = scene.X[:, 0].max()
    first_col = min(o.p[0] for o in scene.obstacles)
    q[:, 0] += (first_col - x_front) + placement
    v = np.zeros_like(q)
    v[:, 0] = scene.handle_vel[0]
    return q, v


def anchored_handle(scene: Scene, compliance: float = 0.0) -> Scene:
    """The same scene with its pinned handle replaced by anchors: every pinned vertex
    becomes a free vertex tied to a target that starts at its initial position and moves
    with the handle velocity (the bilateral form of the moving positional constraint)."""
    import copy
    sc = copy.deepcopy(scene)
    sc.anchors = [Anchor(int(v), tuple(float(x) for x in scene.q0[v]), tuple(scene.handle_vel),
                         compliance) for v in scene.pinned]
    sc.pinned = np.zeros(0, np.int32)
    sc.name = scene.name + "_anchored"
    return sc


def cloth(n: int = 12, size: float = 0.5, model: int = MODEL_ARAP, E: float = 1e5,
          nu: float = 0.3, rho: float = 200.0, thickness: float = 1e-3, bending: float = 1e-4,
          height: float = 0.3, pin: str = "corners", h: float = 1.0 / 60.0,
          obstacles: Optional[List[Obstacle]] = None, seed: int = 0,
          tilt_deg: float = 0.0) -> Scene:
    """A flat square sheet of n x n vertices (side ``size``, triangles alternating their
    diagonal) in the plane z = height, rotated about the x axis by ``tilt_deg``; ARAP or
    co-rotational membrane with thickness and a Laplace-Beltrami bending stiffness.
    pin: "corners" (the two corners at y = max), "edge" (the row y = max) or "none"."""
    g = np.linspace(-0.5 * size, 0.5 * size, n)
    xx, yy = np.meshgrid(g, g, indexing="ij")
    X = np.stack([xx.ravel(), yy.ravel(), np.zeros(n * n)], axis=1)
    c = math.cos(math.radians(tilt_deg)); sn = math.sin(math.radians(tilt_deg))
    X = X @ np.array([[1, 0, 0], [0, c, sn], [0, -sn, c]]).T
    X[:, 2] += height
    tris = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, cc, d = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
            if (i + j) % 2 == 0:
                tris += [(a, b, cc), (a, cc, d)]
            else:
                tris += [(a, b, d), (b, cc, d)]
    tris = np.array(tris, np.int32)
    if pin == "corners":
        pinned = np.array([n - 1, n * n - 1], np.int32)
    elif pin == "edge":
        pinned = np.array([i * n + n - 1 for i in range(n)], np.int32)
    else:
        pinned = np.zeros(0, np.int32)
    obst = [] if obstacles is None else list(obstacles)
    spacing = size / (n - 1)
    return Scene(f"cloth{n}", X, np.zeros((0, 4), np.int32), np.zeros(0, np.int32),
                 [Material(model, E, nu, rho)], obst, h, pinned=pinned,
                 contact_margin=0.5 * spacing, spacing=spacing, tris=tris,
                 tri_material=np.zeros(len(tris), np.int32), thickness=thickness,
                 bending=bending)


def twisting_bar(nxy: int = 4, nz: int = 16, spacing: float = 0.02, twist_deg: float = 45.0,
                 model: int = MODEL_ARAP, E: float = 1e6, nu: float = 0.45, rho: float = 1000.0,
                 h: float = 1.0 / 60.0) -> Scene:
    """The large-rotation scene of the paper's convergence comparison (Sec. 8): a bar along z
    whose two end layers are pinned, the top one turned by twist_deg about the bar's axis;
    the rest of the bar starts untwisted and at rest, without gravity. The top layer's turn
    shears the elements below it; at 90 degrees some of them start flat (det F = 0, where the
    sign of the rotation is decided by rounding), at the default 45 their smallest singular
    value is 0.28."""
    X, tets = lattice_tets(nxy, nxy, nz, spacing,
                           origin=(-0.5 * (nxy - 1) * spacing, -0.5 * (nxy - 1) * spacing, 0.0))
    zmax = X[:, 2].max()
    bottom = np.nonzero(X[:, 2] < 1e-9)[0]
    top = np.nonzero(X[:, 2] > zmax - 1e-9)[0]
    q0 = X.copy()
    a = math.radians(twist_deg)
    R = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0, 0, 1.0]])
    q0[top] = X[top] @ R.T
    return Scene(f"bar{nxy}x{nz}", X, tets, np.zeros(len(tets), np.int32),
                 [Material(model, E, nu, rho)], [], h, gravity=(0.0, 0.0, 0.0),
                 pinned=np.concatenate([bottom, top]).astype(np.int32), q0=q0,
                 spacing=spacing)


def box_stack(n_boxes: int = 3, m: int = 4, edge: float = 0.1, model: int = MODEL_SNH,
              E: float = 1e8, nu: float = 0.45, rho: float = 1000.0, mu: float = 0.8,
              incline_deg: float = 20.0, gap: float = 0.25, offset: float = 0.2,
              seed: int = 0, h: float = 1.0 / 60.0, n_iters: int = 10) -> Scene:
    """A stack of n_boxes m^3-vertex boxes (edge ``edge``) on a plane inclined by
    ``incline_deg`` about the y axis: each box rests on the one below across a gap of
    ``gap`` lattice spacings (the lowest on the plane), shifted within the plane by a seeded
    offset of up to ``offset`` edges along each axis; friction mu on the plane and between
    the boxes (the stress case's deformable box-box contacts). Rest shape = start."""
    rng = np.random.default_rng(seed)
    sp = edge / (m - 1)
    Xb, tb = lattice_tets(m, m, m, sp, origin=(-edge / 2, -edge / 2, 0.0))
    R = _rot_y(incline_deg)
    Xs, Ts = [], []
    for k in range(n_boxes):
        dx, dy = rng.uniform(-offset, offset, size=2) * edge
        z0 = gap * sp + k * (edge + gap * sp)
        Xs.append((Xb + np.array([dx, dy, z0])) @ R.T)
        Ts.append(tb + k * len(Xb))
    X = np.concatenate(Xs)
    tets = np.concatenate(Ts)
    n_plane = R @ np.array([0.0, 0.0, 1.0])
    obst = [Obstacle(OBST_PLANE, (0.0, 0.0, 0.0), tuple(n_plane), mu=mu)]
    return Scene(f"stack{n_boxes}x{m}", X, tets, np.zeros(len(tets), np.int32),
                 [Material(model, E, nu, rho)], obst, h, contact_margin=0.5 * sp,
                 n_iters=n_iters, spacing=sp, body_contact=True, body_mu=mu)


def stack_stress(copies: int = 8, columns: int = 16, boxes: int = 2, m: int = 12,
                 seed: int = 0) -> List[Scene]:
    """The stress case: copies x (columns x boxes) stiff boxes (SNH, E = 1e8, nu = 0.45) of
    m^3 vertices, mu = 0.8 on a 20 degree incline and between the boxes, 10 local-global
    iterations per frame. Each column of ``boxes`` boxes is a scene of its own (the
    columns stand apart, so they share no contact), with a seeded lateral offset of its
    boxes; the boxes start a twentieth of a lattice spacing into each other and into the
    plane, so that every frame has box-box and box-ground contacts. With the defaults:
    8 x 32 boxes of 12^3 vertices, 128 scenes."""
    return [box_stack(n_boxes=boxes, m=m, model=MODEL_SNH, E=1e8, nu=0.45, mu=0.8,
                      incline_deg=20.0, gap=-0.05, seed=seed * 100003 + k, n_iters=10)
            for k in range(copies * columns)]


def hanging_cube(m: int = 5, edge: float = 0.1, model: int = MODEL_ARAP, E: float = 1e5,
                 nu: float = 0.4, rho: float = 1000.0, compliance: float = 0.0,
                 target_vel=(0.0, 0.0, 0.0), h: float = 1.0 / 60.0, floor: bool = False,
                 mu: float = 0.5) -> Scene:
    """An m^3-vertex cube hanging under gravity from one anchor at the vertex nearest the
    centre of its top face (for odd m right above the centre of mass), optionally above a
    floor plane two edges below the cube."""
    X, tets = lattice_tets(m, m, m, edge / (m - 1))
    c = X.mean(0)
    d = np.abs(X[:, 0] - c[0]) + np.abs(X[:, 1] - c[1]) - 1e3 * X[:, 2]
    top = int(np.argmin(d))
    obst = []
    if floor:
        obst.append(Obstacle(OBST_PLANE, (0.0, 0.0, -2.0 * edge), (0.0, 0.0, 1.0), mu=mu))
    sc = Scene(f"hang{m}", X, tets, np.zeros(len(tets), np.int32), [Material(model, E, nu, rho)],
               obst, h, contact_margin=0.5 * edge / (m - 1), spacing=edge / (m - 1))
    sc.anchors = [Anchor(top, tuple(float(x) for x in X[top]), tuple(target_vel), compliance)]
    return sc


def tied_cubes(m: int = 4, edge: float = 0.1, gap: float = 0.05, model: int = MODEL_ARAP,
               E: float = 1e5, nu: float = 0.4, rho: float = 1000.0, compliance: float = 0.0,
               pull: float = 0.0, h: float = 1.0 / 60.0, floor: bool = True,
               height: float = 0.01, mu: float = 0.5, gravity=GRAVITY_EARTH) -> Scene:
    """Two m^3-vertex cubes side by side along x, ``gap`` apart, tied across the gap by
    two-vertex bilateral rows (App. A.1) between the four corners of the facing faces (each
    row a vertex of cube A against the facing vertex of cube B, target offset their rest
    offset, shrinking at ``pull`` m/s along x: a cable drawing them together); optionally
    ``height`` above a floor plane."""
    Xa, ta = lattice_tets(m, m, m, edge / (m - 1))
    Xb = Xa + np.array([edge + gap, 0.0, 0.0])
    X = np.vstack([Xa, Xb])
    tets = np.vstack([ta, ta + len(Xa)])
    X[:, 2] += height
    lo, hi = Xa[:, 0].min(), Xa[:, 0].max()
    ya, za = Xa[:, 1], Xa[:, 2]
    corners = [i for i in range(len(Xa)) if abs(Xa[i, 0] - hi) < 1e-12 and
               min(abs(ya[i] - ya.min()), abs(ya[i] - ya.max())) < 1e-12 and
               min(abs(za[i] - za.min()), abs(za[i] - za.max())) < 1e-12]
    obst = []
    if floor:
        obst.append(Obstacle(OBST_PLANE, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), mu=mu))
    sc = Scene(f"tied{m}", X, tets, np.zeros(len(tets), np.int32), [Material(model, E, nu, rho)],
               obst, h, gravity=gravity, contact_margin=0.5 * edge / (m - 1),
               spacing=edge / (m - 1))
    for a in corners:
        # the facing vertex of cube B: same y, z on its -x face
        b = len(Xa) + int(np.argmin(np.abs(Xa[:, 0] - lo) * 1e3 + np.abs(ya - ya[a]) +
                                     np.abs(za - za[a])))
        off = X[a] - X[b]
        sc.anchors.append(Anchor(int(a), tuple(float(x) for x in off), (pull, 0.0, 0.0),
                                 compliance, partner=b))
    return sc


def batch(n_scenes: int = 64, seed: int = 0, m_lo: int = 8, m_hi: int = 20,
          h: float = 1.0 / 60.0) -> List[Scene]:
    """Dozens of independent cubes of uneven size: side m ~ U{m_lo..m_hi} vertices, edge
    U(0.1, 0.25) m, materials alternating ARAP/co-rotational versus stable Neo-Hookean, E
    log-uniform in [1e4, 1e7] Pa, nu ~ U(0.3, 0.48), dropped onto planes tilted U(0, 30)
    degrees with mu ~ U(0.1, 0.8)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        m = int(rng.integers(m_lo, m_hi + 1))
        edge = float(rng.uniform(0.1, 0.25))
        if s % 2 == 0:
            model = MODEL_ARAP if (s // 2) % 2 == 0 else MODEL_COROT
        else:
            model = MODEL_SNH
        E = float(10 ** rng.uniform(4, 7))
        nu = float(rng.uniform(0.3, 0.48))
        tilt = float(rng.uniform(0, 30))
        mu = float(rng.uniform(0.1, 0.8))
        sc = cube_drop(m=m, edge=edge, model=model, E=E, nu=nu, height=0.05, mu=mu,
                       seed=seed * 1000 + s, h=h, tilt_deg=tilt)
        sc.name = f"batch{s}_m{m}"
        out.append(sc)
    return out


def warmstart_scenes(seeds, m: int = 6, frames: int = 100) -> List[Scene]:
    """The learned warm start's workload: the 6^3-vertex cube (edge 0.1 m, E = 1e5,
    nu = 0.4), ARAP for even seeds and co-rotational for odd ones, dropped from a seeded
    height in [0.1, 0.3] m with a seeded rotation onto a plane tilted by a seeded angle in
    [0, 20] degrees (mu = 0.5)."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(10_000 + int(s))
        height = float(rng.uniform(0.1, 0.3))
        tilt = float(rng.uniform(0.0, 20.0))
        model = MODEL_ARAP if int(s) % 2 == 0 else MODEL_COROT
        sc = cube_drop(m=m, edge=0.1, model=model, E=1e5, nu=0.4, height=height, mu=0.5,
                       seed=int(s), n_frames=frames, tilt_deg=tilt)
        sc.name = f"ws{s}"
        out.append(sc)
    return out


def perturbed_state(scene: Scene, seed: int, amp: float, vel_amp: float = 0.0):
    """Seeded random perturbation of the initial state (positions and velocities) of the
    free vertices, for single-step comparisons from identical states."""
    rng = np.random.default_rng(seed)
    q = scene.q0 + amp * rng.standard_normal(scene.q0.shape)
    v = scene.v0 + vel_amp * rng.standard_normal(scene.v0.shape)
    if len(scene.pinned):
        q[scene.pinned] = scene.q0[scene.pinned]
        v[scene.pinned] = np.asarray(scene.handle_vel)
    return q, v
