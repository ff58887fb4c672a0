"""CPU-side tests of the product library: it loads, exports every function the header
declares, and its host precompute (ordering, elimination tree, Cholesky, S~ profile) solves
the PD system exactly (checked against the oracle's direct solve). No GPU is needed."""
import ctypes

import numpy as np
import pytest

import scenegen as sg
from paper_2503_15078_b300 import Plan, SimError, Simulator, _abi, lib
from oracle.fem import FEM


def test_library_exports_every_declared_function():
    L = lib()
    declared = _abi.header_declarations()
    assert len(declared) >= 15
    missing = [name for name in declared if not hasattr(L, name)]
    assert missing == []
    assert set(declared) == set(_abi.PROTOTYPES)


def test_strerror_and_defaults():
    assert lib().sim_strerror(0) == b"ok"
    assert b"capacity" in lib().sim_strerror(-5)
    o = _abi.SimOptions()
    lib().sim_default_options(ctypes.byref(o))
    assert o.n_iters == 5 and o.n_cr_iters == 10 and o.gravity[2] == -9.81


def _oracle_solve(sc, b):
    f = FEM(sc)
    x = np.zeros_like(b)
    x[f.free_verts] = f.solve(b[f.free_verts].reshape(-1)).reshape(-1, 3)
    return x


@pytest.mark.parametrize("maker", [
    lambda: sg.cube_drop(m=6),
    lambda: sg.cube_drop(m=9, model=sg.MODEL_SNH, E=1e7),
    lambda: sg.star_pull(n_side=14, layers=6),
    lambda: sg.single_tet(),
])
def test_host_sparse_inverse_matches_direct_solve(maker):
    sc = maker()
    P = Plan(sc)
    rng = np.random.default_rng(0)
    b = rng.normal(size=(sc.n_verts, 3))
    x = P.apply_inverse_host(b)
    xr = _oracle_solve(sc, b)
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    if len(sc.pinned):
        assert np.all(x[sc.pinned] == 0)


def test_profile_is_the_elimination_subtree():
    # postorder: parent[k] > k, subtrees are the contiguous ranges [fd(k), k], and the
    # stored nnz equals the sum of elimination-tree depths (Theorem 1)
    sc = sg.star_pull(n_side=16, layers=8)
    P = Plan(sc)
    order, parent, fd = P.ordering()
    info = P.info()
    nf = info["n_free"]
    assert sorted(order.tolist()) == sorted(set(range(sc.n_verts)) - set(sc.pinned.tolist()))
    assert np.all((parent == -1) | (parent > np.arange(nf)))
    size = np.ones(nf, int)
    for k in range(nf):
        if parent[k] >= 0:
            size[parent[k]] += size[k]
    assert np.array_equal(fd, np.arange(nf) - size + 1)
    for k in range(nf):
        if parent[k] >= 0:
            assert fd[parent[k]] <= fd[k]
    depth = np.zeros(nf, int)
    for k in range(nf - 1, -1, -1):
        depth[k] = 1 + (depth[parent[k]] if parent[k] >= 0 else 0)
    assert info["nnz_S"] == depth.sum()
    assert info["etree_max_depth"] == depth.max()


def test_ordering_reduces_fill():
    # nested dissection keeps S~ far from the dense triangle on a 3D lattice
    P = Plan(sg.cube_drop(m=12))
    info = P.info()
    n = info["n_free"]
    assert info["nnz_S"] < 0.35 * n * (n + 1) / 2


@pytest.mark.parametrize("bad", ["inverted", "index", "material", "h"])
def test_invalid_inputs_are_rejected(bad):
    sc = sg.cube_drop(m=3)
    h = sc.h
    if bad == "inverted":
        sc.tets = sc.tets.copy()
        sc.tets[0, [1, 2]] = sc.tets[0, [2, 1]]
    elif bad == "index":
        sc.tets = sc.tets.copy()
        sc.tets[3, 2] = sc.n_verts + 5
    elif bad == "material":
        sc.materials = [sg.Material(sg.MODEL_SNH, 1e5, 0.5, 1000.0)]
    else:
        h = -1.0
    with pytest.raises(SimError) as e:
        Plan(sc, h=h)
    assert e.value.status == -1


def test_create_without_a_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(SimError) as e:
        Simulator(sg.cube_drop(m=3))
    assert e.value.status == -4


@pytest.mark.parametrize("opts", [{"s_precision": 2}, {"s_precision": -1}, {"refine": 3},
                                  {"refine": -1}, {"n_iters": 65}, {"contact_capacity": 0},
                                  {"ncp": 2}, {"ncp": -1}, {"precond": 2},
                                  {"residual_tol": -1.0}, {"residual_tol": float("nan")},
                                  {"max_iters": 0}, {"max_iters": 64},
                                  {"local_solver": 2}])
def test_invalid_options_are_rejected_before_any_device_work(opts):
    with pytest.raises(SimError) as e:
        Simulator(sg.cube_drop(m=3), **opts)
    assert e.value.status == -1


def test_named_options_map_to_the_abi_values():
    from paper_2503_15078_b300 import _options
    o = _options(sg.cube_drop(m=3), ncp="minmap", precond="mass")
    assert (o.ncp, o.precond) == (1, 1)
    o = _options(sg.cube_drop(m=3))
    assert (o.ncp, o.precond) == (0, 0)
    with pytest.raises(ValueError):
        _options(None, ncp="newton")


@pytest.mark.parametrize("bad", ["pinned", "range", "twice", "compliance"])
def test_invalid_anchors_are_rejected(bad):
    sc = sg.hanging_cube(m=3)
    a = sc.anchors[0]
    if bad == "pinned":
        sc.pinned = np.array([a.vertex], np.int32)
    elif bad == "range":
        a.vertex = sc.n_verts
    elif bad == "twice":
        sc.anchors.append(sg.Anchor(a.vertex, a.target))
    else:
        a.compliance = -1.0
    with pytest.raises(SimError) as e:
        Simulator(sc)
    assert e.value.status == -1


@pytest.mark.parametrize("bad", ["self", "range", "pinned"])
def test_invalid_pair_rows_are_rejected(bad):
    # a two-vertex row's partner: another free vertex of the same scene
    sc = sg.tied_cubes(m=3)
    a = sc.anchors[0]
    if bad == "self":
        a.partner = a.vertex
    elif bad == "range":
        a.partner = sc.n_verts
    else:
        sc.pinned = np.array([a.partner], np.int32)
    with pytest.raises(SimError) as e:
        Simulator(sc)
    assert e.value.status == -1


def test_allocator_hooks_must_come_in_pairs():
    with pytest.raises(SimError) as e:
        Simulator(sg.cube_drop(m=3), dev_alloc=lambda n, c: None)
    assert e.value.status == -1


@pytest.mark.parametrize("bend,model,tilt", [(1e-4, sg.MODEL_COROT, 0.0), (0.0, sg.MODEL_ARAP, 20.0),
                                             (3e-4, sg.MODEL_ARAP, 35.0)])
def test_host_profile_solve_of_a_sheet_equals_the_direct_solve(bend, model, tilt):
    # the host plan's system matrix with membranes and bending, through x = S^T (S b)
    from oracle.fem import FEM
    sc = sg.cloth(n=9, model=model, bending=bend, tilt_deg=tilt, pin="corners")
    p = Plan(sc)
    f = FEM(sc)
    b = np.random.default_rng(0).normal(size=(sc.n_verts, 3))
    x = p.apply_inverse_host(b)
    xr = np.zeros_like(b)
    xr[f.free_verts] = f.solve(b[f.free_verts].reshape(-1)).reshape(-1, 3)
    assert np.linalg.norm(x - xr) < 1e-12 * np.linalg.norm(xr)


@pytest.mark.parametrize("bad", ["snh", "thickness", "admm"])
def test_invalid_sheets_are_rejected(bad):
    sc = sg.cloth(n=5)
    kw = {}
    if bad == "snh":
        sc.materials = [sg.Material(sg.MODEL_SNH, 1e5, 0.3, 200.0)]
    elif bad == "thickness":
        sc.thickness = 0.0
    else:
        kw["local_solver"] = "admm"
    with pytest.raises(SimError) as e:
        Simulator(sc, **kw)
    assert e.value.status == -1


def test_jacobi_global_step_needs_a_scene_without_contact():
    with pytest.raises(SimError) as e:
        Simulator(sg.cube_drop(m=3), global_solver="jacobi")
    assert e.value.status == -1
    with pytest.raises(SimError) as e:
        Simulator(sg.twisting_bar(nxy=3, nz=4), global_solver="jacobi", jacobi_sweeps=0)
    assert e.value.status == -1


def test_body_contact_options_are_checked():
    sc = sg.box_stack(n_boxes=2, m=3)
    for field, bad in (("body_mu", -0.1), ("body_mu", float("nan"))):
        s2 = sg.box_stack(n_boxes=2, m=3)
        setattr(s2, field, bad)
        with pytest.raises(SimError) as e:
            Simulator(s2)
        assert e.value.status == -1
    with pytest.raises(SimError) as e:
        Simulator(sc, global_solver="jacobi")
    assert e.value.status == -1
