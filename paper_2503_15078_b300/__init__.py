"""B300-native sparse-inverse local-global simulator with robust frictional contact.

Python binding over the C ABI of ``libsilg.so`` (include/silg.h). The binding only
marshals arguments: every step of the solve runs in the library's CUDA kernels (sm_103a)
or, for the one-time precompute, its C++ host code. PyTorch supplies the CUDA stream when
it is available; nothing here computes the method.

    from paper_2503_15078_b300 import Simulator
    sim = Simulator(scene)          # any object with the scene fields (see ``_mesh_args``)
    sim.step()                      # one frame (Alg. 4)
    q, v = sim.state()
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi

_lib = None


def lib():
    """The loaded shared library (raises ImportError if it was not built)."""
    global _lib
    if _lib is None:
        _lib = _abi.load()
    return _lib


class SimError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().sim_strerror(status).decode()
        super().__init__(f"{where}: {_abi.STATUS.get(status, status)} ({msg})")


def _check(status, where):
    if status != _abi.SIM_OK:
        raise SimError(status, where)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _mesh_args(scene):
    """Marshal a scene (X, tets, tet_material, materials, pinned, handle_vel, obstacles)
    into the ABI structs; the returned tuple keeps the numpy buffers alive."""
    X = np.ascontiguousarray(scene.X, dtype=np.float64)
    tets = np.ascontiguousarray(scene.tets, dtype=np.int32)
    tm = np.ascontiguousarray(scene.tet_material, dtype=np.int32)
    pin = np.ascontiguousarray(scene.pinned, dtype=np.int32)
    mesh = _abi.SimMesh()
    mesh.n_verts = X.shape[0]
    mesh.n_tets = tets.shape[0]
    mesh.rest_pos = _dptr(X)
    mesh.tets = _iptr(tets)
    mesh.tet_material = _iptr(tm)
    mesh.pinned = _iptr(pin) if len(pin) else None
    mesh.n_pinned = len(pin)
    for r in range(3):
        mesh.handle_vel[r] = float(scene.handle_vel[r])
    tris = np.ascontiguousarray(getattr(scene, "tris", None) if getattr(scene, "tris", None)
                                is not None else np.zeros((0, 3)), dtype=np.int32).reshape(-1, 3)
    trm = np.ascontiguousarray(getattr(scene, "tri_material", None)
                               if getattr(scene, "tri_material", None) is not None
                               else np.zeros(len(tris)), dtype=np.int32)
    mesh.tris = _iptr(tris) if len(tris) else None
    mesh.tri_material = _iptr(trm) if len(tris) else None
    mesh.n_tris = len(tris)
    mesh.thickness = float(getattr(scene, "thickness", 0.0))
    mesh.bending = float(getattr(scene, "bending", 0.0))
    mats = (_abi.SimMaterial * len(scene.materials))()
    for i, m in enumerate(scene.materials):
        mats[i].model, mats[i].E, mats[i].nu, mats[i].rho = int(m.model), m.E, m.nu, m.rho
    obs = (_abi.SimObstacle * max(1, len(scene.obstacles)))()
    for i, o in enumerate(scene.obstacles):
        obs[i].kind = int(o.kind)
        for r in range(3):
            obs[i].p[r] = float(o.p[r])
            obs[i].axis[r] = float(o.axis[r])
            obs[i].vel[r] = float(o.vel[r])
        obs[i].radius = float(o.radius)
        obs[i].mu = float(o.mu)
    return mesh, mats, obs, (X, tets, tm, pin, tris, trm)


def default_options():
    o = _abi.SimOptions()
    lib().sim_default_options(C.byref(o))
    return o


def _options(scene=None, **kw):
    o = default_options()
    if scene is not None:
        o.n_iters = int(getattr(scene, "n_iters", o.n_iters))
        o.n_cr_iters = int(getattr(scene, "n_cr", o.n_cr_iters))
        g = getattr(scene, "gravity", None)
        if g is not None:
            for r in range(3):
                o.gravity[r] = float(g[r])
        o.contact_margin = float(getattr(scene, "contact_margin", 0.0))
    for k, v in kw.items():
        if k == "gravity":
            for r in range(3):
                o.gravity[r] = float(v[r])
        elif k in ("dev_alloc", "dev_free") and v is not None and callable(v) \
                and not isinstance(v, (_abi.DEV_ALLOC, _abi.DEV_FREE)):
            # a Python callable: wrapped (the options struct keeps the wrapper alive)
            setattr(o, k, (_abi.DEV_ALLOC if k == "dev_alloc" else _abi.DEV_FREE)(v))
        elif k in _NAMED and isinstance(v, str):
            if v not in _NAMED[k]:
                raise ValueError(f"{k} must be one of {sorted(_NAMED[k])}")
            setattr(o, k, _NAMED[k][v])
        else:
            setattr(o, k, v)
    return o


# options that also take names: the complementarity functions (App. B.1-B.2), the
# complementarity preconditioner (Sec. 5.4) and the local step (PD or ADMM-PD)
_NAMED = {"ncp": {"fb": 0, "minmap": 1}, "precond": {"delassus": 0, "mass": 1},
          "local_solver": {"pd": 0, "admm": 1},
          "global_solver": {"sparse_inverse": 0, "jacobi": 1}}


class Plan:
    """Host-only precompute (ordering, elimination tree, Cholesky, S~ = L~^-1 P)."""

    def __init__(self, scene, h=None, **opts):
        mesh, mats, _obs, self._keep = _mesh_args(scene)
        o = _options(scene, **opts)
        h = float(scene.h if h is None else h)
        handle = C.c_void_p()
        _check(lib().sim_plan_create(C.byref(mesh), mats, len(scene.materials), h, C.byref(o),
                                     C.byref(handle)), "sim_plan_create")
        self._h = handle
        self.n_verts = mesh.n_verts

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().sim_plan_destroy(h)
            self._h = None

    def info(self):
        i = _abi.SimPlanInfo()
        _check(lib().sim_plan_get_info(self._h, C.byref(i)), "sim_plan_get_info")
        return {f: getattr(i, f) for f, _ in i._fields_}

    def ordering(self):
        nf = self.info()["n_free"]
        order = np.zeros(nf, np.int32)
        parent = np.zeros(nf, np.int32)
        fd = np.zeros(nf, np.int32)
        _check(lib().sim_plan_get_ordering(self._h, _iptr(order), _iptr(parent), _iptr(fd)),
               "sim_plan_get_ordering")
        return order, parent, fd

    def apply_inverse_host(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(self.n_verts, 3)
        x = np.zeros_like(b)
        _check(lib().sim_plan_apply_inverse_host(self._h, _dptr(b), _dptr(x)),
               "sim_plan_apply_inverse_host")
        return x


def measure_phase_boundaries(n_phases=64, ctas_per_sm=1, device=0):
    """Device microseconds per phase boundary: (kernel per phase in a CUDA graph with
    programmatic dependent launch, software grid barrier in one cooperative kernel)."""
    a = np.zeros(1)
    b = np.zeros(1)
    _check(lib().sim_measure_phase_boundaries(int(device), int(n_phases), int(ctas_per_sm),
                                              _dptr(a), _dptr(b)),
           "sim_measure_phase_boundaries")
    return float(a[0]), float(b[0])


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class WarmStartNet:
    """The warm-start network on one GPU (thin wrapper over the sim_mlp_* C ABI)."""

    FEATURES, OUTPUTS, PARAMS = _abi.MLP_FEATURES, _abi.MLP_OUTPUTS, _abi.MLP_PARAMS

    def __init__(self, device=0, max_batch=65536, seed=None):
        h = C.c_void_p()
        _check(lib().sim_mlp_create(int(device), int(max_batch), C.byref(h)), "sim_mlp_create")
        self._h = h
        if seed is not None:
            _check(lib().sim_mlp_init(self._h, int(seed)), "sim_mlp_init")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sim_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_tensor_cores(self, kind):
        """"mma_sync" (warp-level, the default) or "tcgen05" (5th-generation tensor cores with
        tensor-memory accumulators) for the inference."""
        k = {"mma_sync": 0, "tcgen05": 1}[kind]
        _check(lib().sim_mlp_set_tensor_cores(self._h, k), "sim_mlp_set_tensor_cores")

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.PARAMS
        _check(lib().sim_mlp_set_params(self._h, _fptr(t)), "sim_mlp_set_params")

    def params(self):
        t = np.zeros(self.PARAMS, np.float32)
        _check(lib().sim_mlp_get_params(self._h, _fptr(t)), "sim_mlp_get_params")
        return t

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, self.FEATURES)
        Y = np.zeros((X.shape[0], self.OUTPUTS), np.float32)
        _check(lib().sim_mlp_forward(self._h, _fptr(X), X.shape[0], _fptr(Y)), "sim_mlp_forward")
        return Y

    def gradient(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, self.FEATURES)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, self.OUTPUTS)
        g = np.zeros(self.PARAMS, np.float32)
        loss = np.zeros(1, np.float32)
        _check(lib().sim_mlp_gradient(self._h, _fptr(X), _fptr(T), X.shape[0], _fptr(g),
                                      _fptr(loss)), "sim_mlp_gradient")
        return g, float(loss[0])

    def train(self, X, T, epochs, batch=512, lr=1e-3, seed=0):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, self.FEATURES)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, self.OUTPUTS)
        el = np.zeros(max(1, epochs), np.float32)
        _check(lib().sim_mlp_train(self._h, _fptr(X), _fptr(T), X.shape[0], int(epochs),
                                   int(batch), float(lr), int(seed), _fptr(el)), "sim_mlp_train")
        return el[:epochs]


class Simulator:
    """One scene, or a batch of independent scenes (a list), on one GPU. Every method is a
    thin call into the C ABI. A batch numbers vertices scene after scene; scene_offsets
    gives each scene's first vertex."""

    def __init__(self, scene, use_torch_stream=True, **opts):
        batch = isinstance(scene, (list, tuple))
        if not batch and (getattr(scene, "anchors", None) or getattr(scene, "body_contact", False)):
            # anchors and body contact travel in sim_scene (sim_create_batch)
            scene, batch = [scene], True
        first = scene[0] if batch else scene
        o = _options(first, **opts)
        if use_torch_stream and "cuda_stream" not in opts:
            s = _torch_stream()
            if s is not None:
                o.cuda_stream = s
        handle = C.c_void_p()
        if batch:
            scs = (_abi.SimScene * len(scene))()
            self._keep = []
            for k, sc in enumerate(scene):
                mesh, mats, obs, keep = _mesh_args(sc)
                self._keep.append((mats, obs, keep))
                scs[k].mesh = mesh
                scs[k].materials = C.cast(mats, C.POINTER(_abi.SimMaterial))
                scs[k].n_materials = len(sc.materials)
                scs[k].obstacles = C.cast(obs, C.POINTER(_abi.SimObstacle))
                scs[k].n_obstacles = len(sc.obstacles)
                scs[k].contact_margin = float(getattr(sc, "contact_margin", 0.0))
                anchors = getattr(sc, "anchors", None) or []
                if anchors:
                    an = (_abi.SimAnchor * len(anchors))()
                    for i, a in enumerate(anchors):
                        an[i].vertex = int(a.vertex)
                        for r in range(3):
                            an[i].target[r] = float(a.target[r])
                            an[i].vel[r] = float(a.vel[r])
                        an[i].compliance = float(a.compliance)
                        partner = int(getattr(a, "partner", -1))
                        an[i].paired = 1 if partner >= 0 else 0
                        an[i].partner = max(partner, 0)
                    self._keep.append(an)
                    scs[k].anchors = C.cast(an, C.POINTER(_abi.SimAnchor))
                    scs[k].n_anchors = len(anchors)
                scs[k].body_contact = 1 if getattr(sc, "body_contact", False) else 0
                scs[k].body_mu = float(getattr(sc, "body_mu", 0.0))
            self._keep.append(scs)
            _check(lib().sim_create_batch(scs, len(scene), float(first.h), C.byref(o),
                                          C.byref(handle)), "sim_create_batch")
            sizes = [sc.n_verts for sc in scene]
            self.scene_offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
            self.n_verts = int(self.scene_offsets[-1])
            self.n_tets = int(sum(len(sc.tets) for sc in scene))
            self.n_scenes = len(scene)
            q0 = np.concatenate([sc.q0 for sc in scene])
            v0 = np.concatenate([sc.v0 for sc in scene])
        else:
            mesh, mats, obs, self._keep = _mesh_args(scene)
            _check(lib().sim_create(C.byref(mesh), mats, len(scene.materials), obs,
                                    len(scene.obstacles), float(scene.h), C.byref(o),
                                    C.byref(handle)), "sim_create")
            self.n_verts = mesh.n_verts
            self.n_tets = mesh.n_tets
            self.n_scenes = 1
            self.scene_offsets = np.array([0, mesh.n_verts], dtype=np.int64)
            q0 = getattr(scene, "q0", None)
            v0 = getattr(scene, "v0", None)
        self._h = handle
        self.options = o
        if q0 is not None:
            self.set_state(q0, v0 if v0 is not None else np.zeros_like(q0))

    def set_warmstart(self, mode, net=None):
        """0 cold (the paper's start), 1 the network's guess, 2 the previous frame's impulses."""
        _check(lib().sim_set_warmstart(self._h, net.handle if net is not None else None,
                                       int(mode)), "sim_set_warmstart")

    def set_warmstart_gains(self, persist=1.0, fresh=1.0, move=1.0, accept=1.0):
        """Gains of the network's outputs in the learned start (persisting contacts' impulse
        change, new contacts' impulse, change of the normal move) and its acceptance ratio
        (the guess is kept when its residual at k = 0 is below accept x the cold start's)."""
        _check(lib().sim_set_warmstart_gains(self._h, float(persist), float(fresh), float(move),
                                             float(accept)),
               "sim_set_warmstart_gains")

    def set_phase_marks(self, on):
        """Event nodes around every phase of every iteration (True) or only around the
        once-per-frame phases, the iterations timed as one phase (False)."""
        _check(lib().sim_set_phase_marks(self._h, int(bool(on))), "sim_set_phase_marks")

    def set_portfolio(self, copies):
        """Scenes are groups of `copies` identical copies: copy 0 runs cold, the others the
        warm start, and each frame every copy continues from the best one (1: off)."""
        _check(lib().sim_set_portfolio(self._h, int(copies)), "sim_set_portfolio")

    def warmstart_samples(self):
        """(features, targets) of the last frame's contacts."""
        n = C.c_int32()
        _check(lib().sim_get_warmstart_samples(self._h, 0, None, None, C.byref(n)),
               "sim_get_warmstart_samples")
        c = n.value
        X = np.zeros((max(c, 1), WarmStartNet.FEATURES), np.float32)
        T = np.zeros((max(c, 1), WarmStartNet.OUTPUTS), np.float32)
        _check(lib().sim_get_warmstart_samples(self._h, c, _fptr(X), _fptr(T), C.byref(n)),
               "sim_get_warmstart_samples")
        return X[:c], T[:c]

    def tuning(self):
        """Launch configuration of the profile products (autotuned or fixed)."""
        t = _abi.SimTuning()
        _check(lib().sim_get_tuning(self._h, C.byref(t)), "sim_get_tuning")
        return {f: getattr(t, f) for f, _ in t._fields_}

    def scene_residuals(self):
        """(n_scenes, n_iters + 1) residuals of the last frame, per scene."""
        K = self.stats()["n_iters"]
        out = np.zeros((self.n_scenes, K + 1))
        _check(lib().sim_get_scene_residuals(self._h, out.size, _dptr(out)),
               "sim_get_scene_residuals")
        return out

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().sim_destroy(h)
        self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def step(self, n_iters=0, n_frames=1):
        for _ in range(n_frames):
            _check(lib().sim_step(self._h, int(n_iters)), "sim_step")

    def synchronize(self):
        _check(lib().sim_synchronize(self._h), "sim_synchronize")

    def state(self):
        q = np.zeros((self.n_verts, 3))
        v = np.zeros((self.n_verts, 3))
        _check(lib().sim_get_state(self._h, _dptr(q), _dptr(v), 0, None, None, None),
               "sim_get_state")
        return q, v

    def full_state(self):
        """(q, v, lambda, stats) of the last frame in one call: lambda per contact (n, f1, f2)
        in the order of contacts()."""
        q = np.zeros((self.n_verts, 3))
        v = np.zeros((self.n_verts, 3))
        cap = int(self.options.contact_capacity)
        lam = np.zeros((max(cap, 1), 3))
        n = C.c_int32()
        s = _abi.SimStats()
        _check(lib().sim_get_state(self._h, _dptr(q), _dptr(v), max(cap, 1), _dptr(lam),
                                   C.byref(n), C.byref(s)), "sim_get_state")
        st = {f: getattr(s, f) for f, _ in s._fields_ if f != "residual"}
        st["residuals"] = [s.residual[k] for k in range(min(s.n_residuals, _abi.SIM_MAX_RESIDUALS))]
        return q, v, lam[:min(n.value, cap)], st

    def checkpoint(self):
        """Everything a later frame depends on, as bytes (sim_get_checkpoint)."""
        size = C.c_size_t()
        _check(lib().sim_get_checkpoint(self._h, None, 0, C.byref(size)), "sim_get_checkpoint")
        buf = C.create_string_buffer(size.value)
        _check(lib().sim_get_checkpoint(self._h, buf, size.value, C.byref(size)),
               "sim_get_checkpoint")
        return buf.raw

    def restore(self, blob):
        """Continue exactly from a checkpoint() of this simulator (sim_set_checkpoint)."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _check(lib().sim_set_checkpoint(self._h, buf, len(blob)), "sim_set_checkpoint")

    def load_warmstart(self, theta):
        """Load a trained network's FP32 parameter vector and use the learned start."""
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().sim_load_warmstart(self._h, t.ctypes.data_as(C.c_void_p), t.nbytes),
               "sim_load_warmstart")

    def set_state(self, q, v):
        q = np.ascontiguousarray(q, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        _check(lib().sim_set_state(self._h, _dptr(q), _dptr(v)), "sim_set_state")

    def stats(self):
        s = _abi.SimStats()
        _check(lib().sim_get_stats(self._h, C.byref(s)), "sim_get_stats")
        d = {f: getattr(s, f) for f, _ in s._fields_ if f != "residual"}
        d["residuals"] = [s.residual[k] for k in range(min(s.n_residuals, _abi.SIM_MAX_RESIDUALS))]
        return d

    def plan_info(self):
        i = _abi.SimPlanInfo()
        _check(lib().sim_get_plan_info(self._h, C.byref(i)), "sim_get_plan_info")
        return {f: getattr(i, f) for f, _ in i._fields_}

    def ordering(self):
        """(order, parent, first_desc) of the simulator's internal rows: row k is caller
        vertex order[k] (batch numbering for a batch)."""
        nf = self.plan_info()["n_free"]
        order = np.zeros(nf, np.int32)
        parent = np.zeros(nf, np.int32)
        fd = np.zeros(nf, np.int32)
        _check(lib().sim_get_ordering(self._h, _iptr(order), _iptr(parent), _iptr(fd)),
               "sim_get_ordering")
        return order, parent, fd

    def phase_times(self):
        """Device milliseconds per phase of the most recent frame (event nodes in its graph)."""
        ms = np.zeros(_abi.SIM_NUM_PHASES)
        _check(lib().sim_get_phase_times(self._h, _dptr(ms)), "sim_get_phase_times")
        return dict(zip(_abi.PHASES, ms.tolist()))

    def contacts(self):
        n = C.c_int32()
        _check(lib().sim_get_contacts(self._h, 0, None, None, None, None, C.byref(n)),
               "sim_get_contacts")
        c = n.value
        vert = np.zeros(max(c, 1), np.int32)
        obst = np.zeros(max(c, 1), np.int32)
        lam = np.zeros((max(c, 1), 3))
        frame = np.zeros((max(c, 1), 3, 3))
        _check(lib().sim_get_contacts(self._h, c, _iptr(vert), _iptr(obst), _dptr(lam),
                                      _dptr(frame), C.byref(n)), "sim_get_contacts")
        return dict(vertex=vert[:c], obstacle=obst[:c], lam=lam[:c], frame=frame[:c])

    def apply_inverse(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(self.n_verts, 3)
        x = np.zeros_like(b)
        _check(lib().sim_apply_inverse(self._h, _dptr(b), _dptr(x)), "sim_apply_inverse")
        return x

    def apply_inverse_noalloc(self, g_ptr, x_ptr, stream_ptr=None):
        """x = A^-1 g on device buffers without allocating (see sim_apply_inverse_noalloc):
        g_ptr and x_ptr are device addresses of n_free x 3 FP32 arrays in the solver's row
        order; the call is asynchronous on the given stream."""
        _check(lib().sim_apply_inverse_noalloc(self._h, C.c_void_p(g_ptr), C.c_void_p(x_ptr),
                                               C.c_void_p(stream_ptr or 0)),
               "sim_apply_inverse_noalloc")

    def local_project(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(self.n_verts, 3)
        p = np.zeros((self.n_tets, 3, 3))
        _check(lib().sim_local_project(self._h, _dptr(q), _dptr(p)), "sim_local_project")
        return p

    def delassus(self):
        n = C.c_int32()
        _check(lib().sim_get_delassus(self._h, 0, None, None, C.byref(n)), "sim_get_delassus")
        m = n.value
        W = np.zeros((max(m, 1), max(m, 1)))
        cv = np.zeros(max(m, 1), np.int32)
        _check(lib().sim_get_delassus(self._h, m, _dptr(W), _iptr(cv), C.byref(n)),
               "sim_get_delassus")
        return W[:m, :m], cv[:m]
