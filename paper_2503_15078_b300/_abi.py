"""ctypes declarations mirroring include/silg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsilg.so")

SIM_OK = 0
STATUS = {0: "SIM_OK", -1: "SIM_EINVAL", -2: "SIM_ENOMEM", -3: "SIM_ENOTSPD", -4: "SIM_ECUDA",
          -5: "SIM_ECAPACITY", -6: "SIM_ETIMEOUT", -7: "SIM_ENONFINITE", -8: "SIM_ENOTSUP"}
SIM_MAX_RESIDUALS = 64
SIM_NUM_PHASES = 11
PHASES = ["collide", "delassus", "local", "assemble", "spmv1", "solve", "spmv2", "integrate",
          "reduce", "warmstart", "iterations"]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_fp = C.POINTER(C.c_float)
MLP_FEATURES, MLP_OUTPUTS, MLP_PARAMS = 11, 4, 36232


class SimMesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("rest_pos", _dp),
                ("tets", _ip), ("tet_material", _ip), ("pinned", _ip), ("n_pinned", C.c_int32),
                ("handle_vel", C.c_double * 3), ("tris", _ip), ("tri_material", _ip),
                ("n_tris", C.c_int32), ("thickness", C.c_double), ("bending", C.c_double)]


class SimMaterial(C.Structure):
    _fields_ = [("model", C.c_int32), ("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double)]


class SimObstacle(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_double * 3), ("axis", C.c_double * 3),
                ("radius", C.c_double), ("mu", C.c_double), ("vel", C.c_double * 3)]


class SimAnchor(C.Structure):
    _fields_ = [("vertex", C.c_int32), ("target", C.c_double * 3), ("vel", C.c_double * 3),
                ("compliance", C.c_double), ("paired", C.c_int32), ("partner", C.c_int32)]


class SimScene(C.Structure):
    _fields_ = [("mesh", SimMesh), ("materials", C.POINTER(SimMaterial)),
                ("n_materials", C.c_int32), ("obstacles", C.POINTER(SimObstacle)),
                ("n_obstacles", C.c_int32), ("contact_margin", C.c_double),
                ("anchors", C.POINTER(SimAnchor)), ("n_anchors", C.c_int32),
                ("body_contact", C.c_int32), ("body_mu", C.c_double)]


# device allocator hooks of sim_options
DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class SimOptions(C.Structure):
    _fields_ = [("n_iters", C.c_int32), ("n_cr_iters", C.c_int32), ("s_precision", C.c_int32),
                ("refine", C.c_int32), ("contact_capacity", C.c_int32), ("device", C.c_int32),
                ("gravity", C.c_double * 3), ("contact_margin", C.c_double),
                ("spin_limit", C.c_uint64), ("cuda_stream", C.c_void_p),
                ("n_host_threads", C.c_int32), ("autotune", C.c_int32),
                ("ncp", C.c_int32), ("precond", C.c_int32),
                ("residual_tol", C.c_double), ("max_iters", C.c_int32),
                ("local_solver", C.c_int32), ("global_solver", C.c_int32),
                ("jacobi_sweeps", C.c_int32), ("phase_marks", C.c_int32),
                ("dev_alloc", DEV_ALLOC), ("dev_free", DEV_FREE), ("alloc_ctx", C.c_void_p),
                ("cr_exchanges", C.c_int32), ("cr_sync", C.c_int32), ("s_build", C.c_int32),
                ("delassus_reuse", C.c_int32)]


class SimTuning(C.Structure):
    _fields_ = [("tuned", C.c_int32), ("candidates", C.c_int32), ("pass1_ctas", C.c_int32),
                ("pass2_ctas", C.c_int32), ("pass1_unroll", C.c_int32),
                ("pass2_unroll", C.c_int32), ("pass1_balance", C.c_double),
                ("pass2_balance", C.c_double), ("pass1_us", C.c_double), ("pass2_us", C.c_double),
                ("pass1_default_us", C.c_double), ("pass2_default_us", C.c_double)]


class SimStats(C.Structure):
    _fields_ = [("frame", C.c_int64), ("n_contacts", C.c_int32), ("n_contact_verts", C.c_int32),
                ("n_iters", C.c_int32), ("n_residuals", C.c_int32),
                ("residual", C.c_double * SIM_MAX_RESIDUALS), ("max_penetration", C.c_double),
                ("kernels_per_frame", C.c_int32), ("delassus_reused", C.c_int32),
                ("delassus_reuse_frames", C.c_int64)]


class SimPlanInfo(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_free", C.c_int32), ("n_tets", C.c_int32),
                ("nnz_A", C.c_int64), ("nnz_L", C.c_int64), ("nnz_S", C.c_int64),
                ("stored_S", C.c_int64), ("etree_max_depth", C.c_int32),
                ("etree_mean_depth", C.c_double), ("n_roots", C.c_int32),
                ("precompute_seconds", C.c_double), ("s_build_seconds", C.c_double),
                ("s_built_on_device", C.c_int32)]


# name -> (restype, argtypes); every entry must be exported by libsilg.so
PROTOTYPES = {
    "sim_create_batch": (C.c_int, [C.POINTER(SimScene), C.c_int32, C.c_double,
                                   C.POINTER(SimOptions), C.POINTER(C.c_void_p)]),
    "sim_get_scene_residuals": (C.c_int, [C.c_void_p, C.c_int32, _dp]),
    "sim_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sim_mlp_create": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "sim_set_warmstart": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "sim_set_portfolio": (C.c_int, [C.c_void_p, C.c_int32]),
    "sim_set_phase_marks": (C.c_int, [C.c_void_p, C.c_int32]),
    "sim_set_warmstart_gains": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_float,
                                           C.c_float]),
    "sim_get_warmstart_samples": (C.c_int, [C.c_void_p, C.c_int32, _fp, _fp,
                                            C.POINTER(C.c_int32)]),
    "sim_mlp_destroy": (None, [C.c_void_p]),
    "sim_mlp_init": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sim_mlp_set_tensor_cores": (C.c_int, [C.c_void_p, C.c_int32]),
    "sim_mlp_set_params": (C.c_int, [C.c_void_p, _fp]),
    "sim_mlp_get_params": (C.c_int, [C.c_void_p, _fp]),
    "sim_mlp_forward": (C.c_int, [C.c_void_p, _fp, C.c_int32, _fp]),
    "sim_mlp_gradient": (C.c_int, [C.c_void_p, _fp, _fp, C.c_int32, _fp, _fp]),
    "sim_mlp_train": (C.c_int, [C.c_void_p, _fp, _fp, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                C.c_uint64, _fp]),
    "sim_strerror": (C.c_char_p, [C.c_int]),
    "sim_default_options": (None, [C.POINTER(SimOptions)]),
    "sim_plan_create": (C.c_int, [C.POINTER(SimMesh), C.POINTER(SimMaterial), C.c_int32,
                                  C.c_double, C.POINTER(SimOptions), C.POINTER(C.c_void_p)]),
    "sim_plan_destroy": (None, [C.c_void_p]),
    "sim_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(SimPlanInfo)]),
    "sim_plan_get_ordering": (C.c_int, [C.c_void_p, _ip, _ip, _ip]),
    "sim_plan_apply_inverse_host": (C.c_int, [C.c_void_p, _dp, _dp]),
    "sim_create": (C.c_int, [C.POINTER(SimMesh), C.POINTER(SimMaterial), C.c_int32,
                             C.POINTER(SimObstacle), C.c_int32, C.c_double,
                             C.POINTER(SimOptions), C.POINTER(C.c_void_p)]),
    "sim_destroy": (None, [C.c_void_p]),
    "sim_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "sim_synchronize": (C.c_int, [C.c_void_p]),
    "sim_get_state": (C.c_int, [C.c_void_p, _dp, _dp, C.c_int32, _dp, _ip,
                                C.POINTER(SimStats)]),
    "sim_get_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t,
                                     C.POINTER(C.c_size_t)]),
    "sim_set_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sim_load_warmstart": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sim_set_state": (C.c_int, [C.c_void_p, _dp, _dp]),
    "sim_get_stats": (C.c_int, [C.c_void_p, C.POINTER(SimStats)]),
    "sim_get_contacts": (C.c_int, [C.c_void_p, C.c_int32, _ip, _ip, _dp, _dp, _ip]),
    "sim_get_phase_times": (C.c_int, [C.c_void_p, _dp]),
    "sim_get_plan_info": (C.c_int, [C.c_void_p, C.POINTER(SimPlanInfo)]),
    "sim_get_ordering": (C.c_int, [C.c_void_p, _ip, _ip, _ip]),
    "sim_apply_inverse": (C.c_int, [C.c_void_p, _dp, _dp]),
    "sim_local_project": (C.c_int, [C.c_void_p, _dp, _dp]),
    "sim_get_delassus": (C.c_int, [C.c_void_p, C.c_int32, _dp, _ip, _ip]),
    "sim_apply_inverse_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_measure_phase_boundaries": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _dp, _dp]),
}


def header_declarations(path=None):
    """Function names declared in include/silg.h (parsed from the header text)."""
    import re
    path = path or os.path.join(os.path.dirname(HERE), "include", "silg.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_2503_15078_b300.build` "
            "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib
