"""ctypes declarations of the C ABI in include/pbbem.h (no arithmetic here).

Loading builds the library first if it is missing or stale (nvcc is required);
there is no fallback: without libpbbem.so every call raises."""
import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_double, c_int64, c_void_p, c_char_p = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_char_p


class pb_params(ctypes.Structure):
    _fields_ = [("eps_int", c_double), ("eps_ext", c_double), ("kappa", c_double)]


class pb_quad_plan(ctypes.Structure):
    _fields_ = [("far_q", c_int), ("n_ss", c_int), ("band_eta", c_double), ("band_q", c_int),
                ("n_ss_coin", c_int), ("n_ss_edge", c_int), ("n_ss_vert", c_int)]


class pb_solve_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_it", c_int), ("restart", c_int), ("precision", c_int),
                ("inner_tol", c_double), ("max_outer", c_int), ("alpha", c_double), ("beta", c_double),
                ("pc_a", c_double), ("pc_b", c_double)]


class pb_solve_info(ctypes.Structure):
    _fields_ = [("status", c_int), ("iters", c_int), ("outer_iters", c_int), ("system_applies", c_int),
                ("rel_residual", c_double), ("time_ms", c_double)]


class pb_request(ctypes.Structure):
    _fields_ = [("verts", c_void_p), ("n_verts", c_int64), ("tris", c_void_p), ("n_tris", c_int64),
                ("xq", c_void_p), ("q", c_void_p), ("n_q", c_int64), ("params", pb_params), ("form", c_int),
                ("precond", c_int), ("opts", pb_solve_opts), ("plan", pb_quad_plan), ("tag", ctypes.c_uint64)]


class pb_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", c_int), ("iters", c_int), ("outer_iters", c_int),
                ("dG_kcal", c_double), ("dG_paper", c_double), ("rel_residual", c_double),
                ("latency_ms", c_double), ("queue_ms", c_double)]


class pb_tune_choice(ctypes.Structure):
    _fields_ = [("kernel", c_int), ("shape", c_int), ("tile_records", c_int), ("stages", c_int),
                ("targets_per_thread", c_int), ("tiles_per_fp64_sum", c_int), ("split_scale", c_double),
                ("best_ms", c_double),
                ("default_ms", c_double)]


class pb_tune_result(ctypes.Structure):
    _fields_ = [("fast", pb_tune_choice), ("accurate", pb_tune_choice)]


P = c_void_p
# name -> argtypes (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "pb_init": [c_int, ctypes.POINTER(c_void_p)],
    "pb_free_ctx": [P],
    "pb_last_error": [],
    "pb_version": [],
    "pb_mesh_load": [P, P, c_int64, P, c_int64, ctypes.POINTER(pb_quad_plan), c_int, ctypes.POINTER(c_void_p)],
    "pb_free_mesh": [P],
    "pb_mesh_info": [P, P],
    "pb_near_build": [P, P, c_double, ctypes.POINTER(c_void_p), P],
    "pb_free_near": [P],
    "pb_op_apply": [P, P, P, c_int, c_int, c_int, P, P, P],
    "pb_system_apply": [P, P, P, ctypes.POINTER(pb_params), c_int, c_double, c_double, c_int, P, P, P],
    "pb_rhs_charges": [P, P, P, P, c_int64, ctypes.POINTER(pb_params), c_int, c_double, c_double, P, c_int, P],
    "pb_solve": [P, P, P, ctypes.POINTER(pb_params), c_int, c_int, ctypes.POINTER(pb_solve_opts), P, P,
                 ctypes.POINTER(pb_solve_info), P],
    "pb_precond_apply": [P, P, P, ctypes.POINTER(pb_params), c_int, c_int, ctypes.POINTER(pb_solve_opts), c_int, P, P,
                         P],
    "pb_solve_many": [P, P, P, ctypes.POINTER(pb_params), c_int, c_int, ctypes.POINTER(pb_solve_opts), c_int, P, P,
                      P, P],
    "pb_solve_pc": [P, P, P, P, P, ctypes.POINTER(pb_params), c_int, c_int, ctypes.POINTER(pb_solve_opts), P, P,
                    ctypes.POINTER(pb_solve_info), P],
    "pb_energy": [P, P, P, c_int, P, P, c_int64, ctypes.POINTER(pb_params), P, ctypes.POINTER(c_double),
                  ctypes.POINTER(c_double), c_int, P],
    "pb_solvation_energy": [P, P, c_int64, P, c_int64, P, P, c_int64, ctypes.POINTER(pb_params),
                            ctypes.POINTER(pb_quad_plan), c_int, c_int, ctypes.POINTER(pb_solve_opts),
                            ctypes.POINTER(c_double), ctypes.POINTER(pb_solve_info), P],
    "pb_system_apply_noalloc": [P, P, P, ctypes.POINTER(pb_params), c_int, c_double, c_double, P, P, P],
    "pb_server_create": [P, c_int64, c_int, ctypes.POINTER(c_void_p)],
    "pb_server_destroy": [P],
    "pb_submit": [P, ctypes.POINTER(pb_request)],
    "pb_server_step": [P, ctypes.POINTER(c_int), ctypes.POINTER(c_int)],
    "pb_poll": [P, ctypes.POINTER(pb_result), c_int, ctypes.POINTER(c_int)],
    "pb_autotune": [P, P, P, ctypes.POINTER(pb_params), c_int, ctypes.POINTER(pb_tune_result), P],
    "pb_autotune_plan": [P, P, c_int64, P, c_int64, P, P, c_int64, ctypes.POINTER(pb_params),
                         ctypes.POINTER(pb_quad_plan), c_int, c_int, ctypes.POINTER(pb_solve_opts), c_double,
                         ctypes.POINTER(pb_quad_plan), ctypes.POINTER(c_double), P],
    "pb_profile": [P, c_int],
    "pb_profile_read": [P, c_int, ctypes.POINTER(c_int64), ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                        ctypes.POINTER(c_double)],
    "pb_launch_count": [],
    "pb_selftest_wait": [P, c_int64, ctypes.POINTER(c_int)],
    "pb_selftest_exp": [P, P, P, c_int64, P],
    "pb_measure_peak": [P, c_int, ctypes.POINTER(c_double)],
    "pb_set_graphs": [P, c_int],
    "pb_set_treecode": [P, c_int, c_int, c_double, c_int64],
    "pb_tree_info": [P, ctypes.POINTER(c_int64)],
}
_RESTYPE = {"pb_last_error": c_char_p, "pb_version": c_char_p, "pb_launch_count": c_int64}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpbbem.so (building it first if needed) and declare every symbol."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libpbbem.so not found at {path}")
            L = ctypes.CDLL(path)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = _RESTYPE.get(name, c_int)
            _lib = L
    return _lib
