"""ctypes binding of libpdgb300.so (argument marshalling only).

Every function of include/pd.h is exposed under the same name.  The
library must be built (``paper_2405_12484_gb300.build.build()``); importing
this module without it raises ImportError -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdgb300.so")

PD_OK = 0
PD_ERR_INVALID_ARG = -1
PD_ERR_BAD_MESH = -2
PD_ERR_BAD_MATERIAL = -3
PD_ERR_NOT_PREFACTORED = -4
PD_ERR_NOT_SPD = -5
PD_ERR_NO_MEMORY = -6
PD_ERR_NONFINITE = -7
PD_ERR_TIMEOUT = -8
PD_ERR_CUDA = -9
PD_ERR_UNSUPPORTED = -10

PD_PREC_FP32 = 0
PD_PREC_BF16 = 1
PD_PREC_TF32 = 2

PD_SOLVE_CORRECTION = 1
PD_SOLVE_SINGLE_LEVEL = 2
PD_SOLVE_STREAMING = 4
PD_SOLVE_MODAL = 8


class pd_solver_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("refine_steps", C.c_int32), ("use_graphs", C.c_int32),
                ("flags", C.c_int32), ("modes", C.c_int32), ("jacobi_sweeps", C.c_int32), ("jacobi_rho", C.c_double)]


class pd_mesh_info(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_tets", C.c_int32), ("n_domains", C.c_int32),
                ("n_pinned", C.c_int32), ("n_interface", C.c_int32), ("n_internal", C.c_int32),
                ("max_domain_internal", C.c_int32), ("max_domain_boundary", C.c_int32),
                ("device_bytes", C.c_int64), ("prefactor_seconds", C.c_double),
                ("launches_per_iter", C.c_int32), ("launches_per_frame", C.c_int32),
                ("phase_bytes", C.c_int64 * 24), ("n_groups", C.c_int32), ("n_top_interface", C.c_int32),
                ("two_level", C.c_int32), ("phase_launches", C.c_int32 * 24)]


class pd_fit_opts(C.Structure):
    _fields_ = [("n_gd", C.c_int32), ("n_gn", C.c_int32), ("gd_step", C.c_float), ("gn_step", C.c_float),
                ("kappa_rel", C.c_double), ("floor", C.c_float), ("max_halvings", C.c_int32),
                ("max_pivots", C.c_int32), ("n_pd_iter", C.c_int32), ("n_newton", C.c_int32),
                ("outer_iters", C.c_int32), ("dt", C.c_double), ("solver", C.POINTER(pd_solver_opts))]


class pd_fit_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("trials", C.c_int32), ("clamped", C.c_int32), ("pivots", C.c_int32),
                ("loss0", C.c_double), ("loss", C.c_double), ("seconds", C.c_double)]


PD_REQ_QUEUED, PD_REQ_ACTIVE, PD_REQ_DONE, PD_REQ_FAILED = 0, 1, 2, 3


class pd_request(C.Structure):
    _fields_ = [("rest_xyz", C.c_void_p), ("n_v", C.c_int32), ("tets", C.c_void_p), ("n_t", C.c_int32),
                ("tet_domain", C.c_void_p), ("n_domains", C.c_int32), ("pinned", C.c_void_p),
                ("gamma_s", C.c_void_p), ("gamma_v", C.c_void_p), ("density", C.c_double), ("dt", C.c_double),
                ("n_frames", C.c_int32), ("gravity", C.c_float * 3), ("drive_amp", C.c_float),
                ("drive_freq", C.c_float), ("drive_axis", C.c_int32)]


# (name, restype, argtypes) exactly as declared in include/pd.h
SIGNATURES = [
    ("pd_create_mesh", C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_double,
                                   C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("pd_destroy_mesh", None, [C.c_void_p]),
    ("pd_set_materials", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_prefactor", C.c_int32, [C.c_void_p, C.c_double, C.POINTER(pd_solver_opts)]),
    ("pd_set_state", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_get_state", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_step", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    ("pd_sync", C.c_int32, [C.c_void_p]),
    ("pd_get_info", C.c_int32, [C.c_void_p, C.POINTER(pd_mesh_info)]),
    ("pd_status_string", C.c_char_p, [C.c_int32]),
    ("pd_last_error", C.c_char_p, []),
    ("pd_project", C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_local_rhs", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_solve", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_enable_timing", C.c_int32, [C.c_void_p, C.c_int32]),
    ("pd_set_timing_iteration", C.c_int32, [C.c_void_p, C.c_int32]),
    ("pd_phase_times", C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    ("pd_phase_name", C.c_char_p, [C.c_int32]),
    ("pd_test_offset_phase_counter", C.c_int32, [C.c_void_p, C.c_int32, C.c_int32]),
    ("pd_test_inflate_copy", C.c_int32, [C.c_void_p, C.c_int32]),
    ("pd_solve_noalloc", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_adjoint_create", C.c_int32, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    ("pd_adjoint_destroy", None, [C.c_void_p]),
    ("pd_adjoint_reset", C.c_int32, [C.c_void_p]),
    ("pd_equilibrium_step", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                        C.c_void_p]),
    ("pd_adjoint_step", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_adjoint_step64", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_adjoint_get_state64", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_adjoint_set_state64", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_hessian_vec", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_residual", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_pose_misfit", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_pose_misfit_accumulate", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pd_tied_gradient", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    ("pd_gn_product", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                  C.c_void_p]),
    ("pd_gn_direction", C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                    C.c_float, C.c_int32, C.c_void_p, C.c_void_p]),
    ("pd_fit_pose", C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(pd_fit_opts), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(pd_fit_report)]),
    ("pd_harmonic_basis", C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    ("pd_fit_pose_reduced", C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(pd_fit_opts), C.c_void_p, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.POINTER(pd_fit_report)]),
    ("pd_server_create", C.c_int32, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("pd_server_destroy", None, [C.c_void_p]),
    ("pd_submit", C.c_int32, [C.c_void_p, C.POINTER(pd_request), C.POINTER(C.c_int64)]),
    ("pd_server_tick", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    ("pd_server_run", C.c_int32, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    ("pd_poll", C.c_int32, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("pd_fetch", C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    ("pd_release", C.c_int32, [C.c_void_p, C.c_int64]),
    ("pd_server_stats", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libpdgb300.so not built at {path}: run paper_2405_12484_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class PDError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status
