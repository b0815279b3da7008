"""ctypes declarations of the C ABI in include/wcs.h (argument marshalling only)."""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwcs.so")

WCS_OK, WCS_ERR_ARG, WCS_ERR_NOT_CONVERGED, WCS_ERR_RANK_CAP = 0, 1, 7, 6
STATUS_NAMES = {0: "WCS_OK", 1: "WCS_ERR_ARG", 2: "WCS_ERR_NOT_CONVEX", 3: "WCS_ERR_CUDA",
                4: "WCS_ERR_OOM", 5: "WCS_ERR_SINGULAR", 6: "WCS_ERR_RANK_CAP",
                7: "WCS_ERR_NOT_CONVERGED", 8: "WCS_ERR_TIMEOUT", 9: "WCS_ERR_STATE",
                10: "WCS_ERR_UNSUPPORTED"}

OPS = {"C": 0, "CH": 1, "CC": 2, "CCH": 3, "CC_INV": 4, "S": 5, "D": 6, "DT": 7, "N": 8, "G": 9,
       "SKEL": 10, "GINV": 11, "CCH_INV": 12}


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("q_far", C.c_int), ("q_near", C.c_int),
                ("near_band", C.c_int), ("block", C.c_int), ("max_refine", C.c_int),
                ("refine_tol", C.c_double), ("rhs_chunk", C.c_int), ("mixed_planes", C.c_int),
                ("rhs_planes", C.c_int), ("zfast", C.c_double), ("sample_planes", C.c_int),
                ("exact_residual", C.c_int)]


class Info(C.Structure):
    _fields_ = [("N", C.c_int64), ("L", C.c_double), ("h", C.c_double), ("a", C.c_double),
                ("k", C.c_double), ("kt_re", C.c_double), ("kt_im", C.c_double),
                ("rank", C.c_int), ("norm_cc", C.c_double), ("min_curvature", C.c_double),
                ("zfast", C.c_double), ("capacitance_residual", C.c_double)]


WCS_HISTORY = 32


class SolveInfo(C.Structure):
    _fields_ = [("refine_steps", C.c_int), ("rel_residual", C.c_double), ("history_len", C.c_int),
                ("history", C.c_double * WCS_HISTORY)]


class BatchStats(C.Structure):
    _fields_ = [("status", C.c_int), ("rank", C.c_int), ("refine_steps", C.c_int), ("rel_residual", C.c_double),
                ("setup_s", C.c_double), ("solve_s", C.c_double), ("worker", C.c_int)]


# exported symbol -> (restype, argtypes); mirrors include/wcs.h
P, I, I64, D, U64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
SIGNATURES = {
    "wcs_version": (C.c_char_p, []),
    "wcs_last_error": (C.c_char_p, []),
    "wcs_default_options": (I, [C.POINTER(Options)]),
    "wcs_create": (I, [C.POINTER(P), C.POINTER(Options), P]),
    "wcs_destroy": (I, [P]),
    "wcs_contour_circle": (I, [P, D]),
    "wcs_contour_ellipse": (I, [P, D, D]),
    "wcs_contour_superellipse": (I, [P, D, D, D]),
    "wcs_contour_fourier": (I, [P, I, P, P]),
    "wcs_mesh": (I, [P, I64, D]),
    "wcs_query": (I, [P, C.POINTER(Info)]),
    "wcs_geometry_sample": (I, [P, I64, P, P]),
    "wcs_assemble": (I, [P]),
    "wcs_operator_entries": (I, [P, I64, P, P, P]),
    "wcs_circulant_eigs": (I, [P, I, P]),
    "wcs_apply": (I, [P, I, I64, P, I64, P, I64]),
    "wcs_skeleton": (I, [P, D, I, U64, C.POINTER(I)]),
    "wcs_factor": (I, [P]),
    "wcs_save": (I, [P, C.c_char_p]),
    "wcs_load": (I, [P, C.c_char_p]),
    "wcs_woodbury_apply": (I, [P, I64, P, I64, P, I64]),
    "wcs_solve_planewaves": (I, [P, I64, P, P, I64, C.POINTER(SolveInfo)]),
    "wcs_solve_planewaves_host": (I, [P, I64, P, P, I64, C.POINTER(SolveInfo)]),
    "wcs_solve_rhs": (I, [P, I64, P, P, I64, P, I64, C.POINTER(SolveInfo)]),
    "wcs_solve": (I, [P, I64, P, I64, P, I64, C.POINTER(SolveInfo)]),
    "wcs_contour_perturb": (I, [P, C.c_int, P, P]),
    "wcs_shape_gradient": (I, [P, I64, P, C.c_int, P, C.c_int, C.c_double, P, P]),
    "wcs_shape_gradient_range": (I, [P, I64, P, C.c_int, P, C.c_int, C.c_double, C.c_int, C.c_int, P, P]),
    "wcs_solve_adjoint": (I, [P, I64, P, I64, P, I64, C.POINTER(SolveInfo)]),
    "wcs_planewave_rhs": (I, [P, I64, P, P, P, I64]),
    "wcs_farfield": (I, [P, I64, P, I64, I, P, P, I64]),
    "wcs_gemm_split_bf16": (I, [I64, I64, I64, P, I64, P, I64, I, P, I64, P]),
    "wcs_gemm_split_bf16_ex": (I, [I64, I64, I64, P, I64, P, I64, I, I, P, I64, P]),
    "wcs_gemm_split_bf16_noalloc": (I, [I64, I64, I64, P, I64, P, I64, I, P, I64, P]),
    "wcs_launch_count": (U64, []),
    "wcs_profile": (I, [P, I]),
    "wcs_profile_read": (I, [P, I, P]),
    "wcs_quadrature_tables": (I, [I, P]),
    "wcs_fma_rate": (I, [I, I, P, C.POINTER(C.c_double)]),
    "wcs_gemm_exact": (I, [I64, I64, I64, P, I64, P, I64, P, I64, P]),
    "wcs_shape_operator_forms": (I, [P, I, I64, P, P, I64, I, C.c_double, I, I, P]),
    "wcs_batch_solve_fourier": (I, [C.POINTER(Options), I, I, P, P, P, P, I64, P, C.c_double, I, U64, I, P,
                                    P]),
}

_lib = None


def load(path=None):
    """Load libwcs.so; raises OSError when the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with python -m paper_2203_13283_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class WCSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status, allow=()):
    if status != WCS_OK and status not in allow:
        raise WCSError(status, load().wcs_last_error().decode())
    return status
