"""ctypes declarations of the libdgns C ABI (include/dgns.h).

Argument marshalling only: every computation runs in the CUDA library.  The
library must exist (``build()`` compiles it); there is no fallback.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libdgns.so")

DGNS_OK = 0
DGNS_ERR_INVALID_ARG = 1
DGNS_ERR_CUDA = 2
DGNS_ERR_OOM = 3
DGNS_ERR_NOT_CONVERGED = 4
DGNS_ERR_NONFINITE = 5
DGNS_ERR_ALIAS = 6
DGNS_ERR_UNSUPPORTED = 7
SPACE_U = 0
# terms of the projection operator (dgns_vmult_projection_terms)
PROJ_MASS, PROJ_DIV, PROJ_CONT, PROJ_ALL = 1, 2, 4, 7
SPACE_P = 1
MAX_LEVELS = 16


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("degree", ctypes.c_int),
                ("degree_p", ctypes.c_int), ("n_q_conv", ctypes.c_int),
                ("penalty_factor", ctypes.c_double), ("nu", ctypes.c_double),
                ("mg_coarse_n", ctypes.c_int), ("mg_precision", ctypes.c_int),
                ("fp64_mode", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("smoothing_range", ctypes.c_double), ("cheb_coarse_iters", ctypes.c_int),
                ("project_mean", ctypes.c_int), ("use_initial_guess", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("initial_res", ctypes.c_double), ("status", ctypes.c_int),
                ("lambda_max_fine", ctypes.c_double), ("seconds", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong

# name -> (restype, argtypes)
SIGNATURES = {
    "dgns_default_desc": (None, [ctypes.POINTER(MeshDesc)]),
    "dgns_create": (_I, [ctypes.POINTER(MeshDesc), _P, ctypes.POINTER(_P)]),
    "dgns_destroy": (_I, [_P]),
    "dgns_set_stream": (_I, [_P, _P]),
    "dgns_debug_fail_alloc": (_I, [_LL]),
    "dgns_debug_conv_mix": (_I, [_I, _I]),
    "dgns_debug_laplace_f32_kernel": (_I, [_I]),
    "dgns_debug_laplace_f32_timeouts": (ctypes.c_longlong, []),
    "dgns_debug_live_allocations": (_LL, []),
    "dgns_debug_widen_f32": (_I, [_P, _P, _LL]),
    "dgns_status_string": (ctypes.c_char_p, [_I]),
    "dgns_last_error": (ctypes.c_char_p, []),
    "dgns_sizes": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "dgns_nodes_1d": (_I, [_P, _I, _P]),
    "dgns_vmult_laplace": (_I, [_P, _P, _P, _I]),
    "dgns_vmult_laplace_split": (_I, [_P, _P, _P, _I]),
    "dgns_vmult_laplace_f32": (_I, [_P, _P, _P, _I]),
    "dgns_laplace_diagonal": (_I, [_P, _P, _I]),
    "dgns_vmult_viscous": (_I, [_P, _P, _P]),
    "dgns_vmult_helmholtz": (_I, [_P, _P, _P, _D]),
    "dgns_vmult_mass": (_I, [_P, _P, _P, _I, _I]),
    "dgns_apply_inverse_mass": (_I, [_P, _P, _P, _I, _I]),
    "dgns_vmult_divergence": (_I, [_P, _P, _P]),
    "dgns_vmult_gradient": (_I, [_P, _P, _P]),
    "dgns_vmult_convective": (_I, [_P, _P, _P]),
    "dgns_convective_face_size": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "dgns_convective_faces": (_I, [_P, _P, _P]),
    "dgns_convective_cells": (_I, [_P, _P, _P, _P]),
    "dgns_vjp_convective": (_I, [_P, _P, _P, _P]),
    "dgns_dissipation": (_I, [_P, _P, ctypes.POINTER(_D)]),
    "dgns_dissipation_grad": (_I, [_P, _P, _P]),
    "dgns_axpby": (_I, [_P, _P, _P, _LL, _D, _D]),
    "dgns_dot": (_I, [_P, _P, _P, _LL, ctypes.POINTER(_D)]),
    "dgns_penalty_parameters": (_I, [_P, _P, _D, _D, _D, _P, _P]),
    "dgns_vmult_projection": (_I, [_P, _P, _P, _P, _P]),
    "dgns_vmult_projection_terms": (_I, [_P, _P, _P, _P, _P, _I]),
    "dgns_mg_chebyshev_step_f32": (_I, [_P, _P, _P, _P, _P, _D, _D, _I]),
    "dgns_cg_projection_solve": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(SolveParams),
                                      ctypes.POINTER(SolveInfo)]),
    "dgns_default_solve_params": (None, [ctypes.POINTER(SolveParams)]),
    "dgns_cg_mg_solve": (_I, [_P, _P, _P, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
    "dgns_mg_info": (_I, [_P, ctypes.POINTER(_I), _P, _P]),
    "dgns_mg_vcycle": (_I, [_P, _P, _P, ctypes.POINTER(SolveParams)]),
    "dgns_mg_prolongate_f32": (_I, [_P, _P, _P, _I]),
    "dgns_mg_restrict_f32": (_I, [_P, _P, _P, _I]),
    "dgns_cg_invmass_solve": (_I, [_P, _P, _P, _D, ctypes.POINTER(SolveParams),
                                   ctypes.POINTER(SolveInfo)]),
    "dgns_cg_invmass_solve_noalloc": (_I, [_P, _P, _P, _D, ctypes.POINTER(SolveParams),
                                           ctypes.POINTER(SolveInfo)]),
}

_lib = None


def load(path=None):
    """Load libdgns.so (once) and declare every entry point."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libdgns.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_1802_01439_gb300.build" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class DgnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dgns error %d (%s): %s" % (code, load().dgns_status_string(code).decode(), msg))
        self.code = code


def check(rc):
    if rc != DGNS_OK:
        raise DgnsError(rc, load().dgns_last_error().decode())
    return rc
