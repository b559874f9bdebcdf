"""ctypes declarations of include/jfnk.h (argument marshalling only)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# JFNK_LIB selects another build of the library (e.g. the bounds-checked one)
LIB_PATH = os.environ.get("JFNK_LIB") or os.path.join(HERE, "lib", "libjfnk.so")

MAX_LEVELS = 16
MAX_HIST = 64

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NONFINITE", 4: "NOT_CONVERGED", 5: "BREAKDOWN",
          6: "LINESEARCH", 7: "TIMEOUT", 8: "NOT_IMPLEMENTED", 9: "WORKSPACE"}
F32, F64 = 0, 1
BRATU2D, ND3D, NDK3D, MINSURF2D, BEAM3D = 0, 1, 2, 3, 4
KINDS = {"bratu2d": BRATU2D, "nd3d": ND3D, "ndk3d": NDK3D, "minsurf2d": MINSURF2D, "beam3d": BEAM3D}
EPS_PAPER, EPS_FP32 = 0, 1
RESTRICT, PROLONG_ADD, PROJECT = 0, 1, 2
OUTER_FGMRES, OUTER_CG = 0, 1
COARSE_GMRES, COARSE_CGQN = 0, 1


class ProblemDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_elem", ctypes.c_int), ("levels", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("load", ctypes.c_void_p), ("kappa", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double), ("power_iters", ctypes.c_int),
                ("power_tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_linear", ctypes.c_int),
                ("rtol_newton", ctypes.c_double), ("atol_newton", ctypes.c_double), ("eta_mode", ctypes.c_int),
                ("eta_max", ctypes.c_double), ("coarse_tol", ctypes.c_double), ("coarse_tol_mode", ctypes.c_int),
                ("coarse_maxit", ctypes.c_int), ("pc_dtype", ctypes.c_int), ("eps_mode_pc", ctypes.c_int),
                ("max_newton", ctypes.c_int), ("line_search", ctypes.c_int), ("ls_max", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("use_graph", ctypes.c_int),
                ("outer", ctypes.c_int), ("coarse_method", ctypes.c_int), ("lbfgs_pairs", ctypes.c_int),
                ("shift_gamma", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("linear_its", ctypes.c_int), ("status", ctypes.c_int),
                ("converged", ctypes.c_int), ("res_hist", ctypes.c_double * MAX_HIST),
                ("alpha_hist", ctypes.c_double * MAX_HIST), ("lin_hist", ctypes.c_int * MAX_HIST),
                ("ge", ctypes.c_double), ("nF", ctypes.c_longlong * MAX_LEVELS),
                ("lambda_max", ctypes.c_double * MAX_LEVELS), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("coarse_shifts", ctypes.c_int),
                ("coarse_negcurv", ctypes.c_int), ("outer_negcurv", ctypes.c_int),
                ("nJv", ctypes.c_longlong * MAX_LEVELS), ("ls_hist", ctypes.c_int * MAX_HIST)]


# (name, restype, argtypes) of every exported symbol declared in include/jfnk.h
_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = [
    ("jfnk_default_options", None, [ctypes.POINTER(Options)]),
    ("jfnk_paper_options", None, [ctypes.POINTER(Options)]),
    ("jfnk_problem_create", _i, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(_vp)]),
    ("jfnk_problem_destroy", _i, [_vp]),
    ("jfnk_workspace_size", _i, [_vp, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_size_t)]),
    ("jfnk_set_workspace", _i, [_vp, ctypes.POINTER(Options), _vp, ctypes.c_size_t, _vp]),
    ("jfnk_residual", _i, [_vp, _i, _i, _vp, _vp, _vp]),
    ("jfnk_jvp", _i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _d, _i, _vp]),
    ("jfnk_mg_setup", _i, [_vp, ctypes.POINTER(Options), _vp, _i, _vp]),
    ("jfnk_mg_vcycle", _i, [_vp, ctypes.POINTER(Options), _vp, _vp, _vp]),
    ("jfnk_solve", _i, [_vp, ctypes.POINTER(Options), _vp, ctypes.POINTER(Stats), _vp]),
    ("jfnk_solve_batched", _i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(Options), ctypes.POINTER(_vp),
                                ctypes.POINTER(Stats), _vp]),
    ("jfnk_transfer", _i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    ("jfnk_smooth", _i, [_vp, ctypes.POINTER(Options), _i, _vp, _vp, _i, _i, _vp]),
    ("jfnk_coarse_solve", _i, [_vp, ctypes.POINTER(Options), _vp, _vp, _vp]),
    ("jfnk_level_info", _i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d), _vp]),
    ("jfnk_level_vector", _i, [_vp, _i, _i, _vp, _vp]),
    ("jfnk_last_error", ctypes.c_char_p, []),
    ("jfnk_kernel_launches", ctypes.c_longlong, [_i]),
    ("jfnk_jvp_noalloc", _i, [_i, _i, _d, _vp, _vp, _i, _vp, _vp, _vp, _vp, _d, _i, _vp]),
    ("jfnk_vjp", _i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    ("jfnk_set_kappa", _i, [_vp, _vp, _vp]),
    ("jfnk_adjoint_solve", _i, [_vp, ctypes.POINTER(Options), _vp, _vp, _vp, _vp, _d, ctypes.POINTER(Stats), _vp]),
    ("jfnk_measure_peaks", _i, [ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d), _vp]),
    ("jfnk_debug_bounds", _i, [ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_uint), _i]),
    ("jfnk_profile_enable", None, [_i]),
    ("jfnk_profile_read", _i, [_i, ctypes.c_char_p, _i, ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(_d), ctypes.POINTER(_d)]),
]


def load_library(path=LIB_PATH):
    """Load libjfnk.so and attach the signatures.  Raises if it is missing: there
    is no fallback implementation."""
    if not os.path.exists(path):
        raise RuntimeError(f"libjfnk.so not found at {path}; build it with "
                           "`python -m paper_2103_13890_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
