"""ctypes loader for libmk.so and the ABI's structs (mirrors include/mk.h)."""
from __future__ import annotations

import ctypes
import os

MK_MAX_LEVELS = 12
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmk.so")

STATUS = {0: "MK_OK", 1: "MK_ERR_INVALID", 2: "MK_ERR_NOMEM", 3: "MK_ERR_CUDA",
          4: "MK_ERR_NONFINITE", 5: "MK_ERR_NOT_CONVERGED", 6: "MK_ERR_TIMEOUT",
          7: "MK_ERR_TOO_LARGE"}
MK_OK, MK_ERR_INVALID, MK_ERR_NOMEM, MK_ERR_CUDA, MK_ERR_NONFINITE, MK_ERR_NOT_CONVERGED, \
    MK_ERR_TIMEOUT, MK_ERR_TOO_LARGE = range(8)
# static scratch of mk_op_residual_noalloc
MK_NOALLOC_MAX_PARTIALS = 65536
MK_NOALLOC_CHUNK = 2048


class mk_stencil(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double)]


class mk_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("nu", ctypes.c_int32 * MK_MAX_LEVELS),
                ("space", ctypes.c_int32 * MK_MAX_LEVELS), ("m_inner", ctypes.c_int32 * MK_MAX_LEVELS),
                ("n_cgs", ctypes.c_int32), ("mu_mode", ctypes.c_int32), ("mu_value", ctypes.c_double),
                ("precision", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("orth", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("transfer", ctypes.c_int32),
                ("inner_kernel", ctypes.c_int32), ("augment", ctypes.c_int32)]

MK_TRANSFER_MK = 0      # Y, Z of Eq. (blockYZ) with Galerkin coarse levels
MK_TRANSFER_MGRIT = 1   # Eqs. (mgritY), (mgritZ) with the coarse matrix of Eq. (coarsemat)
MK_INNER_AUTO, MK_INNER_SEPARATE, MK_INNER_COOP = 0, 1, 2


class mk_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("f_norm", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int32),
                ("levels", ctypes.c_int32)]


class mk_level_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nt", ctypes.c_int32), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("mu", ctypes.c_double)]


class mk_tune_info(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("best_iterations", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("tune_ms", ctypes.c_double)]


MK_TUNE_LEVELS = 1
MK_TUNE_RESTART_CAP = 2

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int32

# name -> (restype, argtypes)
SIGNATURES = {
    "mk_default_opts": (None, [ctypes.POINTER(mk_solve_opts)]),
    "mk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mk_schedule_alternate": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                             ctypes.POINTER(mk_solve_opts)]),
    "mk_last_cuda_error": (ctypes.c_char_p, []),
    "mk_kernel_launch_count": (ctypes.c_int64, []),
    "mk_set_profiling": (None, [_I]),
    "mk_profile_reset": (None, []),
    "mk_profile_read": (ctypes.c_int, [_I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "mk_profile_class_name": (ctypes.c_char_p, [_I]),
    "mk_create_problem": (ctypes.c_int, [ctypes.POINTER(mk_stencil), _D, _D, _I, _P, ctypes.POINTER(_P)]),
    "mk_set_source": (ctypes.c_int, [_P, _P, _P]),
    "mk_destroy": (None, [_P]),
    "mk_trim": (ctypes.c_int, [_P]),
    "mk_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(mk_solve_opts), _P, ctypes.POINTER(mk_solve_info), _P]),
    "mk_create_batch": (ctypes.c_int, [_P, _I, ctypes.POINTER(mk_solve_opts), _I, ctypes.POINTER(_P)]),
    "mk_solve_batch": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(mk_solve_info), _P]),
    "mk_destroy_batch": (None, [_P]),
    "mk_solve_rhs": (ctypes.c_int, [_P, _P, ctypes.POINTER(mk_solve_opts), _P, ctypes.POINTER(mk_solve_info), _P]),
    "mk_march": (ctypes.c_int, [_P, _P, _P, _P]),
    "mk_tune": (ctypes.c_int, [_P, _P, ctypes.POINTER(mk_solve_opts), _I, _I,
                               ctypes.POINTER(mk_solve_opts), ctypes.POINTER(mk_tune_info), _P]),
    "mk_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(mk_solve_opts), _P, _P, _P, _P,
                                  ctypes.POINTER(mk_solve_info), _P]),
    "mk_problem_shape": (ctypes.c_int, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                        ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                        ctypes.POINTER(_D)]),
    "mk_level_info": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, ctypes.POINTER(mk_level_desc),
                                     _P, _P]),
    "mk_op_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "mk_op_apply": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, _I, _P, _P, _P]),
    "mk_op_residual": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "mk_op_residual_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "mk_op_restrict": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, _I, _P, _P, _P]),
    "mk_op_interp_correct": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, _I, _P, _P, _P, _P, _P]),
    "mk_op_interp_combine": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, _I, _P, _D, _P, _I,
                                            _P, _P, _P, _P]),
    "mk_op_coarsest": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, _P, _P, _P]),
    "mk_op_precond": (ctypes.c_int, [_P, ctypes.POINTER(mk_solve_opts), _I, _P, _P, _P]),
    "mk_op_orthogonalize": (ctypes.c_int, [_P, _I, _P, _P, _P, _P]),
    "mk_op_lsq": (ctypes.c_int, [_I, _P, _D, _P, ctypes.POINTER(_D), _P]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmk.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmk.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MKError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {STATUS.get(code, code)}"
        if code == MK_ERR_CUDA and _lib is not None:
            msg += f" ({_lib.mk_last_cuda_error().decode()})"
        super().__init__(msg)


def check(code: int, where: str, allow=()) -> int:
    if code != MK_OK and code not in allow:
        raise MKError(code, where)
    return code
