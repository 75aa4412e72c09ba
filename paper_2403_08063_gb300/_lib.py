"""ctypes binding of libocmg.so (include/octmg.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  There is no CPU fallback: if the shared library
has not been built (``__graft_entry__.build()`` or ``python -m paper_2403_08063_gb300.build``) loading fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libocmg.so")

MG_STATUS = {
    0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_UNBALANCED", 3: "MG_ERR_BLOCK_SIZE", 4: "MG_ERR_OOM",
    5: "MG_ERR_CUDA", 6: "MG_ERR_NOT_CONVERGED", 7: "MG_ERR_TIMEOUT", 8: "MG_ERR_NONFINITE", 9: "MG_ERR_STATE",
}


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{MG_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = MG_STATUS.get(status, str(status))


class MGConfig(ctypes.Structure):
    _fields_ = [
        ("roots", ctypes.c_int32),
        ("n", ctypes.c_int32),
        ("n_leaves", ctypes.c_int32),
        ("leaves", ctypes.POINTER(ctypes.c_int32)),
        ("coeff", ctypes.c_int32),
        ("interface_flux", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("nu1", ctypes.c_int32),
        ("nu2", ctypes.c_int32),
        ("max_coarse", ctypes.c_int32),
        ("inner_cycles", ctypes.c_int32),
        ("n_problems", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("c2f_variant", ctypes.c_int32),
        ("smoother", ctypes.c_int32),
        ("omega", ctypes.c_double),
        ("coarse_iters", ctypes.c_int32),
        ("coarse_coef", ctypes.c_int32),
        ("prolongation", ctypes.c_int32),
    ]


_c = ctypes
P = _c.c_void_p
I32 = _c.c_int32
DP = _c.POINTER(_c.c_double)
IP = _c.POINTER(_c.c_int32)

# name -> (restype, argtypes); every symbol include/octmg.h declares
SIGNATURES = {
    "mg_forest_create": (I32, [_c.POINTER(MGConfig), _c.POINTER(P)]),
    "mg_forest_destroy": (None, [P]),
    "mg_forest_levels": (I32, [P, IP, IP, IP]),
    "mg_level_keys": (I32, [P, I32, IP]),
    "mg_set_rhs": (I32, [P, P, P]),
    "mg_set_boundary": (I32, [P, P]),
    "mg_vcycle": (I32, [P, P, I32, DP]),
    "mg_solve": (I32, [P, P, _c.c_double, I32, IP, DP]),
    "mg_solve_host": (I32, [P, P, P, P, P, _c.c_double, I32, IP, DP]),
    "mg_adjoint_solve": (I32, [P, P, P, P, P, _c.c_double, I32]),
    "mg_apply": (I32, [P, P, P]),
    "mg_apply_transpose": (I32, [P, P, P]),
    "mg_exchange_level": (I32, [P, I32, P, P]),
    "mg_exchange_level_noalloc": (I32, [P, I32, P, P]),
    "mg_profile": (I32, [P, I32]),
    "mg_smoother_shapes": (I32, [P, I32, I32, IP, IP]),
    "mg_staged_copy_plan": (I32, [I32, I32, I32, I32, IP, IP, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64),
                                  _c.c_int64, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64)]),
    "mg_restrict_copy_plan": (I32, [I32, I32, IP, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64), _c.c_int64,
                                    _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64)]),
    "mg_get_tail": (I32, [P, IP]),
    "mg_set_tail": (I32, [P, I32]),
    "mg_selftest_waits": (I32, [P, I32]),
    "mg_alu_peaks": (I32, [DP, DP]),
    "mg_get_smoother_shape": (I32, [P, I32, IP]),
    "mg_set_smoother_shape": (I32, [P, I32, IP]),
    "mg_profile_read": (I32, [P, I32, _c.c_char_p, DP, _c.POINTER(_c.c_int64), IP]),
    "mg_batch_create": (I32, [_c.POINTER(MGConfig), IP, _c.POINTER(P)]),
    "mg_batch_destroy": (None, [P]),
    "mg_batch_set_rhs": (I32, [P, P, P]),
    "mg_batch_solve": (I32, [P, P, _c.c_double, I32, IP, DP]),
    "mg_batch_info": (I32, [P, IP, _c.POINTER(_c.c_int64), IP, IP]),
    "mg_batch_profile": (I32, [P, I32]),
    "mg_batch_group": (P, [P, I32]),
    "mg_batch_set_tail_mode": (I32, [P, I32]),
    "mg_batch_get_tail_mode": (I32, [P, IP]),
    "mg_last_error": (_c.c_char_p, []),
}

_LIB = None


def load(path: str = LIB_PATH):
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int):
    if status != 0:
        msg = load().mg_last_error().decode(errors="replace")
        raise MGError(status, msg)
