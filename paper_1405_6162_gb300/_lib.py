"""ctypes declarations of liblb's C ABI (include/lb.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading



from . import nvbuild as _build

LB_OK = 0
LB_ERR_INVALID = -1
LB_ERR_NOMEM = -2
LB_ERR_CUDA = -3
LB_ERR_NONFINITE = -4
LB_ERR_TIMEOUT = -5

LB_FP64 = 0
LB_FP32_SHIFTED = 1
LB_FP64_DF = 2
LB_HOST = 0
LB_DEVICE = 1
LB_COLLISION_BGK = 0
LB_COLLISION_MRT = 1

LB_KERNEL_AUTO = 0
LB_KERNEL_TWO_PASS = 1
LB_KERNEL_FUSED = 2
LB_KERNEL_STAGED = 3
LB_KERNEL_SLAB = 4
LB_KERNEL_LAG = 5
LB_KERNEL_TAUG1 = 6
LB_KERNEL_BULK = 7


class lb_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("tau_g", ctypes.c_double), ("rho0", ctypes.c_double),
                ("gamma", ctypes.c_double), ("A", ctypes.c_double), ("B", ctypes.c_double),
                ("kappa", ctypes.c_double), ("precision", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "lb_set_allocator": (_I, [ALLOC_FN, FREE_FN, _P]),
    "lb_create": (_I, [ctypes.POINTER(lb_params), _P, ctypes.POINTER(_P)]),
    "lb_destroy": (None, [_P]),
    "lb_init": (_I, [_P, _P, _P, _I]),
    "lb_step": (_I, [_P, _I]),
    "lb_moments": (_I, [_P, _P, _P, _P, _I]),
    "lb_reduce": (_I, [_P, _P]),
    "lb_get_state": (_I, [_P, _P, _P, _I]),
    "lb_set_state": (_I, [_P, _P, _P, _I]),
    "lb_set_kernel": (_I, [_P, _I, _I, _I, _I]),
    "lb_set_stencil": (_I, [_P, _I]),
    "lb_moments_masked": (_I, [_P, _P, _P, _P, _P, _P, _I]),
    "lb_get_state_masked": (_I, [_P, _P, _P, _P, _P, _I]),
    "lb_set_state_masked": (_I, [_P, _P, _P, _P, _I]),
    "lb_set_collision": (_I, [_P, _I, ctypes.c_double, ctypes.c_double]),
    "lb_set_force": (_I, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lb_get_info": (_I, [_P, _P, _P, _P, _P]),
    "lb_sync": (_I, [_P]),
    "lb_set_wait_timeout": (_I, [_P, ctypes.c_longlong]),
    "lb_debug_wait_skew": (_I, [_P, ctypes.c_ulonglong]),
    "lb_step_fp64_noalloc": (_I, [ctypes.POINTER(lb_params), _P, _P, _P, _P, _P]),
    "lb_adjoint_step": (_I, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "lb_adjoint_seed": (_I, [_P, _P, _P, _P]),
    "lb_adjoint_init": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "lb_batch_create": (_I, [_I, ctypes.POINTER(lb_params), _P, ctypes.POINTER(_P)]),
    "lb_batch_destroy": (None, [_P]),
    "lb_batch_lattice": (_P, [_P, _I]),
    "lb_batch_run": (_I, [_P, _I]),
    "lb_batch_sync": (_I, [_P]),
    "lb_batch_set_launch": (_I, [_P, _I, _I]),
    "lb_batch_set_form": (_I, [_P, _I]),
    "lb_batch_size": (_I, [_P, _P, _P, _P, _P]),
    "lb_batch_groups": (_I, [_P, _P]),
    "lb_batch_set_plan": (_I, [_P, _I]),
    "lb_batch_plan": (_I, [_I, _P, _I, _I, _P, _P, _P, _P]),
    "lb_batch_set_wait_timeout": (_I, [_P, ctypes.c_longlong]),
    "lb_batch_debug_skip_arrival": (_I, [_P, _I]),
    "lb_probe_fp64_fma": (_I, [_I, ctypes.c_longlong, _P, _P, _P]),
    "lb_strerror": (ctypes.c_char_p, [_I]),
    "lb_last_error": (ctypes.c_char_p, []),
}

_LIB = None
_LOCK = threading.Lock()


class LBError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        lib = _LIB
        msg = lib.lb_strerror(code).decode() if lib else str(code)
        extra = lib.lb_last_error().decode() if (lib and code == LB_ERR_CUDA) else ""
        super().__init__(f"{where}: {msg}" + (f" ({extra})" if extra else ""))


def lib():
    """The loaded liblb (raises if it is missing)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"liblb.so is not built ({path}); run paper_1405_6162_gb300.build.build() "
                    "-- there is no CPU fallback")
            h = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = h
        return _LIB


def check(rc: int, where: str) -> None:
    if rc != LB_OK:
        raise LBError(rc, where)
