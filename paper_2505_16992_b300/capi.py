"""ctypes binding of the C ABI in include/piso.h (argument marshalling only).

Loading fails loudly when ``libpiso.so`` is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpiso.so")

PISO_FP64, PISO_FP32 = 0, 1
PISO_GRAD_ADV, PISO_GRAD_P = 1, 2          # piso_options.grad_paths bits (Sec. 2.4 gradient paths)
PISO_PRECOND_AUTO, PISO_PRECOND_JACOBI, PISO_PRECOND_LINE = 0, 1, 2   # piso_options.p_precond
PISO_ADV_PRECOND_NONE, PISO_ADV_PRECOND_ILU, PISO_ADV_PRECOND_ILU_ON_FAILURE = 0, 1, 2   # .adv_precond
STATUS = {0: "PISO_OK", 1: "PISO_EINVAL", 2: "PISO_ECUDA", 3: "PISO_ENOCONV", 4: "PISO_EBREAKDOWN",
          5: "PISO_ENAN", 6: "PISO_ETIMEOUT", 7: "PISO_ESTATE", 8: "PISO_ENOMEM"}


class Options(C.Structure):
    _fields_ = [("n_correctors", C.c_int32), ("pred_grad_p", C.c_int32), ("adv_rtol", C.c_double),
                ("p_rtol", C.c_double), ("atol", C.c_double), ("adv_maxit", C.c_int32),
                ("p_maxit", C.c_int32), ("block_threads", C.c_int32), ("ctas", C.c_int32),
                ("timeout_s", C.c_double), ("fault_withhold_cta", C.c_int32), ("p_refine_rtol", C.c_double),
                ("p_inner_rtol", C.c_double), ("grad_paths", C.c_int32), ("p_precond", C.c_int32),
                ("adv_precond", C.c_int32), ("n_nonortho", C.c_int32), ("p_line_split", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("error_bits", C.c_int32), ("adv_iters", C.c_int32 * 3),
                ("p_iters", C.c_int32 * 4), ("adv_resid", C.c_double * 3), ("p_resid", C.c_double * 4),
                ("p_rounds", C.c_int32 * 4), ("p_rhs_norm", C.c_double * 4), ("adv_precond_used", C.c_int32)]

    def as_dict(self):
        return dict(status=STATUS.get(self.status, self.status), error_bits=self.error_bits,
                    adv_iters=list(self.adv_iters), p_iters=list(self.p_iters),
                    adv_resid=list(self.adv_resid), p_resid=list(self.p_resid), p_rounds=list(self.p_rounds),
                    p_rhs_norm=list(self.p_rhs_norm), adv_precond_used=self.adv_precond_used)


class PisoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "piso_version": (C.c_char_p, []),
    "piso_default_options": (None, [C.POINTER(Options)]),
    "piso_domain_create": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(_P)]),
    "piso_block_add": (C.c_int, [_P, C.POINTER(C.c_int32), _D, C.POINTER(C.c_int32)]),
    "piso_connect": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "piso_set_dirichlet": (C.c_int, [_P, C.c_int32, C.c_int32, _D]),
    "piso_set_advective_outflow": (C.c_int, [_P, C.c_int32, C.c_int32, _D, _D]),
    "piso_finalize": (C.c_int, [_P, C.POINTER(Options)]),
    "piso_set_options": (C.c_int, [_P, C.POINTER(Options)]),
    "piso_get_options": (C.c_int, [_P, C.POINTER(Options)]),
    "piso_pressure_precond": (C.c_int32, [_P]),
    "piso_pressure_line_fused": (C.c_int32, [_P]),
    "piso_pressure_cg_vec4": (C.c_int32, [_P]),
    "piso_num_cells": (C.c_int64, [_P]),
    "piso_num_boundary_faces": (C.c_int32, [_P]),
    "piso_tape_bytes": (C.c_size_t, [_P]),
    "piso_step": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_double, _P, _P, _P, C.POINTER(Stats)]),
    "piso_last_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "piso_step_static": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_double, _P, _P, C.POINTER(Stats)]),
    "piso_autotune": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, _P, _P, C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "piso_step_adjoint": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _D, _P, C.POINTER(Stats)]),
    "piso_get_boundary": (C.c_int, [_P, _D]),
    "piso_set_boundary": (C.c_int, [_P, _D]),
    "piso_get_boundary_adjoint": (C.c_int, [_P, _D]),
    "piso_last_error": (C.c_char_p, [_P]),
    "piso_domain_destroy": (None, [_P]),
    "piso_batch_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(Options), C.POINTER(_P)]),
    "piso_batch_step": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), _D, _D,
                                  C.POINTER(_P), _P, C.POINTER(Stats)]),
    "piso_batch_step_adjoint": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                          C.POINTER(_P), _D, _P, C.POINTER(Stats)]),
    "piso_batch_autotune": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), _D, _D, C.POINTER(_P), _P,
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      _D]),
    "piso_batch_destroy": (None, [_P]),
    "piso_stats_create": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(_P)]),
    "piso_stats_record_size": (C.c_int32, [_P]),
    "piso_stats_planes": (C.c_int32, [_P]),
    "piso_stats_frame": (C.c_int, [_P, _P, _P, _P, _P]),
    "piso_stats_merge": (C.c_int, [_P, _P, _P, _P]),
    "piso_stats_frame_adjoint": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "piso_cell_gradients": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "piso_stats_budget": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_double, _P, _P]),
    "piso_stats_destroy": (None, [_P]),
}

_lib = None


def load():
    """Load libpiso.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2505_16992_b300._build.build() "
                              "(the CUDA path has no fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    load().piso_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def check(status, handle=None):
    if status != 0:
        msg = load().piso_last_error(handle)
        raise PisoError(status, msg.decode() if msg else "")


def dptr(x):
    """Device address of a tensor (or None/0 for NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x or None
    return x.data_ptr()


def dbuf(arr):
    import numpy as np
    a = np.ascontiguousarray(arr, dtype=np.float64)
    return a, a.ctypes.data_as(_D)
