"""ctypes declarations of the C ABI in include/gmres_gb300.h (argument marshalling only).

The shared library must exist (built by ``paper_1906_04051_gb300.build``); there is no
fallback of any kind: every entry point runs the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmres_gb300.so")

GMRES_OK = 0
GMRES_NOT_CONVERGED = 1
GMRES_ERR_INVALID_ARG = -1
GMRES_ERR_CUDA = -2
GMRES_ERR_OOM = -3
GMRES_ERR_SINGULAR_COARSE = -4
GMRES_ERR_NAN = -5
GMRES_ERR_TIMEOUT = -6
STATUS_NAMES = {
    0: "OK", 1: "NOT_CONVERGED", -1: "ERR_INVALID_ARG", -2: "ERR_CUDA", -3: "ERR_OOM",
    -4: "ERR_SINGULAR_COARSE", -5: "ERR_NAN", -6: "ERR_TIMEOUT",
}

FP64, FP32_INNER, BF16_BASIS = 0, 1, 2
DEFL_EBP, DEFL_PROJECTOR, DEFL_NONE, DEFL_ADAPTIVE = 0, 1, 2, 3
MU_RITZ_FIRST_CYCLE, MU_USER, MU_NORM_INF = 0, 1, 2
ORTHO_CGS2, ORTHO_MGS, ORTHO_MGS_LOWSYNC = 0, 1, 2
DOT_FP64, DOT_DF32 = 0, 1
PHASES = ["setup", "residual", "spmv", "dot1", "upd1dot2", "upd2norm", "defl", "cycle_end",
          "ritz", "proj_final", "adapt", "mgs", "arnoldi"]


class gmres_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class gmres_defl(C.Structure):
    _fields_ = [("r", C.c_int32), ("agg", C.c_void_p), ("dense", C.c_void_p)]


class gmres_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("deflation_mode", C.c_int32),
                ("mu_mode", C.c_int32), ("mu_user", C.c_double),
                ("fixed_iterations", C.c_int32), ("r0_norm_ref", C.c_double),
                ("timeout_ms", C.c_int32), ("inner_tol", C.c_double),
                ("profile", C.c_int32), ("rmax", C.c_int32), ("ninv", C.c_int32),
                ("ortho", C.c_int32), ("dot_arith", C.c_int32)]


class gmres_info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("cycles", C.c_int64), ("refinements", C.c_int64),
                ("rel_res_est", C.c_double), ("rel_res_true", C.c_double),
                ("mu", C.c_double), ("ms_total", C.c_float), ("status", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class gmres_layout(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("r", C.c_int32), ("npieces", C.c_int32),
                ("ndiag", C.c_int32), ("adapt_q", C.c_int32), ("nau", C.c_int64),
                ("ldv", C.c_int64), ("spmv_lanes", C.c_int32), ("coarse_band", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class q2_newton_info(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("status", C.c_int32),
                ("gmres_iters", C.c_int64), ("du_inf", C.c_double),
                ("last_rel_res", C.c_double), ("ms_total", C.c_float),
                ("ms_assemble", C.c_float), ("ms_solve", C.c_float), ("reserved", C.c_int32),
                ("step_iters", C.c_int64 * 32), ("step_du", C.c_double * 32)]

    def as_dict(self) -> dict:
        k = min(self.newton_iters, 32)
        out = {f: getattr(self, f) for f, _ in self._fields_
               if f not in ("reserved", "step_iters", "step_du")}
        out["step_iters"] = list(self.step_iters[:k])
        out["step_du"] = list(self.step_du[:k])
        return out


# name -> (restype, argtypes); every symbol declared in include/gmres_gb300.h
_P = C.c_void_p
SIGNATURES = {
    "gmres_opts_default": (None, [C.POINTER(gmres_opts)]),
    "gmres_create": (C.c_int, [C.POINTER(_P), C.POINTER(gmres_csr), C.POINTER(gmres_defl),
                               C.POINTER(gmres_opts), _P]),
    "gmres_solve": (C.c_int, [_P, _P, _P, C.c_int32, C.c_double, C.c_int64, _P,
                              C.POINTER(gmres_info)]),
    "gmres_adjoint_solve": (C.c_int, [_P, _P, _P, C.c_int32, C.c_double, C.c_int64, _P,
                                      C.POINTER(gmres_info)]),
    "gmres_solve_noalloc": (C.c_int, [_P, _P, _P, C.c_int32, C.c_double, C.c_int64, _P,
                                      C.POINTER(gmres_info)]),
    "gmres_batch_solve": (C.c_int, [C.c_int32, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                    C.c_int32, C.c_double, C.c_int64, C.POINTER(_P),
                                    C.POINTER(gmres_info), _P]),
    "gmres_layout_query": (C.c_int, [_P, C.POINTER(gmres_layout)]),
    "gmres_adaptive_space": (C.c_int, [_P, C.POINTER(C.c_int32), _P, C.c_int64, _P]),
    "gmres_set_stream": (C.c_int, [_P, _P]),
    "gmres_profile": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                C.POINTER(C.c_int64)]),
    "gmres_last_error": (C.c_char_p, [_P]),
    "gmres_destroy": (None, [_P]),
    "q1_nnz": (C.c_int64, [C.c_int32]),
    "q1_assemble": (C.c_int, [C.c_int32, _P, C.c_double, C.c_double, _P, _P, _P, _P, _P, _P,
                              _P]),
    "q1_kappa_grad": (C.c_int, [C.c_int32, _P, _P, _P, _P]),
    "q2_nnz": (C.c_int64, [C.c_int32]),
    "q2_bratu_assemble": (C.c_int, [C.c_int32, C.c_double, _P, _P, _P, _P, _P, _P]),
    "q2_bratu_newton": (C.c_int, [C.c_int32, C.c_double, C.POINTER(gmres_opts),
                                  C.POINTER(gmres_defl), C.c_int32, C.c_double, C.c_int64,
                                  C.c_double, C.c_int32, _P, C.POINTER(q2_newton_info), _P]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Loads the library (once).  Raises if it has not been built: no fallback exists."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"{p} is missing: build it with `python -m paper_1906_04051_gb300.build` "
                    "(the CUDA library is the only implementation)")
            L = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class GmresError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
