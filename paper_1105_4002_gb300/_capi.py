"""ctypes declarations of libtvr.so (include/tvr.h).  Loading fails loudly when
the CUDA library has not been built: there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtvr.so")

TVR_OK = 0
TVR_NOT_CONVERGED = 1
TVR_ERR_ARG = -1
TVR_ERR_OOM = -2
TVR_ERR_CUDA = -3
TVR_ERR_LINESEARCH = -4
TVR_ERR_NONFINITE = -5

TVR_CONE = 0
TVR_PARALLEL = 1
TVR_STORAGE_FP32 = 0
TVR_STORAGE_BF16_ROWSCALE = 1
TVR_STORAGE_MATRIX_FREE = 2
TVR_STORAGE_U16_ROWSCALE = 3
TVR_STOP_REL = 0
TVR_STOP_PER_N = 1
TVR_VIEW_FIELDS = 12
TVR_HIST_FIELDS = 8


class Geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_views", ctypes.c_int32), ("det_cols", ctypes.c_int32),
                ("det_rows", ctypes.c_int32), ("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("views", ctypes.c_void_p)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("stop_mode", ctypes.c_int32), ("gpbb_K", ctypes.c_int32),
                ("gpbb_max_trials", ctypes.c_int32), ("bt_max", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("gpbb_points", ctypes.c_int32), ("sweep_lanes", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("gpbb_sigma", ctypes.c_double), ("gpbb_beta0", ctypes.c_double),
                ("rho_L", ctypes.c_double), ("L_bar", ctypes.c_double), ("mu_bar", ctypes.c_double),
                ("history", ctypes.c_void_p), ("history_len", ctypes.c_int64)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("f_evals", ctypes.c_int32),
                ("g_evals", ctypes.c_int32), ("trials", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("history_used", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("phi", ctypes.c_double), ("gnorm", ctypes.c_double), ("gnorm0", ctypes.c_double),
                ("stop_value", ctypes.c_double), ("L", ctypes.c_double), ("theta", ctypes.c_double),
                ("mu", ctypes.c_double)]


# every function declared in include/tvr.h: name -> (restype, argtypes)
_P = ctypes.c_void_p
_D = ctypes.c_double
_I64 = ctypes.c_int64
SIGNATURES = {
    "tvr_build_system": (ctypes.c_int, [ctypes.POINTER(Geometry), ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "tvr_system_free": (ctypes.c_int, [_P]),
    "tvr_system_shape": (ctypes.c_int, [_P, _P, _P, _P]),
    "tvr_system_export_csr": (ctypes.c_int, [_P, _P, _P, _P]),
    "tvr_system_export_csc": (ctypes.c_int, [_P, _P, _P, _P]),
    "tvr_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "tvr_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "tvr_phi_and_grad": (ctypes.c_int, [_P, _P, _P, _D, _D, _P, _P, _P, _P, _P]),
    "tvr_phi_and_grad_noalloc": (ctypes.c_int, [_P, _P, _P, _D, _D, _P, _P, _P, _P]),
    "tvr_phi_and_grad_f64": (ctypes.c_int, [_P, _P, _P, _D, _D, _P, _P, _P, _P, _P]),
    "tvr_phi_vjp": (ctypes.c_int, [_P, _P, _P, _D, _D, _P, _P, _P, _P]),
    "tvr_phi_vjp_f64": (ctypes.c_int, [_P, _P, _P, _D, _D, _P, _P, _P, _P]),
    "tvr_project_Q": (ctypes.c_int, [_P, _I64, _P]),
    "tvr_gradient_map_norm": (ctypes.c_int, [_P, _P, _P, _D, _P, _P]),
    "tvr_trial_sums": (ctypes.c_int, [_P, _P, _P, _P, _D, _D, _P, _P, _P, _P]),
    "tvr_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "tvr_solve_gp": (ctypes.c_int, [_P, _P, _D, _D, _D, ctypes.POINTER(SolveOpts), _P,
                                    ctypes.POINTER(SolveInfo), _P]),
    "tvr_solve_gpbb": (ctypes.c_int, [_P, _P, _D, _D, _D, ctypes.POINTER(SolveOpts), _P,
                                      ctypes.POINTER(SolveInfo), _P]),
    "tvr_solve_upn": (ctypes.c_int, [_P, _P, _D, _D, _D, ctypes.POINTER(SolveOpts), _P,
                                     ctypes.POINTER(SolveInfo), _P]),
    "tvr_solve_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _D, _D,
                                       ctypes.POINTER(SolveOpts), _P, ctypes.POINTER(SolveInfo), _P]),
    "tvr_solve_sweep": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _D, _D,
                                       ctypes.POINTER(SolveOpts), _P, ctypes.POINTER(SolveInfo), _P]),
    "tvr_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tvr_profile_read": (ctypes.c_int, [_P, _P, _P]),
    "tvr_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tvr_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libtvr.so with typed entry points (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libtvr.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                "python -m paper_1105_4002_gb300.build -- there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class TVRError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.tvr_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.tvr_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str, allow=(TVR_OK,)) -> int:
    if status not in allow:
        raise TVRError(status, where)
    return status
