"""ctypes binding of libcheb (include/cheb.h): argument marshalling only.

Every step of the computation runs in the CUDA library. If libcheb.so is
missing this module raises instead of falling back to anything else. Tensors
are torch CUDA tensors; torch provides the device memory and the streams.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcheb.so")
# the checked build (device bounds checks, CHEB_EBOUNDS), chosen for a process
# by CHEB_LIBRARY=check before the first load()
LIB_CHECK_PATH = os.path.join(HERE, "libcheb_check.so")

CHEB_OK, CHEB_EINVAL, CHEB_ENOMEM, CHEB_ECUDA, CHEB_ENOCONV, CHEB_ESTALL, CHEB_ETIMEOUT, \
    CHEB_EUNSUPPORTED, CHEB_EBOUNDS = range(9)
STATUS_NAMES = {0: "CHEB_OK", 1: "CHEB_EINVAL", 2: "CHEB_ENOMEM", 3: "CHEB_ECUDA", 4: "CHEB_ENOCONV",
                5: "CHEB_ESTALL", 6: "CHEB_ETIMEOUT", 7: "CHEB_EUNSUPPORTED", 8: "CHEB_EBOUNDS"}
CHEB_FP64, CHEB_TF32X3, CHEB_BF16X3, CHEB_BF16X6 = range(4)
CHEB_DF64 = 4
CHEB_WAIT_LIMIT_DEFAULT = 1 << 32
PRECISIONS = {"fp64": CHEB_FP64, "tf32x3": CHEB_TF32X3, "bf16x3": CHEB_BF16X3, "bf16x6": CHEB_BF16X6,
              "df64": CHEB_DF64}


class ChebError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GameParams(C.Structure):
    _fields_ = [("J", C.c_int32), ("K", C.c_double * 16), ("m", C.c_double),
                ("A", C.c_double * 4), ("beta", C.c_double * 4), ("phi", C.c_double * 4),
                ("c", C.c_double * 4), ("rho", C.c_double), ("gamma", C.c_double * 16)]


class GameOpts(C.Structure):
    _fields_ = [("h", C.c_double), ("P_M", C.c_double), ("U_M", C.c_double), ("tol", C.c_double),
                ("n", C.c_int32), ("n_u", C.c_int32), ("max_iter", C.c_int64), ("prec", C.c_int32),
                ("polish_fp64", C.c_int32), ("g_interp", C.c_int32)]


class GameResult(C.Structure):
    _fields_ = [("V", C.c_void_p), ("u", C.c_void_p), ("V0", C.c_void_p), ("u0", C.c_void_p),
                ("iters", C.c_int64), ("iters_split", C.c_int64), ("residual", C.c_double),
                ("status", C.c_int32), ("Vn", C.c_void_p), ("restarts", C.c_int32)]


_lib = None


def library_path() -> str:
    """libcheb.so, or libcheb_check.so when CHEB_LIBRARY=check."""
    v = os.environ.get("CHEB_LIBRARY", "")
    if v not in ("", "default", "check"):
        raise RuntimeError(f"CHEB_LIBRARY must be 'check' or unset, not {v!r}")
    return LIB_CHECK_PATH if v == "check" else LIB_PATH


def load():
    """Load libcheb.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run __graft_entry__.build() first")
    L = C.CDLL(path)
    vp, ip = C.c_void_p, C.POINTER(C.c_int32)
    dp = C.POINTER(C.c_double)
    L.cheb_create.argtypes = [C.POINTER(vp), C.c_int]
    L.cheb_destroy.argtypes = [vp]
    L.cheb_last_error.restype = C.c_char_p
    L.cheb_version.restype = C.c_char_p
    L.cheb_device_status.argtypes = [vp]
    L.cheb_fit.argtypes = [vp, C.c_int, ip, vp, vp, vp]
    L.cheb_eval_grid.argtypes = [vp, C.c_int, ip, vp, dp, dp, ip, C.POINTER(vp), vp, C.c_int, vp]
    L.cheb_eval_grid_host.argtypes = [vp, C.c_int, ip, vp, dp, dp, ip, C.POINTER(vp), vp, C.c_int, vp]
    L.cheb_eval_points.argtypes = [vp, C.c_int, ip, vp, dp, dp, C.c_int64, vp, vp, C.c_int, vp]
    L.game_solve.argtypes = [vp, C.c_int32, C.POINTER(GameParams), C.POINTER(GameOpts),
                             C.POINTER(GameResult), vp]
    L.cheb_filter.argtypes = [vp, C.c_int, ip, vp, C.c_double, C.c_int32, vp]
    L.cheb_filter.restype = C.c_int
    L.cheb_smooth.argtypes = [vp, C.c_int, ip, vp, C.c_double, C.c_int32, vp]
    L.cheb_smooth.restype = C.c_int
    L.cheb_profile.argtypes = [vp, C.c_int]
    L.cheb_profile_count.argtypes = [vp]
    L.cheb_profile_get.argtypes = [vp, C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double)]
    L.game_paths.argtypes = [vp, C.POINTER(GameParams), C.POINTER(GameOpts), vp, C.c_int64, vp, C.c_int64, vp,
                             vp, vp]
    L.cheb_set_tuning.argtypes = [vp, C.c_int]
    L.cheb_set_wait_limit.argtypes = [vp, C.c_int64]
    L.cheb_tuning_report.argtypes = [vp, C.c_char_p, C.c_int64]
    L.surrogate_create.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(vp)]
    L.surrogate_destroy.argtypes = [vp]
    L.surrogate_params.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_int64)]
    L.surrogate_loss_grad.argtypes = [vp, vp, vp, vp, C.c_int32, C.POINTER(C.c_float), vp, vp]
    L.surrogate_train.argtypes = [vp, vp, vp, C.c_int64, vp, C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                  C.c_float, C.c_uint64, C.POINTER(C.c_float), vp]
    L.surrogate_predict.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, vp, C.c_int64, vp]
    L.surrogate_adam_step.argtypes = [vp, vp, vp, C.c_float, vp]
    for f in ("surrogate_create", "surrogate_destroy", "surrogate_params", "surrogate_loss_grad",
              "surrogate_train", "surrogate_predict", "surrogate_adam_step", "cheb_profile", "cheb_profile_count", "cheb_profile_get", "cheb_set_tuning", "cheb_set_wait_limit",
              "cheb_tuning_report", "cheb_create", "cheb_destroy", "cheb_device_status", "cheb_fit", "cheb_eval_grid", "cheb_eval_grid_host",
              "cheb_eval_points", "game_solve", "game_paths"):
        getattr(L, f).restype = C.c_int
    if hasattr(L, "cheb_check_selftest"):      # the checked build only
        L.cheb_check_selftest.argtypes = [vp]
        L.cheb_check_selftest.restype = C.c_int
    _lib = L
    return L


def check(status: int) -> None:
    if status != CHEB_OK:
        raise ChebError(status, load().cheb_last_error().decode())
