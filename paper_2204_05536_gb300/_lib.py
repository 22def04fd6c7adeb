"""ctypes declarations of the C ABI in ``include/hodlr2d.h`` (argument
marshalling only).  Loading fails loudly if the compiled library is missing:
there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MAX_LEVELS = 15
NPHASE = 10
PHASES = ["gather", "near", "proj", "tsum", "exp", "combine", "pair_big", "finest", "pair_small",
          "unused"]

OK = 0
ERR_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_NOCONV = -4
ERR_TIMEOUT = -5
ERR_DEPTH = -6
ERR_STATE = -7

KINDS = {"imq": 0, "mq": 1, "log": 2, "inv_r": 3, "phi1": 4, "phi2": 5}
MODES = {"f64": 0, "df32": 1, "f32": 2, "bf16": 3}


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("diag_mode", C.c_int),
                ("diag_value", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("root", C.c_double * 3), ("levels", C.c_int), ("compress", C.c_int),
                ("max_rank", C.c_int), ("mode", C.c_int), ("rank_model", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("kappa", C.c_int), ("root", C.c_double * 3),
                ("npairs", C.c_int64), ("pairs_per_level", C.c_int64 * MAX_LEVELS),
                ("values_per_level", C.c_int64 * MAX_LEVELS),
                ("max_rank_per_level", C.c_int * MAX_LEVELS), ("max_rank", C.c_int),
                ("far_values", C.c_int64), ("near_entries", C.c_int64),
                ("unconverged", C.c_int64), ("compression_ratio", C.c_double),
                ("build_ms", C.c_double * 4), ("bytes_per_matvec", C.c_int64 * 4),
                ("aca_fallbacks", C.c_int64), ("aca_workspace_values", C.c_int64)]


_P = C.c_void_p
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)

SIGNATURES = {
    "hodlr2d_default_opts": (None, [C.POINTER(Opts)]),
    "hodlr2d_build": (C.c_int, [_P, C.c_int64, Kernel, C.c_int, C.c_double, C.POINTER(_P)]),
    "hodlr2d_build_ex": (C.c_int, [_P, C.c_int64, Kernel, C.c_int, C.c_double,
                                   C.POINTER(Opts), C.POINTER(_P)]),
    "hodlr2d_matvec": (C.c_int, [_P, _P, _P, C.c_int]),
    "hodlr2d_matvec_ex": (C.c_int, [_P, _P, _P, C.c_int, C.c_int]),
    "hodlr2d_prepare": (C.c_int, [_P, C.c_int]),
    "hodlr2d_release": (C.c_int, [_P, C.c_int]),
    "hodlr2d_check": (C.c_int, [_P]),
    "hodlr2d_gmres": (C.c_int, [_P, _P, _P, C.c_double]),
    "hodlr2d_gmres_ex": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(C.c_int), _dp]),
    "hodlr2d_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "hodlr2d_set_stream": (C.c_int, [_P, _P]),
    "hodlr2d_profile": (C.c_int, [_P, C.c_int]),
    "hodlr2d_get_profile": (C.c_int, [_P, _P, _P, _P]),
    "hodlr2d_get_profile_flops": (C.c_int, [_P, _P]),
    "hodlr2d_get_perm": (C.c_int, [_P, _P]),
    "hodlr2d_get_pairs": (C.c_int, [_P, _i64p, _P]),
    "hodlr2d_import_factors": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "hodlr2d_export_factors": (C.c_int, [_P, _i64p, _i64p, _P, _P, _P]),
    "hodlr2d_matvec_noalloc": (C.c_int, [_P, _P, _P, C.c_int]),
    "hodlr2d_rank_model_create": (C.c_int, [C.c_int, _P, C.POINTER(_P)]),
    "hodlr2d_rank_model_params": (C.c_int, [_P, _P, _i64p]),
    "hodlr2d_rank_model_loss_grad": (C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(C.c_float), _P]),
    "hodlr2d_rank_model_train": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, C.c_int, C.c_float,
                                           C.POINTER(C.c_float)]),
    "hodlr2d_rank_model_predict": (C.c_int, [_P, _P, C.c_int64, _P]),
    "hodlr2d_rank_model_free": (None, [_P]),
    "hodlr2d_pair_features": (C.c_int, [_P, _i64p, _P, _P]),
    "hodlr2d_batch_create": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "hodlr2d_batch_set_stream": (C.c_int, [_P, _P]),
    "hodlr2d_batch_matvec": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "hodlr2d_batch_set_form": (C.c_int, [_P, C.c_int]),
    "hodlr2d_batch_set_wait_limit": (C.c_int, [_P, C.c_uint32]),
    "hodlr2d_batch_check": (C.c_int, [_P]),
    "hodlr2d_batch_last_form": (C.c_int, [_P]),
    "hodlr2d_batch_persistent_recorded": (C.c_int, [_P]),
    "hodlr2d_batch_set_shapes": (C.c_int, [_P, C.c_int, C.c_int]),
    "hodlr2d_batch_get_shapes": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "hodlr2d_batch_autotune": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int,
                                         C.POINTER(C.c_double)]),
    "hodlr2d_batch_phase_ms": (C.c_int, [_P, _P]),
    "hodlr2d_batch_tune_table": (C.c_int, [_P, C.POINTER(C.c_int), _P, _P, _P, _P, _P]),
    "hodlr2d_batch_set_placement": (C.c_int, [_P, C.c_int]),
    "hodlr2d_batch_set_blocks_per_sm": (C.c_int, [_P, C.c_int]),
    "hodlr2d_batch_free": (None, [_P]),
    "hodlr2d_free": (None, [_P]),
    "hodlr2d_strerror": (C.c_char_p, [C.c_int]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """The loaded library.  Builds it first if it is missing or stale and
    nvcc is available; raises if it still cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libhodlr2d.so is not built (run __graft_entry__.build())")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class HodlrError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().hodlr2d_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (where, msg, code))
        self.code = code


def check(code: int, where: str) -> None:
    if code != OK:
        raise HodlrError(code, where)
