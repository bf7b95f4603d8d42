"""ctypes declarations of the C ABI in include/odmd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB

ODMD_OK = 0
STATUS_NAMES = {0: "ODMD_OK", 1: "ODMD_ERR_ARG", 2: "ODMD_ERR_STATE", 3: "ODMD_ERR_NOMEM",
                4: "ODMD_ERR_CUDA", 5: "ODMD_ERR_NUMERIC", 6: "ODMD_ERR_TIMEOUT"}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}

EXPORTED = [
    "odmd_config_default", "odmd_footprint", "odmd_create", "odmd_update", "odmd_predict",
    "odmd_check", "odmd_sync", "odmd_get_rank", "odmd_get_singular_values", "odmd_get_eigs",
    "odmd_get_basis", "odmd_get_counts", "odmd_destroy", "odmd_last_error",
    "odmd_profile_enable", "odmd_profile_read", "odmd_check_noalloc", "odmd_hybrid_step",
    "odmd_update_batch", "odmd_predict_batch", "odmd_refine", "odmd_checkpoint_size", "odmd_save",
    "odmd_load", "odmd_hybrid_step_residual", "odmd_hybrid_run", "odmd_update_host",
    "odmd_pairs_footprint", "odmd_pairs_create", "odmd_pairs_update", "odmd_pairs_predict",
    "odmd_pairs_get_singular_values", "odmd_pairs_get_count", "odmd_pairs_last_error", "odmd_pairs_destroy",
    "odmd_pairs_hybrid_step_residual", "odmd_tc_selftest", "odmd_set_row_shards", "odmd_get_row_blocks",
    "odmd_get_batch_split",
]
# host callbacks of odmd_hybrid_step_residual: (user, step, u, r, b, stream) and (user, step, u, stream)
RESIDUAL_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
FOM_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)


class RunReport(C.Structure):
    _fields_ = [("steps", C.c_int64), ("fom_calls", C.c_int64), ("accepted", C.c_int64), ("converged", C.c_int32),
                ("pad", C.c_int32), ("converged_at", C.c_int64), ("skipped", C.c_int64)]
KERNEL_CLASSES = ["pass_a", "small", "pass_b", "eig", "coef", "rollout", "check", "first", "refine", "gap"]


class OdmdConfig(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("r_max", C.c_int32),
        ("slack", C.c_int32),
        ("trunc_tol", C.c_double),
        ("check_tol", C.c_double),
        ("prec", C.c_int),
        ("refine_every", C.c_int32),
        ("flags", C.c_uint32),
    ]


class OdmdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str | None = None) -> C.CDLL:
    """Load libodmd.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with paper_2311_18715_gb300.build()")
    lib = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    cfgp = C.POINTER(OdmdConfig)
    sig = {
        "odmd_config_default": [cfgp, i64, i32],
        "odmd_footprint": [cfgp, C.POINTER(C.c_size_t)],
        "odmd_create": [cfgp, vp, C.c_size_t, vp, C.POINTER(vp)],
        "odmd_update": [vp, vp],
        "odmd_predict": [vp, C.POINTER(dbl), i32, vp, i64],
        "odmd_check": [vp, dbl, vp, dbl, C.POINTER(dbl), C.POINTER(i32)],
        "odmd_check_noalloc": [vp, vp, i64, dbl, vp, C.POINTER(dbl), C.POINTER(i32)],
        "odmd_hybrid_step": [vp, vp, dbl, vp, C.POINTER(i32), C.POINTER(dbl)],
        "odmd_update_batch": [C.POINTER(vp), C.POINTER(vp), i32],
        "odmd_get_batch_split": [C.POINTER(vp), i32, C.POINTER(i32)],
        "odmd_refine": [vp],
        "odmd_checkpoint_size": [vp, C.POINTER(C.c_size_t)],
        "odmd_save": [vp, vp, C.c_size_t],
        "odmd_load": [vp, vp, C.c_size_t],
        "odmd_update_host": [vp, vp, C.c_int64, C.c_int64],
        "odmd_hybrid_step_residual": [vp, RESIDUAL_FN, FOM_FN, vp, C.c_double, vp, vp, vp, C.POINTER(i32),
                                      C.POINTER(C.c_double)],
        "odmd_hybrid_run": [vp, RESIDUAL_FN, FOM_FN, vp, C.c_double, C.c_int64, i32, i32, C.c_double, vp, vp, vp,
                            vp, C.POINTER(RunReport)],
        "odmd_predict_batch": [C.POINTER(vp), C.POINTER(C.POINTER(dbl)), C.POINTER(i32), C.POINTER(vp),
                               C.POINTER(i64), i32],
        "odmd_sync": [vp],
        "odmd_get_rank": [vp, C.POINTER(i32)],
        "odmd_get_singular_values": [vp, C.POINTER(dbl), i32, C.POINTER(i32)],
        "odmd_get_eigs": [vp, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl), i32, C.POINTER(i32)],
        "odmd_get_basis": [vp, vp, i64, C.POINTER(i32)],
        "odmd_get_counts": [vp, C.POINTER(i64), C.POINTER(i64)],
        "odmd_destroy": [vp],
        "odmd_profile_enable": [vp, i32],
        "odmd_profile_read": [vp, C.POINTER(dbl), C.POINTER(i64), i32, C.POINTER(dbl)],
        "odmd_pairs_footprint": [i64, i32, C.POINTER(C.c_size_t)],
        "odmd_pairs_create": [i64, i32, dbl, vp, C.c_size_t, vp, C.POINTER(vp)],
        "odmd_pairs_update": [vp, vp, vp],
        "odmd_pairs_predict": [vp, vp, C.POINTER(dbl), i32, vp, i64],
        "odmd_pairs_get_singular_values": [vp, C.POINTER(dbl), i32, C.POINTER(i32)],
        "odmd_pairs_get_count": [vp, C.POINTER(i64)],
        "odmd_pairs_destroy": [vp],
        "odmd_tc_selftest": [vp, vp, vp, vp, i32],
        "odmd_set_row_shards": [vp, i32],
        "odmd_get_row_blocks": [vp, C.POINTER(i32), C.POINTER(i64), i32],
        "odmd_pairs_hybrid_step_residual": [vp, RESIDUAL_FN, FOM_FN, vp, dbl, i64, vp, vp, vp, vp, C.POINTER(i32),
                                            C.POINTER(dbl)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.odmd_last_error.argtypes = [vp]
    lib.odmd_last_error.restype = C.c_char_p
    lib.odmd_pairs_last_error.argtypes = [vp]
    lib.odmd_pairs_last_error.restype = C.c_char_p
    if path is None:
        _lib = lib
    return lib


def check(lib, status: int, handle=None) -> None:
    if status != ODMD_OK:
        msg = lib.odmd_last_error(handle)
        raise OdmdError(status, msg.decode() if msg else "")


def check_pairs(lib, status: int, handle=None) -> None:
    if status != ODMD_OK:
        msg = lib.odmd_pairs_last_error(handle)
        raise OdmdError(status, msg.decode() if msg else "")
