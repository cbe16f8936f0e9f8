"""ctypes declarations of the C ABI in include/edm.h (no computation here)."""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

EDM_OK = 0
EDM_ERR_INVALID = 1
EDM_ERR_CUDA = 2
EDM_ERR_WORKSPACE = 3
EDM_ERR_TIMEOUT = 4
EDM_ERR_UNSUPPORTED = 5
EDM_MAX_E = 20
EDM_MAX_T = 65535
EDM_PRECISION_FP32 = 0
EDM_PRECISION_FP16_TARGETS = 1
EDM_FLAG_LOOKUP_SCALAR = 1
EDM_FLAG_VALIDATE = 2
EDM_FLAG_KNN_WARP = 4


class edm_params(ctypes.Structure):
    _fields_ = [
        ("E_max", ctypes.c_int32),
        ("tau", ctypes.c_int32),
        ("Tp", ctypes.c_int32),
        ("exclusion_radius", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
    ]


class edm_dataset(ctypes.Structure):
    _fields_ = [
        ("Y", ctypes.c_void_p),
        ("N", ctypes.c_int64),
        ("T", ctypes.c_int64),
        ("ldY", ctypes.c_int64),
        ("optE", ctypes.c_void_p),
        ("rho", ctypes.c_void_p),
        ("ld_rho", ctypes.c_int64),
    ]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_pp = ctypes.POINTER(edm_params)

# name -> (restype, argtypes); mirrors include/edm.h
SIGNATURES = {
    "edm_optimal_E": (ctypes.c_int, [_vp, _i64, _i64, _i64, _pp, _vp, _vp, _vp]),
    "edm_knn_table": (ctypes.c_int, [_vp, _i64, _i64, _i64, _i32, _pp, _vp, _vp, _i64, _vp]),
    "edm_ccm_rho": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _i64, _i64, _pp, _vp, _i64, _vp, ctypes.c_size_t, _vp]),
    "edm_ccm_workspace_bytes": (ctypes.c_size_t, [_i64, _i64, _pp]),
    "edm_ccm_rho_lags": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _i32, _i32, _pp, _vp, _i64, _vp, ctypes.c_size_t,
                                        _vp]),
    "edm_ccm_rho_lags_workspace_bytes": (ctypes.c_size_t, [_i64, _i64, _i32, _i32, _pp]),
    "edm_ccm_rho_subsets": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _i32, _i64, _pp, _vp, _i64, _vp,
                                           ctypes.c_size_t, _vp]),
    "edm_ccm_host": (ctypes.c_int, [_vp, _i64, _i64, _pp, _vp, _vp, _i64, _i64, _vp, ctypes.c_size_t, _vp]),
    "edm_ccm_host_workspace_bytes": (ctypes.c_size_t, [_i64, _i64, _i64, _pp]),
    "edm_ccm_rho_noalloc": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _i64, _i64, _pp, _vp, _i64, _vp]),
    "edm_ccm_rho_backward": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _i64, _pp, _vp, _vp, ctypes.c_size_t,
                                            _vp]),
    "edm_ccm_backward_workspace_bytes": (ctypes.c_size_t, [_i64, _i64, _pp]),
    "edm_ccm_rho_batched": (ctypes.c_int, [ctypes.POINTER(edm_dataset), _i32, _pp, _vp, ctypes.c_size_t, _vp]),
    "edm_ccm_rho_batched_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(edm_dataset), _i32, _pp]),
    "edm_ccm_rho_batched_reset": (ctypes.c_int, []),
    "edm_last_bad_series": (ctypes.c_int64, []),
    "edm_knn_counters": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    "edm_wait_timeouts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    "edm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "edm_last_cuda_error": (ctypes.c_int, []),
    "edm_version": (ctypes.c_int, []),
    "edm_launch_count": (ctypes.c_int64, [ctypes.c_int]),
    "edm_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "edm_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double)]),
}

EDM_KERNEL_SIMPLEX = 0
EDM_KERNEL_KNN = 1
EDM_KERNEL_PREP = 2
EDM_KERNEL_LOOKUP = 3
EDM_KERNEL_PLAN = 4
EDM_KERNEL_BATCH = 5
EDM_KERNEL_COUNT = 6
KERNEL_NAMES = {0: "simplex_kernel", 1: "knn_tables_kernel", 2: "prep_targets_kernel", 3: "lookup_kernel",
                4: "batch_plan_kernel", 5: "batched_graph"}

_lock = threading.Lock()
_lib = None


class EdmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libedm.so (building it first if needed).  Raises if unavailable:
    there is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
            if not build_if_missing:
                raise ImportError(f"{path} is missing; run paper_2011_11082_gb300.build.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str):
    if status != EDM_OK:
        lib = load()
        msg = lib.edm_status_string(status).decode()
        bad = int(lib.edm_last_bad_series())
        if status == EDM_ERR_INVALID and bad >= 0:
            msg += f" (series {bad} holds a non-finite value)"
        raise EdmError(status, where, msg)
