"""ctypes loader for libcrsolve.so (the C ABI of include/crsolve.h).

There is no fallback: if the library is missing or cannot be loaded, every
entry point raises.  Argument marshalling only; all arithmetic runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

CRSOLVE_OK = 0
CRSOLVE_NOT_PD = 1
CRSOLVE_EINVAL = -1
CRSOLVE_ENOMEM = -2
CRSOLVE_ECUDA = -3
CRSOLVE_ETIMEOUT = -4
CRSOLVE_ENOTFACTORED = -5
CRSOLVE_EUNSUPPORTED = -6
CRSOLVE_FP64 = 0
CRSOLVE_MIXED = 1
CRSOLVE_PLAN_HOST_STAGING = 1
CRSOLVE_PLAN_ALG1 = 2
CRSOLVE_PLAN_FP64_RESIDUAL = 4
CRSOLVE_RESIDUAL_FP64 = 0
CRSOLVE_RESIDUAL_SPLIT = 1
CRSOLVE_RESIDUAL_SPLIT_IMAGE = 2
CRSOLVE_PROBE_FP64_FMA = 0
CRSOLVE_PROBE_FP32_FMA = 1
CRSOLVE_MAX_M = 64
CRSOLVE_MAX_K = 4096

# every symbol include/crsolve.h declares: name -> (restype, argtypes)
_P = ctypes.c_void_p
_I64, _I32, _U32, _SZ = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t


class CrsolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("level", ctypes.c_int32),
                ("block", ctypes.c_int64), ("orig_block", ctypes.c_int64)]


class CrsolveKernelTime(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32),
                ("units", ctypes.c_int64), ("ms", ctypes.c_float)]


KERNEL_KINDS = {0: "factor_odd", 1: "factor_fix", 2: "solve_down_odd", 3: "solve_down_fix",
                4: "solve_up", 5: "adjoint_outer", 6: "nan_fill", 7: "residual", 8: "convert", 9: "update",
                10: "alg1_border", 11: "alg1_merge"}

SIGNATURES = {
    "crsolve_plan_create": (ctypes.c_int, [_I64, _I32, _I32, _I32, _U32, ctypes.POINTER(_P)]),
    "crsolve_workspace_bytes": (ctypes.c_int, [_P, ctypes.POINTER(_SZ)]),
    "crsolve_set_workspace": (ctypes.c_int, [_P, _P, _SZ]),
    "crsolve_plan_keep_levels": (ctypes.c_int, [_P, ctypes.c_int32]),
    "crsolve_scratch_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "crsolve_set_scratch": (ctypes.c_int, [_P, _P, _SZ]),
    "crsolve_factor": (ctypes.c_int, [_P, _P, _P, _P]),
    "crsolve_solve": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "crsolve_backward": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _P, _P]),
    "crsolve_solve_host": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _P]),
    "crsolve_info_get": (ctypes.c_int, [_P, ctypes.POINTER(CrsolveInfo), _P]),
    "crsolve_destroy": (ctypes.c_int, [_P]),
    "crsolve_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "crsolve_plan_levels": (ctypes.c_int, [_P, ctypes.POINTER(_I32), _P]),
    "crsolve_debug_level_system": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "crsolve_timing_enable": (ctypes.c_int, [_P, _I32]),
    "crsolve_timing_read": (ctypes.c_int, [_P, ctypes.POINTER(CrsolveKernelTime), _I32, ctypes.POINTER(_I32)]),
    "crsolve_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "crsolve_mixed_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I32)]),
    "crsolve_mixed_precondition": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "crsolve_tile_set": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, _I32]),
    "crsolve_batch_create": (ctypes.c_int, [_I32, _P, _P, _P, ctypes.POINTER(_P)]),
    "crsolve_batch_tile_set": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32]),
    "crsolve_batch_workspace_bytes": (ctypes.c_int, [_P, _SZ, ctypes.POINTER(_SZ), ctypes.POINTER(_I32)]),
    "crsolve_batch_set_workspace": (ctypes.c_int, [_P, _P, _SZ]),
    "crsolve_batch_offsets": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "crsolve_batch_solve": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "crsolve_batch_graph_launch": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "crsolve_batch_info": (ctypes.c_int, [_P, _P, _P]),
    "crsolve_batch_destroy": (ctypes.c_int, [_P]),
    "crsolve_solve_noalloc": (ctypes.c_int, [_I64, _I32, _I32, _P, _P, _P, _P, ctypes.POINTER(CrsolveInfo), _P]),
    "crsolve_tile_get": (ctypes.c_int, [_I32] + [ctypes.POINTER(_I32)] * 5),
    "crsolve_tile_set_mixed": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, _I32]),
    "crsolve_tile_get_mixed": (ctypes.c_int, [_I32] + [ctypes.POINTER(_I32)] * 5),
    "crsolve_peak_probe": (ctypes.c_int, [_I32] + [ctypes.POINTER(ctypes.c_double)] * 3 + [_P]),
    "crsolve_check_bounded_wait": (ctypes.c_int, [_I32, _P, _P]),
    "crsolve_debug_bounds": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), _P]),
    "crsolve_batch_debug_bounds": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), _P]),
    "crsolve_residual_workspace_bytes": (ctypes.c_int, [_I64, _I32, _I32, _I32, ctypes.POINTER(_SZ)]),
    "crsolve_residual": (ctypes.c_int, [_I64, _I32, _I32, _P, _P, _P, _P, _P, _I32, _P, _SZ, _P]),
}


class CrsolveError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


def lib_path() -> str:
    """The library to load: libcrsolve.so, or the bounds-checked
    libcrsolve_debug.so when CRSOLVE_LIBRARY=debug."""
    return _build.DEBUG_LIB if os.environ.get("CRSOLVE_LIBRARY") == "debug" else _build.LIB


def load(build_if_missing: bool = True):
    """Load libcrsolve.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        debug = path == _build.DEBUG_LIB
        if build_if_missing and _build.is_stale(debug):
            _build.build(debug=debug)
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run paper_1807_00370_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().crsolve_strerror(int(code)).decode()
    except Exception:  # noqa: BLE001 - error text only
        return "unknown"


def check(code: int, where: str) -> int:
    if code < 0:
        raise CrsolveError(code, where)
    return code
