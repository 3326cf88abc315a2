"""ctypes binding of the C ABI in include/fdtd.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

FDTD_OK = 0
ERRORS = {
    -1: "FDTD_ERR_INVALID_ARG",
    -2: "FDTD_ERR_OOM",
    -3: "FDTD_ERR_CUDA",
    -4: "FDTD_ERR_TIMEOUT",
    -5: "FDTD_ERR_UNSTABLE",
    -6: "FDTD_ERR_UNSUPPORTED",
    -7: "FDTD_ERR_STATE",
    -8: "FDTD_ERR_BOUNDS",
}

SCHEMES = {"fadi": 0, "flod": 1, "fss": 2, "flod2": 3}
PRECISIONS = {"f64": 0, "f32": 1}
COMPS = {"ex": 0, "ey": 1, "ez": 2, "hx": 3, "hy": 4, "hz": 5}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = (
    "fdtd_create", "fdtd_destroy", "fdtd_get_dt", "fdtd_set_material", "fdtd_set_media", "fdtd_set_order", "fdtd_set_field",
    "fdtd_get_field", "fdtd_get_state", "fdtd_set_state", "fdtd_set_source", "fdtd_add_probe",
    "fdtd_step", "fdtd_get_probe", "fdtd_energy", "fdtd_steps_done", "fdtd_synchronize",
    "fdtd_strerror", "fdtd_set_timing", "fdtd_get_stats", "fdtd_reset_stats",
    "fdtd_energy_noalloc", "fdtd_batch_create", "fdtd_batch_step", "fdtd_batch_destroy",
    "fdtd_batch_launches", "fdtd_batch_get_config", "fdtd_batch_set_config", "fdtd_batch_set_mode",
    "fdtd_batch_get_mode", "fdtd_adj_create", "fdtd_adj_forward", "fdtd_adj_backward", "fdtd_adj_memory",
    "fdtd_adj_destroy", "fdtd_selftest_bounded_wait", "fdtd_debug_fail_alloc", "fdtd_probe_fp64_fma",
)


class FdtdDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
        ("scheme", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("tune", ctypes.c_int32 * 2),
    ]


class FdtdStats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64),
        ("timed_launches", ctypes.c_int64 * 3),
        ("timed_ms", ctypes.c_double * 3),
        ("bytes_per_launch", ctypes.c_double * 3),
    ]


class FdtdError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({strerror(code)})")


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (FDTD_LIBRARY in the environment names another
    build of it, e.g. the bounds-checked one); raises if it has not been
    built."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("FDTD_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing "
                          "(run paper_2011_14043_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i32 = ctypes.c_int
    i64 = ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "fdtd_create": (i32, [ctypes.POINTER(FdtdDesc), vp, ctypes.POINTER(vp)]),
        "fdtd_destroy": (i32, [vp]),
        "fdtd_get_dt": (i32, [vp, dp]),
        "fdtd_set_material": (i32, [vp, vp, vp]),
        "fdtd_set_media": (i32, [vp, vp, vp, vp]),
        "fdtd_set_order": (i32, [vp, i32]),
        "fdtd_set_field": (i32, [vp, i32, vp, i32]),
        "fdtd_get_field": (i32, [vp, i32, vp, i32]),
        "fdtd_get_state": (i32, [vp, i32, vp, i32]),
        "fdtd_set_state": (i32, [vp, i32, vp, i32]),
        "fdtd_set_source": (i32, [vp, i32, i32, i32, i32, vp, i64]),
        "fdtd_add_probe": (i32, [vp, i32, i32, i32, i32, ctypes.POINTER(i32)]),
        "fdtd_step": (i32, [vp, i64]),
        "fdtd_get_probe": (i32, [vp, i32, vp, i64]),
        "fdtd_energy": (i32, [vp, vp]),
        "fdtd_steps_done": (i32, [vp, ctypes.POINTER(i64)]),
        "fdtd_synchronize": (i32, [vp]),
        "fdtd_strerror": (ctypes.c_char_p, [i32]),
        "fdtd_set_timing": (i32, [vp, i32]),
        "fdtd_get_stats": (i32, [vp, ctypes.POINTER(FdtdStats)]),
        "fdtd_reset_stats": (i32, [vp]),
        "fdtd_batch_create": (i32, [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)]),
        "fdtd_batch_step": (i32, [vp, i64]),
        "fdtd_batch_destroy": (i32, [vp]),
        "fdtd_batch_launches": (i32, [vp, ctypes.POINTER(i64)]),
        "fdtd_batch_get_config": (i32, [vp, ctypes.POINTER(ctypes.c_int32), dp]),
        "fdtd_batch_set_config": (i32, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "fdtd_batch_set_mode": (i32, [vp, i32]),
        "fdtd_batch_get_mode": (i32, [vp, ctypes.POINTER(ctypes.c_int32), dp]),
        "fdtd_adj_create": (i32, [vp, ctypes.POINTER(ctypes.c_int32), i64, ctypes.c_int32, ctypes.POINTER(vp)]),
        "fdtd_adj_forward": (i32, [vp, dp]),
        "fdtd_adj_backward": (i32, [vp, ctypes.c_double, vp, i32]),
        "fdtd_adj_memory": (i32, [vp, ctypes.POINTER(i64)]),
        "fdtd_adj_destroy": (i32, [vp]),
        "fdtd_selftest_bounded_wait": (i32, [i64, i32, vp]),
        "fdtd_debug_fail_alloc": (i32, [i64]),
        "fdtd_probe_fp64_fma": (i32, [i64, dp, vp]),
        "fdtd_energy_noalloc": (i32, [i32, i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, i32, ctypes.POINTER(vp),
                                      ctypes.POINTER(ctypes.c_double), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().fdtd_strerror(code).decode()
    except ImportError:
        return ERRORS.get(code, str(code))


def check(code: int, what: str) -> None:
    if code != FDTD_OK:
        raise FdtdError(code, what)
