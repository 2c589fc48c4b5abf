"""ctypes binding to ``libtde.so`` (argument marshalling only; every step of the
solver runs in the library's CUDA kernels).  Importing this module never falls
back to a CPU path: if the shared library is missing or fails to load, every
entry point raises."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtde.so")

TDE_OK = 0
TDE_EINVAL = -1
TDE_ECUDA = -2
TDE_EWORKSPACE = -3
TDE_ENOCONV = 1
TDE_ENONFINITE = 2
TDE_ETIMEOUT = 3
STATUS_NAMES = {0: "TDE_OK", -1: "TDE_EINVAL", -2: "TDE_ECUDA", -3: "TDE_EWORKSPACE",
                1: "TDE_ENOCONV", 2: "TDE_ENONFINITE", 3: "TDE_ETIMEOUT"}

# every symbol include/tde.h declares
EXPORTS = ("tde_eigvals_workspace", "tde_eigvals", "tde_eigvals_batched_workspace",
           "tde_eigvals_batched", "tde_get_info", "tde_measure_fp64_peak",
           "tde_last_launch_count", "tde_profile_enable", "tde_profile_select", "tde_profile_collect", "tde_read_work",
           "tde_eigvals_noalloc", "tde_plan_query", "tde_check_reciprocal",
           "tde_profile_collect_steps", "tde_set_tuning", "tde_get_tuning",
           "tde_eigvals_backward_workspace", "tde_eigvals_backward", "tde_eigvecs_rows_workspace",
           "tde_eigvecs_rows", "tde_dense_eigvals_workspace", "tde_dense_eigvals",
           "tde_set_multipole", "tde_check_rsqrt", "tde_noalloc_get_info",
           "tde_eigvals_backward_workspace_slots")

MAX_SEL_ROWS = 1024  # TDE_MAX_SEL_ROWS

KERNEL_NAMES = ("plan", "scale", "leaves", "form", "deflate", "secular", "lowner", "rows", "place",
                "sel", "sel_rows")
WORK_NAMES = ("secular_pairs", "secular_sweeps", "lowner_pairs", "rows_pairs", "roots", "deflated",
              "rotations", "leaf_rotations", "sorts", "sorted_entries", "secular32_pairs",
              "secular32_sweeps", "sel_row_pairs", "sel_sweep_pairs", "secular_far_blocks",
              "rows_far_series", "lowner_far_blocks", "secular_series_ops", "lowner_series_ops",
              "rows_series_ops")


class TdeError(RuntimeError):
    """A tde_* entry point returned a non-zero status."""

    def __init__(self, func: str, code: int):
        super().__init__(f"{func} returned {STATUS_NAMES.get(code, code)}")
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """Load ``libtde.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2605_26599_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    i64, i32, sz, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_void_p
    szp = ctypes.POINTER(ctypes.c_size_t)
    lib.tde_eigvals_workspace.argtypes = [i64, i32, szp]
    lib.tde_eigvals.argtypes = [i64, vp, vp, vp, i32, vp, sz, vp]
    lib.tde_eigvals_batched_workspace.argtypes = [i64, vp, i32, szp]
    lib.tde_eigvals_batched.argtypes = [i64, vp, vp, vp, vp, vp, i32, vp, sz, vp]
    lib.tde_get_info.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
    lib.tde_eigvecs_rows_workspace.argtypes = [i64, i64, i32, szp]
    lib.tde_dense_eigvals_workspace.argtypes = [i64, i32, szp]
    lib.tde_dense_eigvals.argtypes = [i64, vp, i64, vp, i32, vp, sz, vp]
    lib.tde_eigvecs_rows.argtypes = [i64, vp, vp, i64, vp, vp, vp, i32, vp, sz, vp]
    lib.tde_measure_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.tde_last_launch_count.restype = ctypes.c_int64
    lib.tde_last_launch_count.argtypes = []
    lib.tde_profile_enable.argtypes = [ctypes.c_int]
    lib.tde_profile_select.argtypes = [ctypes.c_uint32]
    lib.tde_profile_collect.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]
    lib.tde_read_work.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
    lib.tde_eigvals_noalloc.argtypes = [i64, vp, vp, vp, i32, vp]
    lib.tde_noalloc_get_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.tde_plan_query.argtypes = [i64, vp, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.tde_check_reciprocal.argtypes = [i64, vp, vp, vp]
    lib.tde_check_rsqrt.argtypes = [i64, vp, vp, vp]
    lib.tde_set_tuning.argtypes = [i32, i32]
    lib.tde_eigvals_backward_workspace.argtypes = [i64, vp, i32, szp]
    lib.tde_eigvals_backward_workspace_slots.argtypes = [i64, vp, i32, i32, szp]
    lib.tde_eigvals_backward.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, sz, vp]
    lib.tde_get_tuning.argtypes = [ctypes.POINTER(ctypes.c_int32)]
    lib.tde_set_multipole.argtypes = [i32, ctypes.POINTER(ctypes.c_int32)]
    lib.tde_profile_collect_steps.argtypes = [ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int64)]
    for name in EXPORTS:
        if name != "tde_last_launch_count":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(func: str, code: int) -> None:
    if code != TDE_OK:
        raise TdeError(func, code)
