"""ctypes binding of libfmm.so (include/fmm.h): argument marshalling only.

Loading fails loudly (ImportError / OSError) when the library has not been
built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfmm.so")

FMM_OK = 0
STATUS_NAMES = {
    0: "FMM_OK", 1: "FMM_ERR_ARG", 2: "FMM_ERR_NOT_MATMUL", 3: "FMM_ERR_SHAPE", 4: "FMM_ERR_ALIGN",
    5: "FMM_ERR_DTYPE", 6: "FMM_ERR_WORKSPACE", 7: "FMM_ERR_CUDA", 8: "FMM_ERR_DEVICE_TIMEOUT",
    9: "FMM_ERR_NONFINITE", 10: "FMM_ERR_UNSUPPORTED",
}
ORDER_ROW, ORDER_COL = 0, 1
DT_F32, DT_BF16, DT_F16 = 0, 1, 2
LEAF_BF16, LEAF_F16, LEAF_BF16X3, LEAF_E4M3B128 = 0, 1, 2, 3
SCHEDULE_AUTO, SCHEDULE_LOAD_STAGE, SCHEDULE_PASS, SCHEDULE_PASS_EPILOGUE, SCHEDULE_PASS_PRODUCTS = 0, 1, 2, 3, 4
SCHEDULE_PASS_ACCUMULATE = 5

# Every symbol include/fmm.h declares.
EXPORTS = [
    "fmm_plan", "fmm_plan_destroy", "fmm_plan_info", "fmm_plan_bound", "fmm_scale_outside",
    "fmm_scale_inside", "fmm_scale", "fmm_workspace_size", "fmm_multiply", "fmm_multiply_backward",
    "fmm_sync_status", "fmm_status_string", "fmm_version", "fmm_last_error", "fmm_multiply_noalloc",
    "fmm_plan_set_schedule", "fmm_kernel_timing", "fmm_kernel_timing_read",
    "fmm_batch_workspace_size", "fmm_batch_create", "fmm_batch_run", "fmm_batch_destroy",
    "fmm_plan_set_between_scaling", "fmm_plan_tree", "fmm_scale_adaptive",
    "fmm_host_create", "fmm_host_submit", "fmm_host_wait", "fmm_host_destroy",
    "fmm_rule_rotate", "fmm_rule_compose", "fmm_rule_transform", "fmm_rule_permute", "fmm_plan_variants",
    "fmm_block_max", "fmm_batch_partition", "fmm_plan_flatten", "fmm_plan_gradient",
]
SELECT_RANDOM, SELECT_ROUND_ROBIN, SELECT_MATRIX = 0, 1, 2
TABLE_LEAVES, TABLE_LISTS, TABLE_GATHER = 0, 1, 2
GRAD_A, GRAD_B = 0, 1

# Bytes of the library's static scratch array (FMM_NOALLOC_SCRATCH_BYTES).
NOALLOC_SCRATCH_BYTES = 32 << 20


class FmmRule(C.Structure):
    _fields_ = [("m0", C.c_int), ("k0", C.c_int), ("n0", C.c_int), ("r", C.c_int),
                ("U", C.POINTER(C.c_double)), ("V", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
                ("order_a", C.c_int), ("order_b", C.c_int), ("order_c", C.c_int)]


class FmmProblem(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("A", C.c_void_p), ("lda", C.c_int64), ("B", C.c_void_p),
                ("ldb", C.c_int64), ("C", C.c_void_p), ("ldc", C.c_int64), ("M", C.c_int64), ("K", C.c_int64),
                ("N", C.c_int64)]


class FmmError(RuntimeError):
    def __init__(self, code: int, what: str):
        detail = lib().fmm_last_error().decode() if code == 7 else ""
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} ({lib().fmm_status_string(code).decode()})"
                         + (f" [{detail}]" if detail else ""))
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfmm.so is not built ({LIB_PATH}); run paper_1507_00687_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    i64, i32p, vp, st = C.c_int64, C.POINTER(C.c_int32), C.c_void_p, C.c_int
    L.fmm_plan.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(FmmRule), C.c_int]
    L.fmm_plan_destroy.argtypes = [vp]
    L.fmm_host_create.argtypes = [C.POINTER(vp), vp, i64, i64, i64, C.c_int, C.c_char_p, C.c_int]
    L.fmm_host_submit.argtypes = [vp, vp, i64, vp, i64, vp, i64]
    L.fmm_host_wait.argtypes = [vp]
    L.fmm_host_destroy.argtypes = [vp]
    L.fmm_plan_tree.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(FmmRule), C.c_int, i64,
                                C.POINTER(C.c_int32), C.c_int]
    rp, dp = C.POINTER(FmmRule), C.POINTER(C.c_double)
    L.fmm_rule_rotate.argtypes = [rp, dp, dp, dp, rp]
    L.fmm_rule_compose.argtypes = [rp, rp, dp, dp, dp, rp]
    L.fmm_rule_transform.argtypes = [rp, dp, dp, dp, dp, dp, dp, rp]
    L.fmm_rule_permute.argtypes = [rp, i32p, i32p, i32p, dp, dp, dp, rp]
    L.fmm_plan_variants.argtypes = [C.POINTER(vp), rp, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_float),
                                    C.POINTER(C.c_float), i32p, C.c_int]
    L.fmm_block_max.argtypes = [vp, C.c_int, i64, i64, i64, C.c_int, C.c_int, vp, vp]
    i64p = C.POINTER(i64)
    L.fmm_batch_partition.argtypes = [i64p, i64p, i64p, C.c_int, C.c_int, i32p]
    L.fmm_plan_set_schedule.argtypes = [vp, C.c_int]
    L.fmm_plan_set_between_scaling.argtypes = [vp, C.c_int]
    L.fmm_kernel_timing.argtypes = [C.c_int]
    L.fmm_batch_workspace_size.argtypes = [C.POINTER(FmmProblem), C.c_int, C.c_int, C.c_char_p,
                                           C.POINTER(C.c_size_t)]
    L.fmm_batch_create.argtypes = [C.POINTER(vp), C.POINTER(FmmProblem), C.c_int, C.c_int, C.c_char_p, vp,
                                   C.c_size_t]
    L.fmm_batch_run.argtypes = [vp, vp]
    L.fmm_batch_destroy.argtypes = [vp]
    L.fmm_kernel_timing_read.argtypes = [C.c_char_p, C.POINTER(C.c_double), C.POINTER(i64)]
    L.fmm_plan_info.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(i64),
                                C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.fmm_plan_bound.argtypes = [vp, i64, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
    L.fmm_plan_flatten.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.fmm_plan_gradient.argtypes = [vp, C.c_int, C.POINTER(vp)]
    L.fmm_scale_outside.argtypes = [vp, vp, C.c_int, i64, i64, i64, i64, i64, vp, vp, vp, vp]
    L.fmm_scale_inside.argtypes = [vp, vp, C.c_int, i64, i64, i64, i64, i64, vp, vp, vp, vp]
    L.fmm_scale_adaptive.argtypes = [vp, vp, C.c_int, i64, i64, i64, i64, i64, C.c_double, C.c_int, C.c_int,
                                     vp, vp, vp, vp, vp, C.c_size_t, vp]
    L.fmm_scale.argtypes = [C.c_char_p, vp, vp, C.c_int, i64, i64, i64, i64, i64, vp, vp, vp, vp]
    L.fmm_workspace_size.argtypes = [vp, i64, i64, i64, C.POINTER(C.c_size_t)]
    L.fmm_multiply.argtypes = [vp, vp, i64, vp, i64, vp, i64, i64, i64, i64, C.c_int, vp, vp, vp, vp,
                               C.c_size_t, vp]
    L.fmm_multiply_noalloc.argtypes = [vp, vp, i64, vp, i64, vp, i64, i64, i64, i64, C.c_int, vp, vp, vp, vp]
    L.fmm_multiply_backward.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, i64, i64, i64,
                                        C.c_int, vp, C.c_size_t, vp]
    L.fmm_sync_status.argtypes = [vp]
    L.fmm_status_string.argtypes = [C.c_int]
    L.fmm_status_string.restype = C.c_char_p
    L.fmm_version.argtypes = []
    L.fmm_version.restype = C.c_char_p
    L.fmm_last_error.argtypes = []
    L.fmm_last_error.restype = C.c_char_p
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("fmm_status_string", "fmm_version", "fmm_last_error"):
            f.restype = st
    _lib = L
    return L


def check(code: int, what: str) -> None:
    if code != FMM_OK:
        raise FmmError(code, what)
