"""ctypes binding of libctfmm (include/ctfmm.h): argument marshalling only.

Loading fails loudly when the compiled library is missing; there is no CPU
fallback anywhere in the product path.
"""
from __future__ import annotations

import ctypes
import os

from . import build_ext

FMM_OK = 0
STATUS = {
    0: "ok", -1: "invalid argument", -2: "unsupported", -3: "CUDA error", -4: "out of memory",
    -5: "device wait timeout", -6: "point outside the root box", -7: "workspace too small",
    -8: "device structure overflowed (incomplete result)",
}
KERNELS = {"laplace": 0, "yukawa": 1, "biharmonic": 2, "helmholtz": 3}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16x3": 4, "f16x3": 5}
M2L_PATHS = {"dense": 0, "fft": 1, "auto": 2}
NUM_PHASES = 7
PHASES = ["tree", "derivatives", "p2m", "m2m", "m2l", "l2l", "leaf"]


class FMMError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")


class Pde(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int), ("multi_idx", ctypes.POINTER(ctypes.c_int)),
                ("coeff", ctypes.POINTER(ctypes.c_double))]


class Stats(ctypes.Structure):
    _fields_ = [("phase_ms", ctypes.c_float * 7), ("m2l_kernel_ms", ctypes.c_float),
                ("boxes", ctypes.c_int64), ("depth", ctypes.c_int),
                ("m2l_translations", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("status", ctypes.c_int), ("launches", ctypes.c_int)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("lam", ctypes.c_double), ("d", ctypes.c_int),
                ("p", ctypes.c_int), ("levels", ctypes.c_int), ("pde", ctypes.POINTER(Pde)),
                ("root_lo", ctypes.c_double * 3), ("root_size", ctypes.c_double),
                ("precision", ctypes.c_int), ("m2l", ctypes.c_int),
                ("max_leaf", ctypes.c_int)]


_LIB = None

EXPORTS = [
    "fmm_plan_create", "fmm_plan_destroy", "fmm_plan_info", "fmm_workspace_size", "fmm_eval",
    "fmm_eval_backward", "fmm_last_status", "fmm_set_timing", "fmm_phase_times",
    "fmm_last_launch_count", "fmm_status_string", "fmm_eval_noalloc", "fmm_m2l_kernel_time",
    "fmm_last_tree", "fmm_set_wait_limit", "fmm_last_stats", "fmm_eval_f32",
    "fmm_workspace_size_f32", "fmm_selftest_dw",
]


def lib_path() -> str:
    return build_ext.LIB


def load(build: bool = True):
    """Load libctfmm.so (building it first if allowed and out of date)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = build_ext.build() if build else build_ext.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libctfmm is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    L.fmm_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PlanDesc)]
    L.fmm_plan_create.restype = i32
    L.fmm_plan_destroy.argtypes = [vp]
    L.fmm_plan_destroy.restype = i32
    L.fmm_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.fmm_plan_info.restype = i32
    L.fmm_workspace_size.argtypes = [vp, i64, i64, ctypes.POINTER(sz)]
    L.fmm_workspace_size.restype = i32
    L.fmm_eval.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp, vp, sz, vp]
    L.fmm_eval.restype = i32
    L.fmm_eval_f32.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp, vp, sz, vp]
    L.fmm_eval_f32.restype = i32
    L.fmm_workspace_size_f32.argtypes = [vp, i64, i64, ctypes.POINTER(sz)]
    L.fmm_workspace_size_f32.restype = i32
    L.fmm_eval_backward.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.fmm_eval_backward.restype = i32
    L.fmm_eval_noalloc.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp, vp]
    L.fmm_eval_noalloc.restype = i32
    L.fmm_last_status.argtypes = [vp]
    L.fmm_last_status.restype = i32
    L.fmm_set_timing.argtypes = [vp, i32]
    L.fmm_set_timing.restype = i32
    L.fmm_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.fmm_phase_times.restype = i32
    L.fmm_m2l_kernel_time.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.fmm_m2l_kernel_time.restype = i32
    L.fmm_last_tree.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.fmm_last_tree.restype = i32
    L.fmm_last_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.fmm_last_stats.restype = i32
    L.fmm_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    L.fmm_set_wait_limit.restype = i32
    L.fmm_last_launch_count.argtypes = [vp]
    L.fmm_last_launch_count.restype = i32
    L.fmm_selftest_dw.argtypes = [i32, i64, vp, vp, vp]
    L.fmm_selftest_dw.restype = i32
    L.fmm_status_string.argtypes = [i32]
    L.fmm_status_string.restype = ctypes.c_char_p
    _LIB = L
    return L


def check(code: int, what: str) -> None:
    if code != FMM_OK:
        raise FMMError(code, what)
