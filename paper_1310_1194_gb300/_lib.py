"""ctypes binding of libfei.so (the C ABI in include/fei.h).

Argument marshalling only: every step of the integration runs in the
library's CUDA kernels.  Importing this module loads the in-tree
``_build/libfei.so`` and raises ImportError when it is missing -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfei.so")

FEI_OK = 0
FEI_ERR_INVALID_ARG = 1
FEI_ERR_INVALID_DEGREE = 2
FEI_ERR_NEGATIVE_JACOBIAN = 3
FEI_ERR_NONFINITE = 4
FEI_ERR_CUDA = 5
FEI_ERR_TIMEOUT = 6
FEI_ERR_UNSUPPORTED = 7
FEI_ERR_OOM = 8

FEI_FP64 = 0
FEI_FP32 = 1
FEI_TC_F16X3 = 2
FEI_TC_3XTF32 = 3
FEI_SF_FP32 = 4
FEI_AUTO = 5

FEI_COEF_PER_ELEMENT = 0
FEI_COEF_PER_POINT = 1

FEI_A_FULL = 0
FEI_A_UPPER = 1

PRECISIONS = {"fp64": FEI_FP64, "fp32": FEI_FP32, "tc_f16x3": FEI_TC_F16X3, "tc_3xtf32": FEI_TC_3XTF32,
              "sf_fp32": FEI_SF_FP32, "auto": FEI_AUTO}
# fei_plan_kernel
KERNELS = {0: "cuda_core", 1: "tensor_core", 2: "sum_factorised"}

FEI_NOALLOC_MAX_ELEM = 262144


class fei_batch(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int64),
        ("geom", ctypes.c_void_p),
        ("degree", ctypes.c_void_p),
        ("uniform_degree", ctypes.c_int32),
        ("coef_mode", ctypes.c_int32),
        ("K", ctypes.c_void_p),
        ("b", ctypes.c_void_p),
        ("c", ctypes.c_void_p),
        ("f", ctypes.c_void_p),
        ("A_offset", ctypes.c_void_p),
        ("b_offset", ctypes.c_void_p),
        ("q_offset", ctypes.c_void_p),
        ("a_layout", ctypes.c_int32),
    ]


class fei_coef_grad(ctypes.Structure):
    _fields_ = [("K", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("f", ctypes.c_void_p)]


class FeiError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where} failed with status {status}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libfei.so is not built ({LIB_PATH}); run `python -m paper_1310_1194_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    ref_p = ctypes.POINTER(vp)
    lib.fei_reference_create.argtypes = [ctypes.c_int, ref_p]
    lib.fei_reference_destroy.argtypes = [vp]
    lib.fei_reference_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]
    lib.fei_reference_copy_table.argtypes = [vp, vp, vp]
    lib.fei_integrate.argtypes = [ref_p, ctypes.c_int, ctypes.POINTER(fei_batch), ctypes.c_int,
                                  vp, vp, vp, vp]
    lib.fei_integrate_backward.argtypes = [ref_p, ctypes.c_int, ctypes.POINTER(fei_batch), ctypes.c_int,
                                           vp, vp, vp, ctypes.POINTER(fei_coef_grad), vp]
    lib.fei_integrate_backward_quadratic.argtypes = [ref_p, ctypes.c_int, ctypes.POINTER(fei_batch), ctypes.c_int,
                                                     vp, vp, ctypes.POINTER(fei_coef_grad), vp]
    lib.fei_plan_offsets.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    lib.fei_plan_offsets_upper.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    lib.fei_status_summary.argtypes = [vp, i64, vp, vp]
    lib.fei_sync_status.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(i64), vp]
    lib.fei_integrate_noalloc.argtypes = [ref_p, ctypes.c_int, ctypes.POINTER(fei_batch), ctypes.c_int,
                                          vp, vp, vp, vp]
    lib.fei_plan_create.argtypes = [ref_p, ctypes.c_int, i64, ctypes.c_int, ref_p]
    lib.fei_plan_destroy.argtypes = [vp]
    lib.fei_plan_execute.argtypes = [vp, ctypes.POINTER(fei_batch), vp, vp, vp, vp]
    lib.fei_plan_tune.argtypes = [vp, ctypes.POINTER(fei_batch), vp, vp, vp, vp]
    lib.fei_plan_choice.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64),
                                    ctypes.POINTER(ctypes.c_float)]
    lib.fei_assembly_create.argtypes = [i64, vp, i32, vp, i64, i32, ref_p]
    lib.fei_assembly_destroy.argtypes = [vp]
    lib.fei_assembly_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32)]
    lib.fei_assembly_pattern.argtypes = [vp, vp, vp, vp]
    lib.fei_assemble.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.fei_integrate_assemble.argtypes = [vp, ref_p, ctypes.c_int, ctypes.POINTER(fei_batch), ctypes.c_int,
                                           vp, vp, vp, vp]
    lib.fei_debug_set_wait_limit.argtypes = [ctypes.c_uint64]
    lib.fei_plan_set_choice.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64]
    lib.fei_plan_kernel.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i32)]
    lib.fei_pipeline_create.argtypes = [ref_p, ctypes.c_int, ctypes.c_int, i64, ref_p]
    lib.fei_pipeline_destroy.argtypes = [vp]
    lib.fei_pipeline_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.fei_integrate_host.argtypes = [vp, ctypes.POINTER(fei_batch), vp, vp, vp, ctypes.POINTER(i64), vp]
    lib.fei_last_error_string.argtypes = []
    lib.fei_last_error_string.restype = ctypes.c_char_p
    for name in ("fei_reference_create", "fei_reference_destroy", "fei_reference_info",
                 "fei_reference_copy_table", "fei_integrate", "fei_integrate_backward",
                 "fei_integrate_backward_quadratic",
                 "fei_plan_offsets", "fei_plan_offsets_upper", "fei_integrate_noalloc", "fei_plan_create", "fei_plan_destroy",
                 "fei_plan_execute", "fei_plan_tune", "fei_plan_choice", "fei_status_summary", "fei_sync_status",
                 "fei_assembly_create", "fei_assembly_destroy", "fei_assembly_info", "fei_assembly_pattern",
                 "fei_assemble", "fei_integrate_assemble", "fei_debug_set_wait_limit", "fei_plan_set_choice",
                 "fei_plan_kernel",
                 "fei_pipeline_create", "fei_pipeline_destroy", "fei_pipeline_info", "fei_integrate_host"):
        getattr(lib, name).restype = i32
    return lib


lib = _load()


def check(status: int, where: str):
    if status != FEI_OK:
        msg = lib.fei_last_error_string()
        raise FeiError(status, where, msg.decode() if msg else "")


def last_error() -> str:
    msg = lib.fei_last_error_string()
    return msg.decode() if msg else ""
