"""ctypes loader for libils.so (the C ABI of include/ils.h).

Argument marshalling only.  There is no fallback: if the shared library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libils.so")

STATUS = {
    0: "ILS_OK",
    1: "ILS_ERR_INVALID_ARG",
    2: "ILS_ERR_UNSUPPORTED_SIZE",
    3: "ILS_ERR_OOM",
    4: "ILS_ERR_CUDA",
    5: "ILS_ERR_TIMEOUT",
    6: "ILS_ERR_FALLBACK_TAKEN",
}

ILS_ERR_FALLBACK_TAKEN = 6

_lib = None

c_int, c_float, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_void_p
P = ctypes.POINTER


class ILSError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


class Frame(ctypes.Structure):
    """Mirror of ils_frame (include/ils.h)."""
    _fields_ = [("H", c_int), ("W", c_int), ("C", c_int), ("N", c_int),
                ("lam", c_float), ("p", c_float), ("eps", c_float),
                ("f", c_void_p), ("u", c_void_p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "ils_status_string": (ctypes.c_char_p, [c_int]),
    "ils_last_error": (ctypes.c_char_p, []),
    "ils_plan_create": (c_int, [c_int, c_int, c_int, c_float, c_float, c_float, c_int, P(c_void_p)]),
    "ils_plan_create_welsch": (c_int, [c_int, c_int, c_int, c_float, c_float, c_int, c_void_p]),
    "ils_plan_create_hqs": (c_int, [c_int, c_int, c_int, c_float, c_float, c_float, c_int, c_void_p]),
    "ils_plan_destroy": (c_int, [c_void_p]),
    "ils_plan_c": (c_float, [c_void_p]),
    "ils_smooth": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_smooth_enhance": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_void_p]),
    "ils_smooth_luma": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_void_p]),
    "ils_smooth_hwc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_gaussian_blur": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_float, c_void_p]),
    "ils_smooth_presmoothed": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_void_p]),
    "ils_log_luma": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "ils_tonemap_log": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_float, c_float, c_void_p]),
    "ils_smooth_from": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_smooth_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_smooth_checkpointed": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_backward_ckpt": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ils_set_checkpointing": (c_int, [c_void_p, c_int]),
    "ils_set_profiling": (c_int, [c_void_p, c_int]),
    "ils_get_profile": (c_int, [c_void_p, P(ctypes.c_double), P(ctypes.c_longlong)]),
    "ils_batch_create": (c_int, [ctypes.c_void_p, c_int, c_int, P(c_void_p)]),
    "ils_batch_run": (c_int, [c_void_p, c_void_p]),
    "ils_batch_destroy": (c_int, [c_void_p]),
    "ils_batch_kernel_choice": (c_int, [c_void_p, c_int, P(c_int), P(c_int)]),
    "ils_smooth_batched": (c_int, [ctypes.c_void_p, c_int, c_void_p]),
    "ils_cnn_param_count": (ctypes.c_longlong, []),
    "ils_cnn_create": (c_int, [ctypes.c_longlong, P(c_void_p)]),
    "ils_cnn_destroy": (c_int, [c_void_p]),
    "ils_cnn_set_weights": (c_int, [c_void_p, c_void_p, ctypes.c_longlong]),
    "ils_cnn_get_weights": (c_int, [c_void_p, c_void_p, ctypes.c_longlong]),
    "ils_cnn_get_adam": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_longlong, P(ctypes.c_longlong)]),
    "ils_cnn_set_adam": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_longlong, ctypes.c_longlong]),
    "ils_cnn_get_grads": (c_int, [c_void_p, c_void_p, ctypes.c_longlong]),
    "ils_cnn_forward": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "ils_cnn_backward": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "ils_cnn_infer": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "ils_cnn_zero_grad": (c_int, [c_void_p, c_void_p]),
    "ils_cnn_uses_tcgen05": (c_int, [c_void_p]),
    "ils_cnn_check": (c_int, [c_void_p]),
    "ils_cnn_adam_step": (c_int, [c_void_p, c_float, c_float, c_float, c_float, c_void_p]),
    "ils_mse": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_longlong, c_void_p, c_void_p]),
    "ils_warm_create": (c_int, [c_int, c_int, c_int, c_float, c_float, c_float, c_int, c_int, c_float, c_void_p,
                                P(c_void_p)]),
    "ils_warm_destroy": (c_int, [c_void_p]),
    "ils_warm_smooth": (c_int, [c_void_p, c_void_p, c_void_p, P(c_int), P(c_float), c_void_p]),
    "ils_warm_result": (c_int, [c_void_p, P(c_int), P(c_float)]),
    "ils_smooth_noalloc": (c_int, [c_int, c_int, c_int, c_float, c_float, c_float, c_int,
                                   c_void_p, c_void_p, c_void_p]),
}

KERNEL_KINDS = ("row_first", "row", "column", "row_inverse")


def lib():
    """The loaded library (loads it on first use; raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2003_07504_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        detail = ""
        if status == 4:
            detail = lib().ils_last_error().decode(errors="replace")
        raise ILSError(status, where, detail)
