"""ctypes binding of libfftc.so (the C ABI in include/fftc.h): argument marshalling only.

The library must have been built (``paper_2308_00497_gb300.build.build()``); there
is no fallback of any kind: loading fails loudly if the shared object is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfftc.so")

# enums of include/fftc.h
LAYOUT_INTERLEAVED, LAYOUT_SPLIT = 0, 1
FORWARD, INVERSE = -1, 1
FP32, FP16_TC, BF16_TC, FP16_TC_SPLIT, BF16_TC_SPLIT, FP64 = 0, 1, 2, 3, 4, 5
(OK, ERR_INVALID_VALUE, ERR_UNSUPPORTED_SIZE, ERR_MISALIGNED, ERR_ALLOC, ERR_CUDA,
 ERR_INVALID_PLAN, ERR_TIMEOUT) = range(8)

LAYOUTS = {"interleaved": LAYOUT_INTERLEAVED, "split": LAYOUT_SPLIT}
PRECISIONS = {"fp32": FP32, "fp16_tc": FP16_TC, "bf16_tc": BF16_TC,
              "fp16_tc_split": FP16_TC_SPLIT, "bf16_tc_split": BF16_TC_SPLIT, "fp64": FP64}

_c_i64, _c_int, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p

# name -> (restype, argtypes), in the order of include/fftc.h
PROTOTYPES = {
    "fftc_plan_create": (_vp, [_c_i64, _c_i64, _c_int, _c_int, _c_int]),
    "fftc_execute": (_c_int, [_vp, _vp, _vp, _vp]),
    "fftc_execute_host": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fftc_plan_bytes": (_c_i64, [_vp]),
    "fftc_destroy": (_c_int, [_vp]),
    "fftc_get_last_error": (_c_int, []),
    "fftc_status_string": (ctypes.c_char_p, [_c_int]),
    "fftc_plan_info": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "fftc_plan_create_uneven": (_vp, [_c_i64, _vp, _vp, _vp, _c_int, _c_int]),
    "fftc_plan_create_nd": (_vp, [_c_int, _vp, _c_i64, _c_int, _c_int, _c_int]),
    "fftc_plan_tune": (_c_int, [_vp, _c_int]),
    "fftc_plan_split": (_c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "fftc_plan_check": (_c_int, [_vp, _vp]),
    "fftc_execute_pointwise": (_c_int, [_vp, _vp, _vp, _vp, ctypes.c_float, _vp]),
    "fftc_plan_timing": (_c_int, [_vp, _c_int]),
    "fftc_plan_pass_times": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_int)]),
    "fftc_execute_noalloc": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _vp, _vp, _vp]),
    "fftc_stage_twiddles": (_c_int, [_c_int, _c_int, _vp, _c_i64, ctypes.POINTER(_c_i64)]),
}

_lib = None


class FftcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        name = status_string(status)
        super().__init__(f"{what}: {name}" if what else name)


def load() -> ctypes.CDLL:
    """Load libfftc.so once and declare its prototypes."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2308_00497_gb300.build.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().fftc_status_string(int(status)).decode()


def check(status: int, what: str = "") -> None:
    if status != OK:
        raise FftcError(status, what)
