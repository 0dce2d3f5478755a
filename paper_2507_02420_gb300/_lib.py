"""ctypes loader for libgtt.so: argument marshalling only.

There is no fallback: if the library is missing or does not load, every call
raises.  Build it with ``python -m paper_2507_02420_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# GTT_LIBRARY=debug loads the debug build (libgtt_debug.so: the same kernels
# with every tile and global index checked, violations reported through
# gtt_plan_check / gtt_group_check); anything else the release build.
DEBUG = os.environ.get("GTT_LIBRARY", "") == "debug"
LIB_PATH = os.path.join(_HERE, "libgtt_debug.so" if DEBUG else "libgtt.so")

_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_S = ctypes.c_size_t

# name -> (restype, argtypes), mirroring include/gtt.h
SIGNATURES = {
    "gtt_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _P, _I, _LL]),
    "gtt_plan_create_mixed": (_I, [ctypes.POINTER(_P), _I, _P, _P, _I, _LL]),
    "gtt_plan_set_precision": (_I, [_P, _I]),
    "gtt_plan_set_w": (_I, [_P, _P]),
    "gtt_plan_set_schedule": (_I, [_P, _LL, _LL]),
    "gtt_plan_set_pipeline": (_I, [_P, _I, _I]),
    "gtt_plan_set_passes": (_I, [_P, _I, _P, _P]),
    "gtt_plan_autotune": (_I, [_P, _I]),
    "gtt_autotune_cache_load": (_I, [ctypes.c_char_p]),
    "gtt_autotune_cache_save": (_I, [ctypes.c_char_p]),
    "gtt_plan_check": (_I, [_P]),
    "gtt_plan_set_chunking": (_I, [_P, _LL]),
    "gtt_forward": (_I, [_P, _P, _P, _P]),
    "gtt_inverse": (_I, [_P, _P, _P, _P]),
    "gtt_backward": (_I, [_P, _P, _P, _P, _P, _P]),
    "gtt_forward_saving": (_I, [_P, _P, _P, _P, _P]),
    "gtt_backward_saved": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "gtt_backward_noalloc": (_I, [_P, _P, _P, _P, _P, _P]),
    "gtt_filter": (_I, [_P, _P, _P, _LL, _I, _P]),
    "gtt_compress": (_I, [_P, _P, _P, _LL, _P, _P, _P]),
    "gtt_decompress": (_I, [_P, _P, _P, _LL, _P, _P]),
    "gtt_forward_host": (_I, [_P, _P, _P, _P]),
    "gtt_inverse_host": (_I, [_P, _P, _P, _P]),
    "gtt_plan_describe": (_I, [_P, ctypes.c_char_p, _S]),
    "gtt_plan_set_timing": (_I, [_P, _I]),
    "gtt_plan_timing": (_I, [_P, ctypes.c_char_p, _S]),
    "gtt_plan_destroy": (_I, [_P]),
    "gtt_last_error": (ctypes.c_char_p, []),
    "gtt_group_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "gtt_group_execute": (_I, [_P, _P]),
    "gtt_group_check": (_I, [_P]),
    "gtt_group_describe": (_I, [_P, ctypes.c_char_p, _S]),
    "gtt_group_destroy": (_I, [_P]),
    "gtt_selftest_bounded_wait": (_I, [_I, ctypes.POINTER(_I), _P]),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -m paper_2507_02420_gb300.build" + (" --debug)" if DEBUG else ")"))
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


STATUS = {0: "GTT_OK", 1: "GTT_ERR_INVALID_ARG", 2: "GTT_ERR_UNSUPPORTED", 3: "GTT_ERR_ALLOC",
          4: "GTT_ERR_CUDA", 5: "GTT_ERR_TIMEOUT", 6: "GTT_ERR_INTERNAL"}


class GTTError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().gtt_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != 0:
        raise GTTError(status, where)
