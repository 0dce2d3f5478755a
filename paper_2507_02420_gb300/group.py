"""Grouped transforms: the gtt_group_* calls of include/gtt.h (marshalling only).

Group(requests) plans many transforms of uneven b, n and dtype for one CUDA
graph: a persistent kernel for the requests under 2 MiB and chains of pass
kernels for the larger ones; execute() replays it.
Each request is a dict with keys b, n, dtype ("f32" or "c64"), W (host
array), x and y (CUDA tensors of b**n elements; y may be x), inverse (bool).
"""
from __future__ import annotations

import ctypes
import json

import numpy as np
import torch

from ._lib import check, load
from .api import _stream_ptr, _w_host_bytes, dtype_code


class Request(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("n", ctypes.c_int), ("dtype", ctypes.c_int),
                ("W", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("inverse", ctypes.c_int)]


class Group:
    def __init__(self, requests):
        lib = load()
        self._lib = lib
        self._keep = []  # host W copies and tensors stay alive as long as the group
        arr = (Request * len(requests))()
        for i, rq in enumerate(requests):
            code = dtype_code(rq["dtype"])
            Wb = _w_host_bytes(np.asarray(rq["W"]), code)
            x, y = rq["x"], rq["y"]
            if not (isinstance(x, torch.Tensor) and x.is_cuda and isinstance(y, torch.Tensor) and y.is_cuda):
                raise TypeError("x and y must be CUDA tensors")
            self._keep += [Wb, x, y]
            arr[i] = Request(int(rq["b"]), int(rq["n"]), code, Wb.ctypes.data, x.data_ptr(),
                             y.data_ptr(), int(bool(rq.get("inverse", False))))
        h = ctypes.c_void_p()
        check(lib.gtt_group_create(ctypes.byref(h), len(requests), arr), "gtt_group_create")
        self._h = h

    def execute(self, stream=None):
        check(self._lib.gtt_group_execute(self._h, _stream_ptr(stream)), "gtt_group_execute")

    def check(self):
        check(self._lib.gtt_group_check(self._h), "gtt_group_check")

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(4096)
        check(self._lib.gtt_group_describe(self._h, buf, len(buf)), "gtt_group_describe")
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gtt_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
