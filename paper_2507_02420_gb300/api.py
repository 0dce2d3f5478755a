"""Python binding of libgtt: the same calls as include/gtt.h, with torch
tensors for device memory and torch's current stream.  Only argument
marshalling happens here; every step of the transform runs in the library's
CUDA kernels.
"""
from __future__ import annotations

import ctypes
import json

import numpy as np
import torch

from ._lib import check, load

F64, F32, C64, C128, I32 = 0, 1, 2, 3, 4
PREC_AUTO, PREC_FP32, PREC_BF16X3, PREC_TF32X3, PREC_BF16X2 = 0, 1, 2, 3, 4

_TORCH_DT = {F64: torch.float64, F32: torch.float32, C64: torch.complex64,
             C128: torch.complex128, I32: torch.int32}
_NP_DT = {F64: np.float64, F32: np.float32, C64: np.complex64, C128: np.complex128,
          I32: np.int32}
_FROM_TORCH = {v: k for k, v in _TORCH_DT.items()}
_NAMES = {"f64": F64, "f32": F32, "c64": C64, "c128": C128, "i32": I32}


def dtype_code(dt) -> int:
    if isinstance(dt, int):
        return dt
    if isinstance(dt, str):
        return _NAMES[dt]
    if isinstance(dt, torch.dtype):
        return _FROM_TORCH[dt]
    return _FROM_TORCH[torch.from_numpy(np.zeros(1, dtype=dt)).dtype]


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _w_host_bytes(W, code: int) -> np.ndarray:
    if isinstance(W, torch.Tensor):
        W = W.detach().cpu().numpy()
    W = np.asarray(W)
    if code == I32:
        W = (W.astype(np.int64) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    return np.ascontiguousarray(W.astype(_NP_DT[code]) if code != I32 else W)


class Plan:
    """gtt_plan_t: a b x b base matrix W, n digits, an element type and a batch."""

    def __init__(self, W, n: int, dtype=None, batch: int = 1):
        lib = load()
        Wn = W.detach().cpu().numpy() if isinstance(W, torch.Tensor) else np.asarray(W)
        if Wn.ndim != 2 or Wn.shape[0] != Wn.shape[1]:
            raise ValueError("W must be a square b x b matrix")
        code = dtype_code(dtype if dtype is not None else Wn.dtype)
        self.b, self.n, self.dtype, self.batch = int(Wn.shape[0]), int(n), code, int(batch)
        self.N = self.b ** self.n
        self._W = _w_host_bytes(Wn, code)
        h = ctypes.c_void_p()
        check(lib.gtt_plan_create(ctypes.byref(h), self.b, self.n,
                                  self._W.ctypes.data_as(ctypes.c_void_p), code, self.batch),
              "gtt_plan_create")
        self._h = h
        self._lib = lib

    @classmethod
    def mixed(cls, Ws, dtype=None, batch: int = 1) -> "Plan":
        """gtt_plan_create_mixed: G = W_0 (x) W_1 (x) ... (x) W_{n-1} with W_k of
        size b_k x b_k (W_0 acts on the most significant index), N = prod b_k."""
        lib = load()
        mats = [W.detach().cpu().numpy() if isinstance(W, torch.Tensor) else np.asarray(W) for W in Ws]
        if not mats or any(m.ndim != 2 or m.shape[0] != m.shape[1] for m in mats):
            raise ValueError("every factor must be a square matrix")
        code = dtype_code(dtype if dtype is not None else np.result_type(*mats))
        self = cls.__new__(cls)
        self.radices = [int(m.shape[0]) for m in mats]
        self.b, self.n, self.dtype, self.batch = None, len(mats), code, int(batch)
        self.N = int(np.prod(self.radices))
        self._rad = np.ascontiguousarray(self.radices, dtype=np.int32)
        self._W = np.ascontiguousarray(np.concatenate([_w_host_bytes(m, code).ravel() for m in mats]))
        h = ctypes.c_void_p()
        check(lib.gtt_plan_create_mixed(ctypes.byref(h), self.n, self._rad.ctypes.data_as(ctypes.c_void_p),
                                        self._W.ctypes.data_as(ctypes.c_void_p), code, self.batch),
              "gtt_plan_create_mixed")
        self._h = h
        self._lib = lib
        return self

    @property
    def torch_dtype(self) -> torch.dtype:
        return _TORCH_DT[self.dtype]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gtt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_w(self, W):
        """Replace W (host copy taken now) without rebuilding the schedule; for
        a mixed plan, W is the list of factors W_0 .. W_{n-1}."""
        if getattr(self, "radices", None) is not None:
            mats = [w.detach().cpu().numpy() if isinstance(w, torch.Tensor) else np.asarray(w) for w in W]
            if [m.shape for m in mats] != [(b, b) for b in self.radices]:
                raise ValueError("factor shapes differ from the plan's")
            self._W = np.ascontiguousarray(np.concatenate([_w_host_bytes(m, self.dtype).ravel() for m in mats]))
            check(self._lib.gtt_plan_set_w(self._h, self._W.ctypes.data_as(ctypes.c_void_p)), "gtt_plan_set_w")
            return
        Wn = W.detach().cpu().numpy() if isinstance(W, torch.Tensor) else np.asarray(W)
        if Wn.shape != (self.b, self.b):
            raise ValueError("W shape differs from the plan's")
        self._W = _w_host_bytes(Wn, self.dtype)
        check(self._lib.gtt_plan_set_w(self._h, self._W.ctypes.data_as(ctypes.c_void_p)), "gtt_plan_set_w")

    def set_precision(self, prec: int):
        check(self._lib.gtt_plan_set_precision(self._h, int(prec)), "gtt_plan_set_precision")

    def set_schedule(self, max_tile_bytes: int, min_run_bytes: int = 128):
        check(self._lib.gtt_plan_set_schedule(self._h, int(max_tile_bytes), int(min_run_bytes)),
              "gtt_plan_set_schedule")

    def set_passes(self, digits, runs):
        """Explicit schedule: pass k applies digits[k] modes on rows of runs[k] elements."""
        d = np.ascontiguousarray(digits, dtype=np.int32)
        r = np.ascontiguousarray(runs, dtype=np.int64)
        if d.shape != r.shape:
            raise ValueError("digits and runs must have the same length")
        check(self._lib.gtt_plan_set_passes(self._h, len(d), d.ctypes.data, r.ctypes.data),
              "gtt_plan_set_passes")

    def autotune(self, max_candidates: int = 64):
        """Time the `max_candidates` best-ranked candidate schedules (ranked by
        a model of HBM and FMA time), re-time the six fastest, and keep the
        winner (recorded in the cache)."""
        check(self._lib.gtt_plan_autotune(self._h, int(max_candidates)), "gtt_plan_autotune")

    def set_pipeline(self, use_tma: bool = True, nbuf: int = 2):
        check(self._lib.gtt_plan_set_pipeline(self._h, int(bool(use_tma)), int(nbuf)),
              "gtt_plan_set_pipeline")

    def set_chunking(self, elems: int = -1):
        """Run the leading passes chunk by chunk, at most `elems` elements per
        chunk, so that they pass data through L2 (-1 automatic, 0 off)."""
        check(self._lib.gtt_plan_set_chunking(self._h, int(elems)), "gtt_plan_set_chunking")

    def check(self):
        """Raise GTTError(GTT_ERR_TIMEOUT) if a kernel of this plan gave up a bounded wait."""
        check(self._lib.gtt_plan_check(self._h), "gtt_plan_check")

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(16384)
        check(self._lib.gtt_plan_describe(self._h, buf, len(buf)), "gtt_plan_describe")
        return json.loads(buf.value.decode())

    def set_timing(self, enable: bool):
        check(self._lib.gtt_plan_set_timing(self._h, int(bool(enable))), "gtt_plan_set_timing")

    def timing(self) -> dict:
        """Per-kernel launches and summed device ms since the last call (waits)."""
        buf = ctypes.create_string_buffer(65536)
        check(self._lib.gtt_plan_timing(self._h, buf, len(buf)), "gtt_plan_timing")
        return json.loads(buf.value.decode())

    # ---------------------------------------------------------- device calls
    def _check_dev(self, t: torch.Tensor, name: str):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.torch_dtype:
            raise TypeError(f"{name} has dtype {t.dtype}, plan expects {self.torch_dtype}")
        if not t.is_contiguous() or t.numel() != self.batch * self.N:
            raise ValueError(f"{name} must be contiguous with batch*N = {self.batch * self.N} elements")

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        self._check_dev(x, "x")
        y = torch.empty_like(x) if out is None else out
        self._check_dev(y, "out")
        check(self._lib.gtt_forward(self._h, x.data_ptr(), y.data_ptr(), _stream_ptr(stream)),
              "gtt_forward")
        return y

    def inverse(self, y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        self._check_dev(y, "y")
        x = torch.empty_like(y) if out is None else out
        self._check_dev(x, "out")
        check(self._lib.gtt_inverse(self._h, y.data_ptr(), x.data_ptr(), _stream_ptr(stream)),
              "gtt_inverse")
        return x

    def filter(self, x: torch.Tensor, cut: int, keep_low: bool = True, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
        """gtt_filter: G_N^dagger (mask * G_N x), keeping spectrum indices p < cut
        (keep_low) or p >= cut, for every vector of the batch."""
        self._check_dev(x, "x")
        y = torch.empty_like(x) if out is None else out
        self._check_dev(y, "out")
        check(self._lib.gtt_filter(self._h, x.data_ptr(), y.data_ptr(), int(cut), int(bool(keep_low)),
                                   _stream_ptr(stream)), "gtt_filter")
        return y

    def compress(self, x: torch.Tensor, k: int, spectrum: torch.Tensor | None = None, stream=None):
        """gtt_compress: (indices [batch, k] int64, values [batch, k]) of the k
        largest-magnitude coefficients of G_N x per vector; the spectrum is
        written to `spectrum` (a new tensor when None; may be x)."""
        self._check_dev(x, "x")
        spec = torch.empty_like(x) if spectrum is None else spectrum
        self._check_dev(spec, "spectrum")
        shape = (self.batch, int(k))
        idx = torch.empty(shape, dtype=torch.int64, device=x.device)
        val = torch.empty(shape, dtype=self.torch_dtype, device=x.device)
        check(self._lib.gtt_compress(self._h, x.data_ptr(), spec.data_ptr(), int(k), idx.data_ptr(),
                                     val.data_ptr(), _stream_ptr(stream)), "gtt_compress")
        return idx, val

    def decompress(self, indices: torch.Tensor, values: torch.Tensor, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """gtt_decompress: G_N^dagger of the spectrum holding `values` at `indices`."""
        if indices.dtype != torch.int64 or not indices.is_cuda or not indices.is_contiguous():
            raise TypeError("indices must be a contiguous CUDA int64 tensor")
        if values.dtype != self.torch_dtype or not values.is_cuda or not values.is_contiguous():
            raise TypeError(f"values must be a contiguous CUDA {self.torch_dtype} tensor")
        k = int(indices.shape[-1])
        if indices.numel() != self.batch * k or values.numel() != self.batch * k:
            raise ValueError("indices and values must be [batch, k]")
        y = torch.empty((self.batch, self.N), dtype=self.torch_dtype, device=values.device) if out is None else out
        self._check_dev(y, "out")
        check(self._lib.gtt_decompress(self._h, indices.data_ptr(), values.data_ptr(), k, y.data_ptr(),
                                       _stream_ptr(stream)), "gtt_decompress")
        return y

    def backward(self, x: torch.Tensor, dy: torch.Tensor, need_dx: bool = True,
                 need_dW: bool = True, stream=None):
        self._check_dev(x, "x")
        self._check_dev(dy, "dy")
        dx = torch.empty_like(dy) if need_dx else None
        # (a mixed plan has no single b; the library rejects its backward)
        dW = torch.empty((self.b, self.b), dtype=self.torch_dtype, device=dy.device) if need_dW and self.b else None
        check(self._lib.gtt_backward(self._h, x.data_ptr(), dy.data_ptr(),
                                     dx.data_ptr() if dx is not None else None,
                                     dW.data_ptr() if dW is not None else None,
                                     _stream_ptr(stream)), "gtt_backward")
        return dx, dW

    def forward_saving(self, x: torch.Tensor, out: torch.Tensor | None = None,
                       ckpt: torch.Tensor | None = None, stream=None):
        """gtt_forward_saving: y = G_N x, keeping in `ckpt` the activation that
        backward_saved needs (so the backward recomputes nothing).  Returns
        (y, ckpt); raises GTTError with status GTT_ERR_UNSUPPORTED (2) when
        the plan's schedules allow no such checkpoint."""
        self._check_dev(x, "x")
        y = torch.empty_like(x) if out is None else out
        ck = torch.empty_like(x) if ckpt is None else ckpt
        self._check_dev(y, "out")
        self._check_dev(ck, "ckpt")
        check(self._lib.gtt_forward_saving(self._h, x.data_ptr(), y.data_ptr(), ck.data_ptr(), _stream_ptr(stream)),
              "gtt_forward_saving")
        return y, ck

    def backward_saved(self, x: torch.Tensor, ckpt: torch.Tensor, dy: torch.Tensor, need_dx: bool = True,
                       need_dW: bool = True, stream=None):
        """gtt_backward_saved: backward() with the checkpoint from forward_saving."""
        self._check_dev(x, "x")
        self._check_dev(ckpt, "ckpt")
        self._check_dev(dy, "dy")
        dx = torch.empty_like(dy) if need_dx else None
        dW = torch.empty((self.b, self.b), dtype=self.torch_dtype, device=dy.device) if need_dW and self.b else None
        check(self._lib.gtt_backward_saved(self._h, x.data_ptr(), ckpt.data_ptr(), dy.data_ptr(),
                                           dx.data_ptr() if dx is not None else None,
                                           dW.data_ptr() if dW is not None else None,
                                           _stream_ptr(stream)), "gtt_backward_saved")
        return dx, dW

    # ------------------------------------------------------------ host calls
    def _host_arrays(self, x):
        xa = x.numpy() if isinstance(x, torch.Tensor) else np.asarray(x)
        if xa.dtype != _NP_DT[self.dtype] or not xa.flags.c_contiguous or xa.size != self.batch * self.N:
            raise ValueError("host buffer must be a contiguous array of the plan's dtype and size")
        return xa

    def forward_host(self, x, out=None, stream=None):
        """y = G_N x on HOST buffers (numpy arrays or CPU tensors); blocks."""
        xa = self._host_arrays(x)
        y = np.empty_like(xa) if out is None else out
        ya = self._host_arrays(y)
        check(self._lib.gtt_forward_host(self._h, xa.ctypes.data, ya.ctypes.data, _stream_ptr(stream)),
              "gtt_forward_host")
        return y

    def inverse_host(self, y, out=None, stream=None):
        ya = self._host_arrays(y)
        x = np.empty_like(ya) if out is None else out
        xa = self._host_arrays(x)
        check(self._lib.gtt_inverse_host(self._h, ya.ctypes.data, xa.ctypes.data, _stream_ptr(stream)),
              "gtt_inverse_host")
        return x


def autotune_cache_load(path: str):
    check(load().gtt_autotune_cache_load(path.encode()), "gtt_autotune_cache_load")


def autotune_cache_save(path: str):
    check(load().gtt_autotune_cache_save(path.encode()), "gtt_autotune_cache_save")


def selftest_bounded_wait(polls: int = 1000, stream=None) -> bool:
    """Run gtt_selftest_bounded_wait: True when the bounded mbarrier wait
    expired (the expected outcome), reported through a device flag."""
    out = ctypes.c_int(0)
    check(load().gtt_selftest_bounded_wait(int(polls), ctypes.byref(out), _stream_ptr(stream)),
          "gtt_selftest_bounded_wait")
    return bool(out.value)
