"""FP64 CPU oracle for the Generalized Tensor Transform -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The
CUDA library never calls it; the two share no code.  Inputs come from
``gtt_inputs`` (random draws only).

Routes (each cites the passage it follows; the C source has the details):

* ``dense(W, x)``           -- G_N(p,q) = prod_j W[p_j, q_j]   (Sec. 2.6)
* ``dense_matrix(W, n)``    -- that matrix itself
* ``basis_matrix(W, n)``    -- G_N(p,q) = f_q(x_p), x_p = (2p+1)/(2N) through the
                               recursive basis functions (Sec. 2.2, Eq. defGNOne)
* ``alg1(W, x)``            -- the recursive FastGTT of Sec. 3 (Algorithm 1)
* ``modes(W, x)``           -- mode-by-mode loop, digit 0 first (Sec. 3.1 cost
                               structure); the timed CPU baseline
* ``adjoint(W, y)``         -- G_N^dagger y = (W^H)^{(x)n} y (Sec. 4 inverse)
* ``topk(W, x, k)``         -- compression step of Sec. 4.1.5: the k
                               coefficients of largest magnitude of G_N x per
                               vector, |c| descending, ties by larger index
* ``reconstruct(W, i, v, N)`` -- decompression: G_N^dagger of the spectrum
                               holding v at i, zero elsewhere
* ``kron_dense(Ws, x)``     -- the heterogeneous transform of the remark after
                               Def. 2.3: G = W_0 (x) W_1 (x) ... (x) W_{n-1}
                               (numpy's Kronecker product), N = prod b_k
* ``modes_mixed(Ws, x)``    -- the same transform one factor at a time: W_k
                               applied along axis k of x viewed as
                               [b_0, ..., b_{n-1}] (axis 0 most significant)
* ``modes_mixed_u32(Ws, x)``-- that loop on int32 data, arithmetic mod 2^32
* ``filter(W, x, cut, low)`` -- natural-order filtering (Sec. 4.3.2): the
                               spectrum G_N x, coefficients with index >= cut
                               (low-pass) or < cut (high-pass) set to zero,
                               then G_N^dagger
* ``grad(W, x, dy)``        -- (dx, dW) of y = G_N x for a real loss, PyTorch's
                               conjugate convention (no counterpart in the paper)
* ``fd_grad_*``             -- central finite differences of a real loss
* ``*_u32``                 -- uint32 (mod 2^32) integer versions

Parity status: every route above is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gtt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/liboracle.so (portable flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        LL = ctypes.c_longlong
        sigs = {
            "oracle_dense_c": [I, I, P, P, P],
            "oracle_dense_matrix_c": [I, I, P, P],
            "oracle_dense_u32": [I, I, P, P, P],
            "oracle_basis_matrix_c": [I, I, P, P],
            "oracle_alg1_c": [I, I, P, P, P],
            "oracle_modes_c": [I, I, P, LL, P, P, I],
            "oracle_modes_r": [I, I, P, LL, P, P, I],
            "oracle_modes_u32": [I, I, P, LL, P, P, I],
            "oracle_mode_pass_c": [I, I, P, I, P, P, I],
            "oracle_adjoint_c": [I, I, P, LL, P, P, I],
            "oracle_adjoint_r": [I, I, P, LL, P, P, I],
            "oracle_grad_c": [I, I, P, LL, P, P, P, P, I],
            "oracle_grad_r": [I, I, P, LL, P, P, P, P, I],
        }
        for name, args in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = I
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nb(W: np.ndarray, N: int) -> tuple[int, int]:
    b = W.shape[0]
    if W.shape != (b, b) or b < 2:
        raise ValueError("W must be b x b with b >= 2")
    n = 0
    m = 1
    while m < N:
        m *= b
        n += 1
    if m != N or n < 1:
        raise ValueError(f"length {N} is not a positive power of b={b}")
    return b, n


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------- routes

def dense(W, x) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    b, n = _nb(W, x.shape[-1])
    y = np.empty_like(x)
    _check(_load().oracle_dense_c(b, n, _ptr(W), _ptr(x), _ptr(y)), "dense")
    return y


def dense_matrix(W, n: int) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.complex128)
    b = W.shape[0]
    N = b ** n
    G = np.empty((N, N), dtype=np.complex128)
    _check(_load().oracle_dense_matrix_c(b, n, _ptr(W), _ptr(G)), "dense_matrix")
    return G


def basis_matrix(W, n: int) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.complex128)
    b = W.shape[0]
    N = b ** n
    G = np.empty((N, N), dtype=np.complex128)
    _check(_load().oracle_basis_matrix_c(b, n, _ptr(W), _ptr(G)), "basis_matrix")
    return G


def alg1(W, x) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    b, n = _nb(W, x.shape[-1])
    y = np.empty_like(x)
    _check(_load().oracle_alg1_c(b, n, _ptr(W), _ptr(x), _ptr(y)), "alg1")
    return y


def _batched(x: np.ndarray, N: int) -> int:
    return int(x.size // N)


def modes(W, x, threads: int | None = None) -> np.ndarray:
    """G_N applied to x[..., N] (any leading batch shape).  Real W and real x
    run in float64, anything complex in complex128."""
    threads = default_threads() if threads is None else threads
    real = not (np.iscomplexobj(W) or np.iscomplexobj(x))
    dt = np.float64 if real else np.complex128
    W = np.ascontiguousarray(W, dtype=dt)
    x = np.ascontiguousarray(x, dtype=dt)
    b, n = _nb(W, x.shape[-1])
    y = np.empty_like(x)
    fn = _load().oracle_modes_r if real else _load().oracle_modes_c
    _check(fn(b, n, _ptr(W), _batched(x, b ** n), _ptr(x), _ptr(y), threads), "modes")
    return y


def mode_pass(W, x, k: int, out=None, threads: int | None = None) -> np.ndarray:
    """One mode-k pass (W applied to digit k) of a single complex vector."""
    threads = default_threads() if threads is None else threads
    W = np.ascontiguousarray(W, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    b, n = _nb(W, x.shape[-1])
    y = np.empty_like(x) if out is None else out
    _check(_load().oracle_mode_pass_c(b, n, _ptr(W), int(k), _ptr(x), _ptr(y), threads), "mode_pass")
    return y


def adjoint(W, y, threads: int | None = None) -> np.ndarray:
    """G_N^dagger y = (W^H)^{(x)n} y."""
    threads = default_threads() if threads is None else threads
    real = not (np.iscomplexobj(W) or np.iscomplexobj(y))
    dt = np.float64 if real else np.complex128
    W = np.ascontiguousarray(W, dtype=dt)
    y = np.ascontiguousarray(y, dtype=dt)
    b, n = _nb(W, y.shape[-1])
    x = np.empty_like(y)
    fn = _load().oracle_adjoint_r if real else _load().oracle_adjoint_c
    _check(fn(b, n, _ptr(W), _batched(y, b ** n), _ptr(y), _ptr(x), threads), "adjoint")
    return x


def topk(W, x, k: int, threads: int | None = None):
    """Compression step of Sec. 4.1.5: the spectrum c = G_N x and, per vector,
    the k coefficients of largest |c|, ordered by |c| descending and, between
    equal magnitudes, by the larger index first.  Returns (indices, values),
    both [batch, k]."""
    c = np.atleast_2d(modes(W, x, threads=threads))
    mag = c.real ** 2 + c.imag ** 2 if np.iscomplexobj(c) else c * c
    idx = np.arange(c.shape[-1])
    order = np.stack([np.lexsort((-idx, -m))[:k] for m in mag])
    return order, np.take_along_axis(c, order, axis=1)


def reconstruct(W, indices, values, N: int, threads: int | None = None) -> np.ndarray:
    """Decompression: G_N^dagger of the spectrum that holds `values` at
    `indices` (both [batch, k]) and zero elsewhere."""
    values = np.atleast_2d(values)
    spec = np.zeros((values.shape[0], N), dtype=np.result_type(values, np.float64))
    np.put_along_axis(spec, np.atleast_2d(indices), values, axis=1)
    return adjoint(W, spec, threads=threads)


def kron_dense(Ws, x) -> np.ndarray:
    """G x with G = W_0 (x) ... (x) W_{n-1} formed explicitly (small N only)."""
    G = np.array([[1.0]])
    for W in Ws:
        G = np.kron(G, np.asarray(W))
    x = np.asarray(x)
    return x @ G.T if x.ndim > 1 else G @ x


def modes_mixed(Ws, x) -> np.ndarray:
    """G x for G = W_0 (x) ... (x) W_{n-1}: view each vector as the tensor
    [b_0, ..., b_{n-1}] (row-major, so axis 0 is the most significant index)
    and apply W_k along axis k, one factor after the other."""
    Ws = [np.asarray(W, dtype=np.complex128 if np.iscomplexobj(W) or np.iscomplexobj(x) else np.float64)
          for W in Ws]
    dt = np.result_type(*Ws, np.asarray(x).dtype, np.float64)
    x = np.atleast_2d(np.asarray(x, dtype=dt))
    dims = [W.shape[0] for W in Ws]
    t = x.reshape([x.shape[0]] + dims)
    for k, W in enumerate(Ws):
        t = np.moveaxis(np.tensordot(W, t, axes=([1], [k + 1])), 0, k + 1)
    return t.reshape(x.shape)


def modes_mixed_u32(Ws, x) -> np.ndarray:
    """The heterogeneous transform on int32 data with arithmetic modulo 2^32
    (the integer reading of the remark after Def. 2.3): the same factor-by-
    factor loop as ``modes_mixed``, on unsigned 64-bit integers reduced mod
    2^32 after every factor.  Every product of two values below 2^32 fits
    64 bits and 2^32 divides 2^64, so a wrapped 64-bit sum is still exact
    modulo 2^32.  Returns uint32 (the bit patterns of the int32 result)."""
    mask = np.uint64(0xFFFFFFFF)
    Ws = [np.asarray(np.asarray(W).astype(np.int64) & 0xFFFFFFFF, dtype=np.uint64) for W in Ws]
    x = np.atleast_2d(np.asarray(np.asarray(x).astype(np.int64) & 0xFFFFFFFF, dtype=np.uint64))
    dims = [W.shape[0] for W in Ws]
    t = x.reshape([x.shape[0]] + dims)
    for k, W in enumerate(Ws):
        t = np.moveaxis(t, k + 1, -1)          # axis k last: [..., b_k]
        acc = np.zeros(t.shape, dtype=np.uint64)
        for i in range(W.shape[0]):
            s = np.zeros(t.shape[:-1], dtype=np.uint64)
            for j in range(W.shape[1]):
                s = (s + W[i, j] * t[..., j]) & mask
            acc[..., i] = s
        t = np.moveaxis(acc, -1, k + 1)
    return np.ascontiguousarray(t.reshape(x.shape).astype(np.uint32))


def filter(W, x, cut: int, keep_low: bool = True, threads: int | None = None) -> np.ndarray:
    """Natural-order spectral filter of Sec. 4.3.2: spectrum s = G_N x; keep
    the coefficients s[p] with p < cut (keep_low) or p >= cut (high-pass),
    zero the others, per vector of the batch; return G_N^dagger of the result."""
    s = modes(W, x, threads=threads)
    p = np.arange(s.shape[-1])
    keep = p < cut if keep_low else p >= cut
    return adjoint(W, np.where(keep, s, 0), threads=threads)


def grad(W, x, dy, threads: int | None = None):
    """(dx, dW) for y = G_N x given dy = dL/dy (real loss L).  dx has x's
    shape; dW is b x b, summed over the batch."""
    threads = default_threads() if threads is None else threads
    real = not (np.iscomplexobj(W) or np.iscomplexobj(x) or np.iscomplexobj(dy))
    dt = np.float64 if real else np.complex128
    W = np.ascontiguousarray(W, dtype=dt)
    x = np.ascontiguousarray(x, dtype=dt)
    dy = np.ascontiguousarray(dy, dtype=dt)
    b, n = _nb(W, x.shape[-1])
    dx = np.empty_like(x)
    dW = np.empty((b, b), dtype=dt)
    fn = _load().oracle_grad_r if real else _load().oracle_grad_c
    _check(fn(b, n, _ptr(W), _batched(x, b ** n), _ptr(x), _ptr(dy), _ptr(dx), _ptr(dW),
              threads), "grad")
    return dx, dW


def dense_u32(W, x) -> np.ndarray:
    W = np.ascontiguousarray(np.asarray(W).astype(np.int64) & 0xFFFFFFFF, dtype=np.uint32)
    x = np.ascontiguousarray(np.asarray(x).astype(np.int64) & 0xFFFFFFFF, dtype=np.uint32)
    b, n = _nb(W, x.shape[-1])
    y = np.empty_like(x)
    _check(_load().oracle_dense_u32(b, n, _ptr(W), _ptr(x), _ptr(y)), "dense_u32")
    return y


def modes_u32(W, x, threads: int | None = None) -> np.ndarray:
    threads = default_threads() if threads is None else threads
    W = np.ascontiguousarray(np.asarray(W).astype(np.int64) & 0xFFFFFFFF, dtype=np.uint32)
    x = np.ascontiguousarray(np.asarray(x).astype(np.int64) & 0xFFFFFFFF, dtype=np.uint32)
    b, n = _nb(W, x.shape[-1])
    y = np.empty_like(x)
    _check(_load().oracle_modes_u32(b, n, _ptr(W), _batched(x, b ** n), _ptr(x), _ptr(y),
                                    threads), "modes_u32")
    return y


# ------------------------------------------------ O7: finite differences

def masked_square_loss(W, x, m) -> float:
    """L = sum(m * |y|^2) with y = G_N x, in FP64."""
    y = modes(W, x, threads=1)
    return float(np.sum(np.asarray(m, dtype=np.float64) * np.abs(y) ** 2))


def fd_grad_real(W, x, m, h_rel: float = 1e-6):
    """Central differences of L = sum(m * y^2) for real W, x: returns
    (dL/dx, dL/dW) with step h = h_rel * max(1, |theta|) per coordinate."""
    W = np.array(W, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    dW = np.zeros_like(W)
    for idx in np.ndindex(*W.shape):
        h = h_rel * max(1.0, abs(W[idx]))
        Wp = W.copy(); Wp[idx] += h
        Wm = W.copy(); Wm[idx] -= h
        dW[idx] = (masked_square_loss(Wp, x, m) - masked_square_loss(Wm, x, m)) / (2 * h)
    dx = np.zeros_like(x)
    for idx in np.ndindex(*x.shape):
        h = h_rel * max(1.0, abs(x[idx]))
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        dx[idx] = (masked_square_loss(W, xp, m) - masked_square_loss(W, xm, m)) / (2 * h)
    return dx, dW
