"""Seeded synthetic inputs for the Generalized Tensor Transform workloads.

This module only draws random numbers and describes workload shapes.  It holds
none of the transform's arithmetic, so both the FP64 oracle (``oracle/``) and
the CUDA library's tests and benchmark can take their inputs from here without
sharing any code with each other.

Workloads (all synthetic; the paper uses no public dataset):

* ``b2_n12_f64`` -- b=2, n=12, batch 1, FP64; W = [[1,1],[1,-1]]/sqrt(2) (the
  normalised Hadamard base matrix of Sec. 2.3, b=2 case), x ~ U[-1, 1].
* ``b4_n13_c64`` -- b=4, n=13, batch 1, complex64; W Haar-random 4x4 unitary,
  x ~ CN(0, 1) (re, im ~ N(0, 1/2)).
* ``b16_n6_batch64_f32`` -- b=16, n=6, batch 64, FP32; W Haar-random 16x16 orthogonal,
  x ~ N(0, 1).
* ``b8_n7_batch32_f32`` -- b=8, n=7, batch 32, FP32; W Haar-random 8x8 orthogonal
  (trainable), x ~ N(0, 1), mask m ~ U[0, 1] with y's shape.
* ``grouped_1000_uneven`` -- 1000 requests, b uniform on {2,3,4,5,8,16}, N log-uniform in
  [2^10, 2^22], dtype 50/50 FP32 / complex64, W Haar per request.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "haar_unitary", "haar_orthogonal", "hadamard_w", "u3",
    "uniform_x", "normal_x", "complex_normal_x", "uniform_mask",
    "Request", "grouped_requests", "WORKLOADS", "workload_inputs", "train_mask",
]


def haar_unitary(b: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed b x b unitary (complex128).

    QR of a complex Gaussian matrix (A + iB)/sqrt(2), with the phase of R's
    diagonal moved into Q (Q <- Q diag(r_ii/|r_ii|)) so the distribution is
    exactly Haar.
    """
    z = (rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def haar_orthogonal(b: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed b x b real orthogonal matrix (float64), sign-fixed QR."""
    z = rng.standard_normal((b, b))
    q, r = np.linalg.qr(z)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def hadamard_w(normalised: bool = True) -> np.ndarray:
    """The 2x2 Hadamard base matrix; [[1,1],[1,-1]] (times 1/sqrt(2) if normalised)."""
    h = np.array([[1.0, 1.0], [1.0, -1.0]])
    return h / math.sqrt(2.0) if normalised else h


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    """The U3(theta, phi, lambda) parameterisation of a 2x2 unitary (Eq. U3)."""
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def uniform_x(shape, rng: np.random.Generator, lo: float = -1.0, hi: float = 1.0,
              dtype=np.float64) -> np.ndarray:
    return rng.uniform(lo, hi, size=shape).astype(dtype)


def normal_x(shape, rng: np.random.Generator, dtype=np.float32) -> np.ndarray:
    if np.dtype(dtype) == np.float32:
        return rng.standard_normal(size=shape, dtype=np.float32)
    return rng.standard_normal(size=shape).astype(dtype)


def complex_normal_x(shape, rng: np.random.Generator, dtype=np.complex64) -> np.ndarray:
    """Circular complex Gaussian CN(0, 1): re, im ~ N(0, 1/2)."""
    scale = 1.0 / math.sqrt(2.0)
    shape = tuple(np.atleast_1d(shape))
    if np.dtype(dtype) == np.complex64:
        # interleaved (re, im) pairs drawn in one sequential stream
        ri = rng.standard_normal(size=shape + (2,), dtype=np.float32)
        ri *= np.float32(scale)
        return ri.view(np.complex64).reshape(shape)
    ri = rng.standard_normal(size=shape + (2,)) * scale
    return ri.view(np.complex128).reshape(shape).astype(dtype)


def uniform_mask(shape, rng: np.random.Generator, dtype=np.float32) -> np.ndarray:
    return rng.uniform(0.0, 1.0, size=shape).astype(dtype)


@dataclass(frozen=True)
class Request:
    """One transform of a grouped (uneven) batch."""
    b: int
    n: int
    dtype: str          # "f32" or "c64"
    seed: int           # seed of this request's own W and x

    @property
    def N(self) -> int:
        return self.b ** self.n


# n range per b so that 2^10 <= b^n <= 2^22.
def _n_range(b: int) -> tuple[int, int]:
    lb = math.log2(b)
    return math.ceil(10.0 / lb - 1e-12), math.floor(22.0 / lb + 1e-12)


def grouped_requests(count: int = 1000, seed: int = 4,
                     bases=(2, 3, 4, 5, 8, 16)) -> list[Request]:
    """The uneven grouped workload: b uniform on `bases`, N log-uniform in
    [2^10, 2^22] (u ~ U(10, 22), n = clamp(round(u / log2 b))), dtype by a
    fair coin between FP32 and complex64."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        b = int(rng.choice(bases))
        u = rng.uniform(10.0, 22.0)
        lo, hi = _n_range(b)
        n = int(min(max(round(u / math.log2(b)), lo), hi))
        dt = "c64" if rng.random() < 0.5 else "f32"
        out.append(Request(b=b, n=n, dtype=dt, seed=int(rng.integers(0, 2**31 - 1))))
    return out


def request_inputs(req: Request):
    """(W, x) for one grouped request: Haar W (unitary for c64, orthogonal for
    f32) and x ~ N(0,1) / CN(0,1), from the request's own seed."""
    rng = np.random.default_rng(req.seed)
    if req.dtype == "c64":
        w = haar_unitary(req.b, rng).astype(np.complex64)
        x = complex_normal_x((req.N,), rng, np.complex64)
    else:
        w = haar_orthogonal(req.b, rng).astype(np.float32)
        x = normal_x((req.N,), rng, np.float32)
    return w, x


WORKLOADS = {
    "b2_n12_f64": dict(b=2, n=12, batch=1, dtype="f64", seed=0),
    "b4_n13_c64": dict(b=4, n=13, batch=1, dtype="c64", seed=1),
    "b16_n6_batch64_f32": dict(b=16, n=6, batch=64, dtype="f32", seed=2),
    "b8_n7_batch32_f32": dict(b=8, n=7, batch=32, dtype="f32", seed=3),
    "grouped_1000_uneven": dict(seed=4, count=1000),
}


def workload_inputs(name: str, batch: int | None = None):
    """(W, x) of a single-transform workload (x has shape [batch, N]).  `batch`
    may shrink the batch for a sampled run; the first items are identical to
    the full run's."""
    c = WORKLOADS[name]
    if "b" not in c:
        raise ValueError(f"{name} is a request list; use grouped_requests()")
    rng = np.random.default_rng(c["seed"])
    bsz = c["batch"] if batch is None else batch
    N = c["b"] ** c["n"]
    if name == "b2_n12_f64":
        w = hadamard_w(True)
        x = uniform_x((bsz, N), rng, dtype=np.float64)
    elif name == "b4_n13_c64":
        w = haar_unitary(4, rng).astype(np.complex64)
        x = complex_normal_x((bsz, N), rng, np.complex64)
    elif name == "b16_n6_batch64_f32":
        w = haar_orthogonal(16, rng).astype(np.float32)
        x = normal_x((bsz, N), rng, np.float32)
    else:  # b8_n7_batch32_f32
        w = haar_orthogonal(8, rng).astype(np.float32)
        x = normal_x((bsz, N), rng, np.float32)
    return w, x


def train_mask(batch: int | None = None):
    """The loss mask m ~ U[0, 1] of the b8_n7_batch32_f32 training step (its own
    stream, seeded from the workload's seed)."""
    c = WORKLOADS["b8_n7_batch32_f32"]
    rng = np.random.default_rng(c["seed"] + 1000)
    bsz = c["batch"] if batch is None else batch
    return uniform_mask((bsz, c["b"] ** c["n"]), rng)


def function_encoding_signal(n: int) -> np.ndarray:
    """The test signal of the function-encoding example (Sec. 4.2): a
    degree-7 polynomial with small sinusoidal and exponential terms on [0, 1],
    sampled at the midpoints of N = 2^n subintervals and normalised."""
    N = 2 ** n
    t = (np.arange(N) + 0.5) / N
    coef = [-978.7, 3677.0, -5575.0, 4366.0, -1875.0, 431.6, -47.57, 1.886]  # x^7 .. x^0
    f = np.polyval(coef, t) + 0.1 * np.sin(0.1 * t) - 0.01 * np.exp(-t)
    return f / np.linalg.norm(f)
