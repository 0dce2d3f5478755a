"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every symbol include/gtt.h declares; argument validation rejects bad
requests before touching CUDA; the oracle and the CUDA path share no code."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gtt_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2507_02420_gb300 import build
    build.build()
    from paper_2507_02420_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("gtt_plan_create", "gtt_forward", "gtt_inverse", "gtt_backward",
                     "gtt_plan_destroy", "gtt_last_error", "gtt_plan_set_precision"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, f"libgtt.so lacks {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2507_02420_gb300 import _lib
    assert set(header_functions()) <= set(_lib.SIGNATURES), \
        set(header_functions()) - set(_lib.SIGNATURES)


@pytest.mark.parametrize("b,n,batch,dtype", [(1, 4, 1, 1), (17, 2, 1, 1), (2, 0, 1, 1),
                                             (2, 4, 0, 1), (2, 4, 1, 9), (2, 37, 1, 1),
                                             (16, 10, 1 << 10, 1)])
def test_plan_create_rejects_invalid_arguments(lib, b, n, batch, dtype):
    W = np.eye(max(b, 1), dtype=np.float32)
    h = ctypes.c_void_p()
    st = lib.gtt_plan_create(ctypes.byref(h), b, n, W.ctypes.data_as(ctypes.c_void_p), dtype, batch)
    assert st == 1  # GTT_ERR_INVALID_ARG
    assert h.value is None
    assert lib.gtt_last_error().decode()


def test_null_arguments_are_errors_not_crashes(lib):
    h = ctypes.c_void_p()
    assert lib.gtt_plan_create(None, 2, 3, None, 1, 1) == 1
    assert lib.gtt_plan_create(ctypes.byref(h), 2, 3, None, 1, 1) == 1
    assert lib.gtt_forward(None, None, None, None) == 1
    assert lib.gtt_inverse(None, None, None, None) == 1
    assert lib.gtt_backward(None, None, None, None, None, None) == 1
    assert lib.gtt_plan_destroy(None) == 0


def test_oracle_and_cuda_path_share_no_code():
    """The two sides import/include nothing of each other."""
    for f in glob.glob(os.path.join(ROOT, "paper_2507_02420_gb300", "**", "*"), recursive=True):
        if os.path.isfile(f) and f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
            assert "gtt_oracle" not in text, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".c", ".h")):
            text = open(f).read()
            assert "paper_2507_02420_gb300" not in text, f
            assert "gtt.h" not in text, f


def test_fastdiv_method_is_exact():
    """The invariant-divisor method the kernels use for index arithmetic
    (Granlund and Montgomery 1994, round-up variant) is exact on 32-bit inputs
    for the divisors that occur (powers of b)."""
    rng = np.random.default_rng(5)
    for b in range(2, 17):
        d = 1
        while d < 2 ** 31:
            if d > 1:
                l = (d - 1).bit_length()
                m = ((1 << 32) * ((1 << l) - d)) // d + 1
                assert m < (1 << 32)
                ns = np.concatenate([rng.integers(0, 2 ** 32, 2000, dtype=np.uint64),
                                     np.array([0, 1, d - 1, d, d + 1, 2 ** 32 - 1], dtype=np.uint64)])
                t = (np.uint64(m) * ns) >> np.uint64(32)
                q = (t + ((ns - t) >> np.uint64(1))) >> np.uint64(l - 1)
                assert np.array_equal(q, ns // np.uint64(d)), (b, d)
            d *= b
