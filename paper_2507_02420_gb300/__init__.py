"""GB300 (sm_103a) implementation of the fast Generalized Tensor Transform.

y = (W (x) ... (x) W) x for a b x b base matrix W and N = b^n (Def. 2.3 and
Sec. 3 of arXiv 2507.02420), in the paper's natural index ordering.  The
computation runs in hand-written CUDA kernels behind the C ABI of
include/gtt.h (libgtt.so); this package is its thin Python binding.
"""
from .api import (C64, C128, F32, F64, I32, PREC_AUTO, PREC_BF16X2, PREC_BF16X3, PREC_FP32, PREC_TF32X3, Plan,  # noqa: F401
                  dtype_code)
from ._lib import GTTError, LIB_PATH, load  # noqa: F401
from .autograd import GTTFunction, gtt  # noqa: F401
from .api import autotune_cache_load, autotune_cache_save, selftest_bounded_wait  # noqa: F401
from .group import Group  # noqa: F401
from . import params  # noqa: F401
