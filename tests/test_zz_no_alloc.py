"""gtt_backward_noalloc: the backward for callers that must not allocate device
memory (for instance under a framework allocator that has reserved the
device, or in loops where cudaMalloc would synchronize the device).  Its dW
scratch is a fixed array in the library's device globals; these tests check
it against gtt_backward through the C ABI, on two calls in a row (the array
keeps the previous call's contents), and that requests beyond its limits are
rejected with an error rather than run.

This file is collected last on purpose, so a failure here leaves every other
test already run."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


def rel(a, ref):
    a, ref = a.cpu().numpy(), ref.cpu().numpy()
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("b,n,batch,dt", [(8, 6, 4, "f32"), (4, 7, 3, "c64"), (2, 10, 2, "f64")])
def test_noalloc_backward_matches_backward_on_two_calls(g, b, n, batch, dt):
    from paper_2507_02420_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(6000 + b)
    if dt == "c64":
        W = (gi.haar_unitary(b, rng) + 0.1).astype(np.complex64)
        x = gi.complex_normal_x((batch, b ** n), rng, np.complex64)
        dy = gi.complex_normal_x((batch, b ** n), rng, np.complex64)
    else:
        npdt = np.float32 if dt == "f32" else np.float64
        W = (gi.haar_orthogonal(b, rng) + 0.1).astype(npdt)
        x = gi.normal_x((batch, b ** n), rng, npdt)
        dy = gi.normal_x((batch, b ** n), rng, npdt)
    plan = g.Plan(W, n, dt, batch)
    xd, dyd = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    ref_dx, ref_dW = plan.backward(xd, dyd)
    torch.cuda.synchronize()
    tol_dx, tol_dW = (1e-12, 1e-12) if dt == "f64" else (1e-5, 1e-4)
    for _ in range(2):
        dx = torch.full_like(xd, 7)
        dW = torch.full((b, b), 7, dtype=xd.dtype, device="cuda")
        st = lib.gtt_backward_noalloc(plan._h, xd.data_ptr(), dyd.data_ptr(), dx.data_ptr(),
                                      dW.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert st == 0, lib.gtt_last_error()
        assert rel(dx, ref_dx) <= tol_dx
        assert rel(dW, ref_dW) <= tol_dW


def test_noalloc_rejects_requests_beyond_its_limits(g):
    from paper_2507_02420_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(6100)
    # three backward passes would need a data-sized checkpoint buffer
    W = gi.haar_unitary(2, rng)
    plan = g.Plan(W, 20, "c128", 1)
    x = torch.zeros(2 ** 20, dtype=torch.complex128, device="cuda")
    dx = torch.zeros_like(x)
    assert lib.gtt_backward_noalloc(plan._h, x.data_ptr(), x.data_ptr(), dx.data_ptr(), None, None) == 1
    assert b"backward passes" in lib.gtt_last_error()
    # dx missing, or aliasing dy
    W8 = gi.haar_orthogonal(8, rng).astype(np.float32)
    p8 = g.Plan(W8, 4, "f32", 1)
    y = torch.zeros(8 ** 4, dtype=torch.float32, device="cuda")
    assert lib.gtt_backward_noalloc(p8._h, y.data_ptr(), y.data_ptr(), None, None, None) == 1
    assert lib.gtt_backward_noalloc(p8._h, y.data_ptr(), y.data_ptr(), y.data_ptr(), None, None) == 1
    # dW partials larger than the static array (b = 16, complex128, many CTAs)
    W16 = gi.haar_unitary(16, rng)
    p16 = g.Plan(W16, 5, "c128", 4)
    z = torch.zeros(4 * 16 ** 5, dtype=torch.complex128, device="cuda")
    dz = torch.zeros_like(z)
    st = lib.gtt_backward_noalloc(p16._h, z.data_ptr(), z.data_ptr(), dz.data_ptr(), None, None)
    if st == 1:
        assert b"static scratch" in lib.gtt_last_error() or b"backward passes" in lib.gtt_last_error()
    else:  # this device's occupancy kept the partials within the array
        assert st == 0
