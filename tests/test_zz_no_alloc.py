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


LIMIT = 1 << 20  # bytes of dW partials the static array holds


def _inputs(b, n, batch, dt, rng):
    if dt in ("c64", "c128"):
        npdt = np.complex64 if dt == "c64" else np.complex128
        W = (gi.haar_unitary(b, rng) + 0.1).astype(npdt)
        x = gi.complex_normal_x((batch, b ** n), rng, npdt)
        dy = gi.complex_normal_x((batch, b ** n), rng, npdt)
    else:
        npdt = np.float32 if dt == "f32" else np.float64
        W = (gi.haar_orthogonal(b, rng) + 0.1).astype(npdt)
        x = gi.normal_x((batch, b ** n), rng, npdt)
        dy = gi.normal_x((batch, b ** n), rng, npdt)
    return W, x, dy


def _noalloc(lib, plan, x, dy, dx, dW):
    return lib.gtt_backward_noalloc(plan._h, x.data_ptr(), dy.data_ptr(), dx.data_ptr(),
                                    None if dW is None else dW.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("b,n,batch,dt", [(8, 6, 4, "f32"), (4, 7, 3, "c64"), (2, 10, 2, "f64"),
                                          (16, 1, 64, "c128")])
def test_noalloc_backward_matches_backward_on_two_calls(g, b, n, batch, dt):
    """Same kernels in the same order as gtt_backward with the same dx, so the
    results are the same bits; run twice so the second call finds the
    previous call's partials in the shared array."""
    from paper_2507_02420_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(6000 + b)
    W, x, dy = _inputs(b, n, batch, dt, rng)
    plan = g.Plan(W, n, dt, batch)
    xd, dyd = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    ref_dx, ref_dW = plan.backward(xd, dyd)
    torch.cuda.synchronize()
    for _ in range(2):
        dx = torch.full_like(xd, 7)
        dW = torch.full((b, b), 7, dtype=xd.dtype, device="cuda")
        st = _noalloc(lib, plan, xd, dyd, dx, dW)
        torch.cuda.synchronize()
        assert st == 0, lib.gtt_last_error()
        assert torch.equal(dx, ref_dx)
        assert torch.equal(dW, ref_dW)
    plan.check()


def test_noalloc_rejects_requests_beyond_its_limits(g):
    from paper_2507_02420_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(6100)
    # three backward passes would need a data-sized checkpoint buffer
    W = gi.haar_unitary(2, rng)
    plan = g.Plan(W, 20, "c128", 1)
    x = torch.zeros(2 ** 20, dtype=torch.complex128, device="cuda")
    dx = torch.zeros_like(x)
    assert _noalloc(lib, plan, x, x, dx, None) == 1
    assert b"backward passes" in lib.gtt_last_error()
    # dx missing, or aliasing dy or x
    W8 = gi.haar_orthogonal(8, rng).astype(np.float32)
    p8 = g.Plan(W8, 4, "f32", 1)
    y = torch.zeros(8 ** 4, dtype=torch.float32, device="cuda")
    y2 = torch.zeros_like(y)
    assert lib.gtt_backward_noalloc(p8._h, y.data_ptr(), y2.data_ptr(), None, None, None) == 1
    assert _noalloc(lib, p8, y, y2, y2, None) == 1
    assert b"dy" in lib.gtt_last_error()
    assert _noalloc(lib, p8, y, y2, y, None) == 1
    assert b"from x" in lib.gtt_last_error()
    # dW partials larger than the static array: b = 16, complex128, two
    # one-digit backward passes with a 4 KiB partial per CTA and a full grid each
    W16 = gi.haar_unitary(16, rng)
    p16 = g.Plan(W16, 2, "c128", 4096)
    z = torch.zeros(4096 * 16 ** 2, dtype=torch.complex128, device="cuda")
    dz = torch.zeros_like(z)
    p16.backward(z, z)  # builds the backward schedule (gtt_backward may allocate)
    torch.cuda.synchronize()
    bwd = p16.describe()["backward"]
    need = sum(p["grid"] for p in bwd) * 16 * 16 * 16
    assert len(bwd) == 2 and need > LIMIT, bwd
    assert _noalloc(lib, p16, z, z, dz, None) == 1
    assert b"static scratch" in lib.gtt_last_error()
