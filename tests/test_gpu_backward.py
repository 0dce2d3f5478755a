"""GPU parity of gtt_backward (dx, dW) and the autograd wrapper against the
FP64 oracle gradient, which is itself pinned to finite differences."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu

DT = {"f64": (np.float64, False), "f32": (np.float32, False), "c64": (np.complex64, True),
      "c128": (np.complex128, True)}
TOL_DX = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-5, "c64": 1e-5}
TOL_DW = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-4, "c64": 1e-4}


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


def up(a):
    a = np.asarray(a)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def rel(a, ref):
    return float(np.linalg.norm(up(a) - ref) / max(np.linalg.norm(ref), 1e-300))


def inputs(b, n, batch, dt, rng, unitary=False):
    npdt, cplx = DT[dt]
    if cplx:
        W = gi.haar_unitary(b, rng)
        if not unitary:
            W = W + 0.2 * (rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b)))
        x = gi.complex_normal_x((batch, b ** n), rng, npdt)
        dy = gi.complex_normal_x((batch, b ** n), rng, npdt)
    else:
        W = gi.haar_orthogonal(b, rng)
        if not unitary:
            W = W + 0.2 * rng.standard_normal((b, b))
        x = gi.normal_x((batch, b ** n), rng, npdt)
        dy = gi.normal_x((batch, b ** n), rng, npdt)
    return W.astype(npdt), x, dy


def run_bwd(g, W, x, dy, n, dt, need_dx=True, need_dW=True):
    plan = g.Plan(W, n, dt, x.shape[0])
    dx, dW = plan.backward(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(),
                           need_dx=need_dx, need_dW=need_dW)
    torch.cuda.synchronize()
    return (dx.cpu().numpy() if dx is not None else None,
            dW.cpu().numpy() if dW is not None else None, plan)


def n_for(b, lim=12):
    n = 1
    while b ** (n + 1) <= 2 ** lim:
        n += 1
    return n


@pytest.mark.parametrize("dt", ["f64", "f32", "c64", "c128"])
@pytest.mark.parametrize("b", [2, 3, 4, 5, 7, 8, 12, 16])
def test_backward_matches_oracle_gradient(g, dt, b):
    rng = np.random.default_rng(5000 + b)
    n = n_for(b)
    W, x, dy = inputs(b, n, 2, dt, rng)
    dx, dW, _ = run_bwd(g, W, x, dy, n, dt)
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    assert rel(dx, rdx) <= TOL_DX[dt], rel(dx, rdx)
    assert rel(dW, rdW) <= TOL_DW[dt], rel(dW, rdW)


def test_b8_n7_batch32_training_step_full_size(g):
    """b=8, n=7, batch 32, FP32, trainable W (Haar-orthogonal init), loss
    sum(m * y^2): dx (rel-L2 <= 1e-5) and dW (Frobenius <= 1e-4) vs the oracle."""
    W, x = gi.workload_inputs("b8_n7_batch32_f32")
    m = gi.train_mask()
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    mt = torch.from_numpy(m).cuda()
    y = g.gtt(xt, Wt, 7)
    loss = (mt * y * y).sum()
    loss.backward()
    torch.cuda.synchronize()
    yo = oracle.modes(up(W), up(x))
    rdx, rdW = oracle.grad(up(W), up(x), 2 * up(m) * yo)
    assert rel(y.detach().cpu().numpy(), yo) <= 1e-5
    edx, edW = rel(xt.grad.cpu().numpy(), rdx), rel(Wt.grad.cpu().numpy(), rdW)
    print("b8_n7 training step: dx rel-L2", edx, "dW rel-Frobenius", edW)
    assert edx <= 1e-5
    assert edW <= 1e-4


@pytest.mark.parametrize("n,batch", [(4, 3), (5, 3), (6, 3), (7, 1), (8, 1)])
def test_b8_f32_tile_kernel_matches_oracle_gradient(g, n, batch):
    """FP32, b = 8 runs the fixed-tile backward kernel: passes of digits 0-3,
    then at most 3 digits on runs of 8^(4-g) elements (n = 5: [4, 1], 6:
    [4, 2], 7: [4, 3], 8: [4, 3, 1] with checkpoints).  dx and dW against the
    oracle gradient; dx aliasing dy through the raw ABI at n = 6."""
    rng = np.random.default_rng(5050 + n)
    W, x, dy = inputs(8, n, batch, "f32", rng)
    dx, dW, plan = run_bwd(g, W, x, dy, n, "f32")
    names = [k["kernel"] for k in plan.describe().get("backward", [])]
    assert names and all("gtt_backward_b8_kernel" in nm for nm in names), names
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    assert rel(dx, rdx) <= TOL_DX["f32"], rel(dx, rdx)
    assert rel(dW, rdW) <= TOL_DW["f32"], rel(dW, rdW)
    if n == 6:
        from paper_2507_02420_gb300 import _lib
        xd, dyd = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
        dWd = torch.empty((8, 8), dtype=xd.dtype, device="cuda")
        st = _lib.load().gtt_backward(plan._h, xd.data_ptr(), dyd.data_ptr(), dyd.data_ptr(), dWd.data_ptr(), None)
        torch.cuda.synchronize()
        assert st == 0
        assert rel(dyd.cpu().numpy(), rdx) <= TOL_DX["f32"] and rel(dWd.cpu().numpy(), rdW) <= TOL_DW["f32"]


@pytest.mark.parametrize("n,batch", [(5, 3), (6, 2), (7, 1)])
def test_forward_saving_and_backward_saved(g, n, batch):
    """gtt_forward_saving keeps the backward's checkpoint; gtt_backward_saved
    then runs the backward passes only.  y, dx and dW are bitwise equal to
    gtt_forward + gtt_backward (the same kernels compute the checkpoint), and
    dx and dW match the oracle gradient."""
    rng = np.random.default_rng(5400 + n)
    W, x, dy = inputs(8, n, batch, "f32", rng)
    plan = g.Plan(W, n, "f32", batch)
    xd, dyd = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    y0 = plan.forward(xd)
    dx0, dW0 = plan.backward(xd, dyd)
    y1, ck = plan.forward_saving(xd)
    dx1, dW1 = plan.backward_saved(xd, ck, dyd)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(y0, y1) and torch.equal(dx0, dx1) and torch.equal(dW0, dW1)
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    assert rel(dx1.cpu().numpy(), rdx) <= TOL_DX["f32"] and rel(dW1.cpu().numpy(), rdW) <= TOL_DW["f32"]
    # dx may alias the checkpoint
    dWd = torch.empty((8, 8), device="cuda")
    from paper_2507_02420_gb300 import _lib
    st = _lib.load().gtt_backward_saved(plan._h, xd.data_ptr(), ck.data_ptr(), dyd.data_ptr(), ck.data_ptr(),
                                        dWd.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0 and torch.equal(ck, dx0) and torch.equal(dWd, dW0)


@pytest.mark.parametrize("b,n,dt", [(16, 4, "f32"), (16, 5, "f32"), (4, 8, "c64"), (2, 14, "f32"), (3, 9, "c128"),
                                    (5, 7, "f64")])
def test_forward_saving_other_shapes(g, b, n, dt):
    """Wherever gtt_forward_saving accepts a plan (the b = 16 tensor-core
    schedule included), y is bitwise the plain forward's and the saved
    backward matches the oracle gradient; elsewhere it is rejected with
    GTT_ERR_UNSUPPORTED and launches nothing."""
    rng = np.random.default_rng(5600 + b + n)
    W, x, dy = inputs(b, n, 2, dt, rng)
    plan = g.Plan(W, n, dt, 2)
    xd, dyd = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    y0 = plan.forward(xd)
    try:
        y1, ck = plan.forward_saving(xd)
    except g.GTTError as e:
        assert e.status == 2
        return
    dx, dW = plan.backward_saved(xd, ck, dyd)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(y0, y1)
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    assert rel(dx.cpu().numpy(), rdx) <= TOL_DX[dt] and rel(dW.cpu().numpy(), rdW) <= TOL_DW[dt]


@pytest.mark.parametrize("b,n,dt", [(8, 4, "f32"), (8, 8, "f32"), (2, 6, "f64")])
def test_forward_saving_unsupported_shapes(g, b, n, dt):
    """One-pass or three-pass backward schedules keep no checkpoint:
    GTT_ERR_UNSUPPORTED, and the autograd wrapper falls back to the plain
    calls (its gradient still matches the oracle)."""
    rng = np.random.default_rng(5500 + b + n)
    W, x, dy = inputs(b, n, 1, dt, rng)
    plan = g.Plan(W, n, dt, 1)
    with pytest.raises(g.GTTError) as ei:
        plan.forward_saving(torch.from_numpy(x).cuda())
    assert ei.value.status == 2
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    (g.gtt(xt, Wt, n) * torch.from_numpy(dy).cuda()).sum().backward()
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    assert rel(xt.grad.cpu().numpy(), rdx) <= TOL_DX[dt] and rel(Wt.grad.cpu().numpy(), rdW) <= TOL_DW[dt]


def test_three_pass_backward_uses_checkpoint_recompute(g):
    """A transform needing >= 3 backward passes (checkpoints recomputed)."""
    rng = np.random.default_rng(5100)
    W, x, dy = inputs(2, 20, 1, "c128", rng)
    dx, dW, plan = run_bwd(g, W, x, dy, 20, "c128")
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    assert rel(dx, rdx) <= 1e-12 and rel(dW, rdW) <= 1e-12


@pytest.mark.parametrize("dt", ["f32", "c64"])
def test_optional_outputs_and_aliasing(g, dt):
    rng = np.random.default_rng(5200)
    W, x, dy = inputs(4, 9, 3, dt, rng)
    rdx, rdW = oracle.grad(up(W), up(x), up(dy))
    dx, dW, _ = run_bwd(g, W, x, dy, 9, dt, need_dx=False)
    assert dx is None and rel(dW, rdW) <= TOL_DW[dt]
    dx, dW, _ = run_bwd(g, W, x, dy, 9, dt, need_dW=False)
    assert dW is None and rel(dx, rdx) <= TOL_DX[dt]
    # dx aliasing dy (through the raw ABI)
    plan = g.Plan(W, 9, dt, 3)
    from paper_2507_02420_gb300 import _lib
    xd = torch.from_numpy(x).cuda()
    dyd = torch.from_numpy(dy).cuda()
    dWd = torch.empty((4, 4), dtype=xd.dtype, device="cuda")
    st = _lib.load().gtt_backward(plan._h, xd.data_ptr(), dyd.data_ptr(), dyd.data_ptr(),
                                  dWd.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0
    assert rel(dyd.cpu().numpy(), rdx) <= TOL_DX[dt]
    assert rel(dWd.cpu().numpy(), rdW) <= TOL_DW[dt]


def test_backward_is_bitwise_repeatable(g):
    rng = np.random.default_rng(5300)
    W, x, dy = inputs(8, 6, 4, "f32", rng)
    a = run_bwd(g, W, x, dy, 6, "f32")
    b = run_bwd(g, W, x, dy, 6, "f32")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_integer_backward_unsupported(g):
    plan = g.Plan(np.array([[1, 1], [1, -1]], dtype=np.int32), 4, "i32", 1)
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GTTError) as ei:
        plan.backward(x, x)
    assert ei.value.status == 2


@pytest.mark.parametrize("dt", [torch.float64, torch.complex128])
def test_autograd_gradcheck(g, dt):
    torch.manual_seed(0)
    W = torch.randn(3, 3, dtype=dt, device="cuda", requires_grad=True)
    x = torch.randn(2, 27, dtype=dt, device="cuda", requires_grad=True)
    # gradcheck perturbs W through W.data, which bypasses the version counter
    # the wrapper's W cache relies on; a fresh tensor per call is seen
    assert torch.autograd.gradcheck(lambda a, w: g.gtt(a, w.clone(), 3), (x, W), eps=1e-6, atol=1e-7)


def test_autograd_unchanged_w_does_not_sync(g):
    """Forward + backward steps with an unchanged W run without a
    device-to-host copy or a device wait (torch's sync debug mode raises on
    either); an optimizer-style in-place update of W is picked up."""
    from paper_2507_02420_gb300 import autograd as ag
    rng = np.random.default_rng(7)
    W0 = gi.haar_orthogonal(8, rng).astype(np.float32)
    W = torch.tensor(W0, device="cuda", requires_grad=True)
    x = torch.randn(3, 8 ** 4, device="cuda", requires_grad=True)
    g.gtt(x, W, 4).sum().backward()  # builds and caches the plan
    torch.cuda.synchronize()
    try:
        torch.cuda.set_sync_debug_mode("error")
        for _ in range(3):
            y = g.gtt(x, W, 4)
            (y * y).sum().backward()
    finally:
        torch.cuda.set_sync_debug_mode("default")
    with torch.no_grad():
        W.mul_(0.5)  # bumps W's version: the next forward uploads the new values
    y = g.gtt(x, W, 4)
    ref = oracle.modes(W0.astype(np.float64) * 0.5, x.detach().cpu().numpy().astype(np.float64))
    assert np.linalg.norm(y.detach().cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    assert len(ag._cache) >= 1
