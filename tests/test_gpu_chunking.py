"""L2-resident chunked execution (gtt_plan_set_chunking): the launch order
changes, the result does not (bitwise), for the CUDA-core, TMA and
tensor-core pass kernels, with chunks of whole batch items and with chunks of
blocks inside an item (the leading passes chunked, the rest run after)."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


@pytest.mark.parametrize("b,n,batch,dt,prec,tma", [
    (16, 4, 7, "f32", "fp32", False), (16, 4, 7, "f32", "fp32", True), (16, 4, 7, "f32", "bf16x3", True),
    (8, 5, 5, "f32", "fp32", True), (4, 7, 6, "c64", "fp32", True), (3, 7, 5, "c64", "fp32", False)])
@pytest.mark.parametrize("chunk", ["item1", "item2", "item3", "block", "block3"])
def test_chunked_passes_are_bitwise_identical(g, b, n, batch, dt, prec, tma, chunk):
    rng = np.random.default_rng(9500 + b + len(chunk))
    if dt == "c64":
        W = gi.haar_unitary(b, rng).astype(np.complex64)
        x = gi.complex_normal_x((batch, b ** n), rng, np.complex64)
    else:
        W = gi.haar_orthogonal(b, rng).astype(np.float32)
        x = gi.normal_x((batch, b ** n), rng, np.float32)
    plan = g.Plan(W, n, dt, batch)
    plan.set_precision(g.PREC_BF16X3 if prec == "bf16x3" else g.PREC_FP32)
    plan.set_pipeline(tma, 2)
    xd = torch.from_numpy(x).cuda()
    passes = plan.describe()["passes"]
    if not chunk.startswith("item") and len(passes) < 2:
        plan.set_passes([n // 2, n - n // 2], [1, 1])  # two passes, so a prefix can be chunked
        passes = plan.describe()["passes"]
    ref = plan.forward(xd).cpu().numpy()
    if chunk.startswith("item"):
        elems = int(chunk[4:]) * b ** n
    else:
        # blocks of b^s elements, s = the top digit of the first two passes
        s = max(p["m0"] + p["g"] for p in passes[:2])
        elems = (3 if chunk == "block3" else 1) * b ** s
    plan.set_chunking(elems)
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    plan.check()
    np.testing.assert_array_equal(y.cpu().numpy(), ref)
    up = (lambda a: a.astype(np.complex128)) if dt == "c64" else (lambda a: a.astype(np.float64))
    o = oracle.modes(up(W), up(x))
    assert np.linalg.norm(up(ref) - o) / np.linalg.norm(o) <= 2e-6
    assert np.linalg.norm(up(xr.cpu().numpy()) - up(x)) / np.linalg.norm(up(x)) <= 4e-6


def test_automatic_chunking_choice(g):
    W, _ = gi.workload_inputs("b16_n6_batch64_f32")
    plan = g.Plan(W, 6, "f32", 64)
    plan.set_chunking(-1)   # 4 GiB: 48 MiB chunks of the first two passes
    small = g.Plan(W, 4, "f32", 2)
    small.set_chunking(-1)  # fits L2 already: stays off
    # (the choice is internal; both must still compute the transform)
    x = torch.randn(2, 16 ** 4, device="cuda")
    y = small.forward(x)
    torch.cuda.synchronize()
    ref = oracle.modes(W.astype(np.float64), x.cpu().numpy().astype(np.float64))
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-6
