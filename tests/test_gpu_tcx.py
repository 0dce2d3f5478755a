"""complex64, b = 4 on the tensor cores (GTT_PREC_TF32X3, opt-in): pairs of base-4
digits as one base-16 digit with W (x) W (Def. 2.3), TF32 products of 2-piece
splits, thread-block clusters exchanging one digit through distributed shared
memory.  Parity against the FP64 oracle at the stated tolerance (1e-5 for
complex64 forward, 2e-5 for inverse(forward)), and against the FP32 CUDA-core
path of the same plan."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu

TOL_FWD, TOL_RT = 1e-5, 2e-5


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


def rel(a, ref):
    a = np.asarray(a).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def inputs(n, batch, seed, unitary=True):
    rng = np.random.default_rng(seed)
    W = gi.haar_unitary(4, rng)
    if not unitary:
        W = W + 0.3 * (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    x = gi.complex_normal_x((batch, 4 ** n), rng, np.complex64)
    return W.astype(np.complex64), x


@pytest.mark.parametrize("n,batch", [(7, 1), (7, 5), (13, 1), (13, 2)])
def test_tf32x3_matches_oracle(g, n, batch):
    W, x = inputs(n, batch, 9000 + 10 * n + batch)
    plan = g.Plan(W, n, "c64", batch)
    assert plan.describe()["precision"] == "fp32"   # AUTO keeps the faster FP32 path
    plan.set_precision(g.PREC_TF32X3)
    d = plan.describe()
    assert d["precision"] == "tf32x3"
    assert len(d["passes"]) == (n - 7) // 6 + 1 and all("gtt_tcx_pass_kernel" in p["kernel"] for p in d["passes"])
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    plan.check()
    ref = oracle.modes(W.astype(np.complex128), x.astype(np.complex128))
    e_f, e_rt = rel(y.cpu().numpy(), ref), rel(xr.cpu().numpy(), x)
    print(f"tf32x3 n={n} batch={batch}: forward rel-L2 {e_f:.3e}, inverse(forward) {e_rt:.3e}")
    assert e_f <= TOL_FWD and e_rt <= TOL_RT


def test_tf32x3_general_w_and_adjoint(g):
    """A non-unitary W (the adjoint is then not the inverse): forward and the
    adjoint transform each against the oracle's."""
    W, x = inputs(7, 3, 9100, unitary=False)
    plan = g.Plan(W, 7, "c64", 3)
    plan.set_precision(g.PREC_TF32X3)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd).cpu().numpy()
    z = plan.inverse(xd).cpu().numpy()
    W64 = W.astype(np.complex128)
    assert rel(y, oracle.modes(W64, x.astype(np.complex128))) <= TOL_FWD
    assert rel(z, oracle.adjoint(W64, x.astype(np.complex128))) <= TOL_FWD


def test_tf32x3_in_place_and_against_fp32_path(g):
    W, x = inputs(13, 1, 9200)
    plan = g.Plan(W, 13, "c64", 1)
    plan.set_precision(g.PREC_TF32X3)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    z = xd.clone()
    plan.forward(z, out=z)            # in place
    torch.cuda.synchronize()
    assert torch.equal(y, z)
    plan.set_precision(g.PREC_FP32)
    assert plan.describe()["precision"] == "fp32"
    y32 = plan.forward(xd)
    assert rel(y.cpu().numpy(), y32.cpu().numpy()) <= TOL_FWD
    plan.set_precision(g.PREC_TF32X3)
    assert torch.equal(plan.forward(xd), y)


def test_tf32x3_set_w(g):
    W, x = inputs(7, 2, 9300)
    W2, _ = inputs(7, 1, 9301)
    plan = g.Plan(W, 7, "c64", 2)
    plan.set_precision(g.PREC_TF32X3)
    plan.set_w(W2)
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, oracle.modes(W2.astype(np.complex128), x.astype(np.complex128))) <= TOL_FWD


@pytest.mark.parametrize("b,n,dt", [(4, 8, "c64"), (4, 12, "c64"), (4, 7, "f32"), (2, 14, "c64"), (4, 7, "c128")])
def test_tf32x3_rejects_other_shapes(g, b, n, dt):
    rng = np.random.default_rng(9400)
    W = gi.haar_unitary(b, rng) if dt.startswith("c") else gi.haar_orthogonal(b, rng)
    plan = g.Plan(W, n, dt, 1)
    assert plan.describe()["precision"] != "tf32x3"
    with pytest.raises(g.GTTError) as ei:
        plan.set_precision(g.PREC_TF32X3)
    assert ei.value.status == 2
