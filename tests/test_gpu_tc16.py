"""GPU parity of the b = 16 tensor-core path (BF16x3 splits, FP32 accumulate in
tensor memory) against the FP64 oracle, and against the FP32 CUDA-core path."""
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


def rel(a, ref):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n,batch", [(3, 4), (4, 3), (5, 2), (6, 1)])
def test_bf16x3_matches_oracle(g, n, batch):
    rng = np.random.default_rng(9000 + n)
    W = gi.haar_orthogonal(16, rng).astype(np.float32)
    x = gi.normal_x((batch, 16 ** n), rng, np.float32)
    plan = g.Plan(W, n, "f32", batch)
    plan.set_precision(g.PREC_BF16X3)
    d = plan.describe()
    assert all("tc16" in p["kernel"] for p in d["passes"]), d
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    plan.check()
    ref = oracle.modes(W.astype(np.float64), x.astype(np.float64))
    e = rel(y.cpu().numpy(), ref)
    print(f"bf16x3 b=16 n={n}: forward rel-L2 {e:.3e}")
    assert e <= 1e-6
    assert rel(xr.cpu().numpy(), x.astype(np.float64)) <= 2e-6


def test_bf16x3_non_orthogonal_w_and_inverse_is_adjoint(g):
    rng = np.random.default_rng(9100)
    W = (rng.standard_normal((16, 16)) * 0.3).astype(np.float32)
    x = gi.normal_x((2, 16 ** 4), rng, np.float32)
    plan = g.Plan(W, 4, "f32", 2)
    plan.set_precision(g.PREC_BF16X3)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    z = plan.inverse(y)
    torch.cuda.synchronize()
    ref = oracle.modes(W.astype(np.float64), x.astype(np.float64))
    assert rel(y.cpu().numpy(), ref) <= 1e-6
    assert rel(z.cpu().numpy(), oracle.adjoint(W.astype(np.float64), ref)) <= 1e-6


def test_b16_n6_batch64_bf16x3_full_size_sampled(g):
    """b=16, n=6, batch 64: BF16x3 tensor-core path, items 0, 21, 42, 63 vs the
    oracle at rel-L2 <= 1e-6; the FP32 CUDA-core path on the same input too."""
    W, x = gi.workload_inputs("b16_n6_batch64_f32")
    plan = g.Plan(W, 6, "f32", 64)
    plan.set_precision(g.PREC_BF16X3)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    torch.cuda.synchronize()
    plan.check()
    plan32 = g.Plan(W, 6, "f32", 64)
    plan32.set_precision(g.PREC_FP32)
    y32 = plan32.forward(xd)
    torch.cuda.synchronize()
    for item in (0, 21, 42, 63):
        ref = oracle.modes(W.astype(np.float64), x[item].astype(np.float64))
        e_tc, e_32 = rel(y[item].cpu().numpy(), ref), rel(y32[item].cpu().numpy(), ref)
        print(f"item {item}: bf16x3 rel-L2 {e_tc:.3e}, fp32 rel-L2 {e_32:.3e}")
        assert e_tc <= 1e-6 and e_32 <= 1e-6


def test_bf16x3_repeatable_and_switchable(g):
    rng = np.random.default_rng(9200)
    W = gi.haar_orthogonal(16, rng).astype(np.float32)
    x = gi.normal_x((3, 16 ** 4), rng, np.float32)
    plan = g.Plan(W, 4, "f32", 3)
    xd = torch.from_numpy(x).cuda()
    plan.set_precision(g.PREC_BF16X3)
    a = plan.forward(xd).cpu().numpy()
    b = plan.forward(xd).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    plan.set_precision(g.PREC_FP32)
    assert not any("tc16" in p["kernel"] for p in plan.describe()["passes"])
    c = plan.forward(xd).cpu().numpy()
    ref = oracle.modes(W.astype(np.float64), x.astype(np.float64))
    assert rel(c, ref) <= 1e-6


def test_bf16x3_rejected_where_unsupported(g):
    rng = np.random.default_rng(9300)
    for b, n, dt in ((8, 4, "f32"), (16, 2, "f32"), (16, 3, "c64")):
        W = gi.haar_orthogonal(b, rng).astype(np.float32 if dt == "f32" else np.complex64)
        plan = g.Plan(W, n, dt, 1)
        with pytest.raises(g.GTTError) as ei:
            plan.set_precision(g.PREC_BF16X3)
        assert ei.value.status == 2


def test_auto_precision_picks_tensor_cores_for_b16_fp32(g):
    """The default (AUTO) runs b = 16 FP32 transforms with n >= 3 on the
    tensor-core path and everything else on CUDA cores; explicit CUDA-core
    schedules switch a plan to FP32."""
    rng = np.random.default_rng(9400)
    cases = [(16, 4, "f32", True), (16, 6, "f32", True), (16, 2, "f32", False),
             (16, 3, "c64", False), (8, 5, "f32", False)]
    for b, n, dt, tc in cases:
        if dt == "c64":
            W = gi.haar_unitary(b, rng).astype(np.complex64)
            x = gi.complex_normal_x((2, b ** n), rng, np.complex64)
        else:
            W = gi.haar_orthogonal(b, rng).astype(np.float32)
            x = gi.normal_x((2, b ** n), rng, np.float32)
        plan = g.Plan(W, n, dt, 2)
        d = plan.describe()
        assert (d["precision"] == "bf16x3") == tc, (b, n, dt, d["precision"])
        assert any("tc16" in p["kernel"] for p in d["passes"]) == tc
        y = plan.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        up = (lambda a: a.astype(np.complex128)) if dt == "c64" else (lambda a: a.astype(np.float64))
        ref = oracle.modes(up(W), up(x))
        assert np.linalg.norm(up(y.cpu().numpy()) - ref) / np.linalg.norm(ref) <= 1e-6, (b, n, dt)
        if tc:
            plan.set_pipeline(True, 3)           # keeps the tensor-core schedule
            assert plan.describe()["precision"] == "bf16x3"
            plan.autotune(8)                     # a tensor-core plan is left as it is
            assert plan.describe()["precision"] == "bf16x3"
            plan.set_schedule(16384, 128)        # a CUDA-core schedule: FP32
            assert plan.describe()["precision"] == "fp32"


@pytest.mark.parametrize("n,batch", [(4, 2), (6, 1)])
def test_bf16x2_two_piece_error_against_three_piece(g, n, batch):
    """The two-piece split (three products) leaves about 2^-16 relative per
    mode; the three-piece split (six products) reaches FP32 accuracy.  Both
    measured against the FP64 oracle on the same input."""
    rng = np.random.default_rng(9500 + n)
    W = gi.haar_orthogonal(16, rng).astype(np.float32)
    x = gi.normal_x((batch, 16 ** n), rng, np.float32)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.modes(W.astype(np.float64), x.astype(np.float64))
    errs = {}
    for name, prec in (("bf16x2", g.PREC_BF16X2), ("bf16x3", g.PREC_BF16X3)):
        plan = g.Plan(W, n, "f32", batch)
        plan.set_precision(prec)
        d = plan.describe()
        assert d["precision"] == name and all(name in p["kernel"] for p in d["passes"]), d
        errs[name] = rel(plan.forward(xd).cpu().numpy(), ref)
        plan.check()
    print(f"b=16 n={n}: bf16x2 rel-L2 {errs['bf16x2']:.3e}, bf16x3 rel-L2 {errs['bf16x3']:.3e}")
    assert errs["bf16x3"] <= 1e-6
    assert 1e-6 < errs["bf16x2"] <= 1e-4
    assert errs["bf16x2"] > 10 * errs["bf16x3"]


def tc_accumulation_probe(g):
    """The tensor core's FP32 accumulation, measured: a b = 16, n = 3 plan with
    W = all ones (exact in BF16, so the split leaves W1 = W2 = 0) applied to a
    vector whose only nonzero fibre is x[k, 0, 0], k = 0..15, with values exact
    in BF16 (x1 = x2 = 0).  Every output y[j, *, *] is then the tensor core's
    FP32 sum of the 16 products of one MMA, passed unchanged through the other
    two modes.  Returns the classification of three cases."""
    W = np.ones((16, 16), dtype=np.float32)
    cases = {
        # 2^24 + 1.5: round to nearest gives 2^24 + 2, truncation 2^24
        "rounding": ([2.0 ** 24, 1.5] + [0.0] * 14, {2.0 ** 24 + 2: "round-to-nearest", 2.0 ** 24: "truncation"}),
        # 1 then fifteen 2^-25: FP32 additions in order lose them all (1.0); a
        # wider sum (or the small terms combined first) gives 1 + 15 * 2^-25 rounded
        "small_terms_after_large": ([1.0] + [2.0 ** -25] * 15,
                                    {1.0: "each product rounded into an FP32 running sum",
                                     float(np.float32(1 + 4 * 2.0 ** -23)): "sum wider than FP32, rounded once (nearest)",
                                     float(np.float32(1 + 3 * 2.0 ** -23)): "sum wider than FP32, rounded once (truncated)"}),
        "small_terms_before_large": ([2.0 ** -25] * 15 + [1.0],
                                     {1.0: "small terms rounded away",
                                      float(np.float32(1 + 4 * 2.0 ** -23)): "small terms kept (exact partial sums), rounded to nearest",
                                      float(np.float32(1 + 3 * 2.0 ** -23)): "small terms kept (exact partial sums), truncated"}),
    }
    out = {}
    plan = g.Plan(W, 3, "f32", 1)
    plan.set_precision(g.PREC_BF16X3)
    for name, (vals, meaning) in cases.items():
        x = np.zeros((16, 16, 16), dtype=np.float32)   # [k2][k1][k0]: natural index k0 + 16 k1 + 256 k2
        x[0, 0, :] = np.asarray(vals, dtype=np.float32)
        y = plan.forward(torch.from_numpy(x.reshape(1, -1)).cuda()).cpu().numpy().reshape(16, 16, 16)
        got = set(float(v) for v in np.unique(y))
        assert len(got) == 1, (name, got)           # every output is the same 16-term sum
        v = got.pop()
        out[name] = {"value": v, "reading": meaning.get(v, "none of the modelled readings")}
    return out


def test_tensor_core_fp32_accumulation_is_measured(g):
    res = tc_accumulation_probe(g)
    print("tensor-core FP32 accumulation:", res)
    for name, r in res.items():
        assert r["reading"] != "none of the modelled readings", (name, r)


@pytest.mark.parametrize("n,batch", [(3, 4), (4, 3), (5, 2), (6, 1)])
def test_tf32x3_b16_matches_oracle(g, n, batch):
    """b = 16 FP32 on the TF32 two-piece path (A operand in tensor memory):
    forward and adjoint against the FP64 oracle within the 1e-6 gate."""
    rng = np.random.default_rng(9600 + n)
    W = gi.haar_orthogonal(16, rng).astype(np.float32)
    x = gi.normal_x((batch, 16 ** n), rng, np.float32)
    plan = g.Plan(W, n, "f32", batch)
    plan.set_precision(g.PREC_TF32X3)
    d = plan.describe()
    assert d["precision"] == "tf32x3" and all("tf32x3" in p["kernel"] for p in d["passes"]), d
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    z = plan.inverse(y)
    torch.cuda.synchronize()
    plan.check()
    ref = oracle.modes(W.astype(np.float64), x.astype(np.float64))
    e, e_rt = rel(y.cpu().numpy(), ref), rel(z.cpu().numpy(), x.astype(np.float64))
    print(f"tf32x3 b=16 n={n}: forward rel-L2 {e:.3e}, inverse(forward) {e_rt:.3e}")
    assert e <= 1e-6 and e_rt <= 2e-6
    # a non-orthogonal W: the adjoint transform against the oracle's
    W2 = (rng.standard_normal((16, 16)) * 0.3).astype(np.float32)
    plan.set_w(W2)
    zz = plan.inverse(xd).cpu().numpy()
    assert rel(zz, oracle.adjoint(W2.astype(np.float64), x.astype(np.float64))) <= 1e-6
