"""Heterogeneous transforms (gtt_plan_create_mixed): G = W_0 (x) ... (x) W_{n-1}
with factors of different sizes (the remark after Def. 2.3), against the
oracle's mixed mode loop (itself pinned to numpy's Kronecker product)."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-6, "c64": 2e-6, "f64": 1e-12, "c128": 1e-12}
NP = {"f32": np.float32, "c64": np.complex64, "f64": np.float64, "c128": np.complex128}


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


def make(radices, batch, dt, rng):
    cplx = dt in ("c64", "c128")
    Ws = [(gi.haar_unitary(b, rng) if cplx else gi.haar_orthogonal(b, rng)).astype(NP[dt]) for b in radices]
    N = int(np.prod(radices))
    x = (gi.complex_normal_x((batch, N), rng, np.complex128) if cplx else gi.normal_x((batch, N), rng, np.float64))
    return Ws, x.astype(NP[dt])


def rel(a, ref):
    return float(np.linalg.norm(up(a) - ref) / np.linalg.norm(ref))


def merged_digits(radices):
    """The plan's digits, fastest first: adjacent factors whose sizes multiply
    to at most 16 form one digit (their Kronecker product)."""
    out, j, digits = [], 0, radices[::-1]
    while j < len(digits):
        m = digits[j]
        j += 1
        while j < len(digits) and m * digits[j] <= 16:
            m *= digits[j]
            j += 1
        out.append(m)
    return out


@pytest.mark.parametrize("radices,dt,batch", [([2, 3, 5, 7], "f64", 2), ([16, 2, 4], "c64", 3),
                                              ([3, 3, 8, 5, 2], "f32", 2), ([7, 11, 13], "c128", 1),
                                              ([16, 3, 9, 5, 7, 2, 2, 4, 11], "c64", 1),
                                              ([2] * 12 + [3], "f32", 2),
                                              ([16, 3, 5, 7, 9, 11], "f32", 2),
                                              ([13, 11, 7, 16, 9, 5], "c64", 2),
                                              ([16] * 5, "c64", 4), ([3] * 9, "c128", 2),
                                              ([11, 13, 7, 5, 3], "f64", 1),
                                              ([5] * 8, "f32", 3), ([3] * 11, "c64", 4)])
def test_mixed_forward_inverse_match_oracle(g, radices, dt, batch):
    rng = np.random.default_rng(10000 + len(radices))
    Ws, x = make(radices, batch, dt, rng)
    plan = g.Plan.mixed(Ws, dt, batch)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    plan.check()
    ref = oracle.modes_mixed([up(W) for W in Ws], up(x))
    assert rel(y.cpu().numpy(), ref) <= TOL[dt]
    assert rel(xr.cpu().numpy(), up(x)) <= 2 * TOL[dt]   # unitary factors: the adjoint inverts
    # consecutive digits share a pass, one stage each, while a tile of at most
    # 48 KiB holds them: the stages of all passes are the merged digits in order
    passes = plan.describe()["passes"]
    assert [b for p in passes for b in p["radices"]] == merged_digits(radices)
    assert all(p["kernel"].startswith("gtt_mixed_pass_kernel") and p["tile_bytes"] <= 48 * 1024 for p in passes)
    if radices == [16, 3, 9, 5, 7, 2, 2, 4, 11]:
        assert [p["radices"] for p in passes] == [[11, 16, 7], [5, 9, 3], [16]]


def test_equal_factors_give_the_single_base_transform(g):
    rng = np.random.default_rng(10100)
    W = gi.haar_unitary(4, rng).astype(np.complex64)
    x = gi.complex_normal_x((2, 4 ** 7), rng, np.complex64)
    y_mixed = g.Plan.mixed([W] * 7, "c64", 2).forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.modes(up(W), up(x))
    assert rel(y_mixed, ref) <= 2e-6


@pytest.mark.parametrize("radices,dt", [([2, 2, 2, 2], "c64"), ([3, 5, 2, 2, 3, 2], "f64"), ([2, 4, 2, 8], "c128"),
                                         ([7, 2, 2, 3], "f32")])
def test_merged_factors_match_oracle(g, radices, dt):
    """Factors that share a pass (their Kronecker product as one factor) against
    the oracle's factor-by-factor mode loop, forward and inverse."""
    rng = np.random.default_rng(10050 + len(radices) + radices[0])
    Ws, x = make(radices, 3, dt, rng)
    plan = g.Plan.mixed(Ws, dt, 3)
    assert len(plan.describe()["passes"]) < len(radices)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    ref = oracle.modes_mixed([up(W) for W in Ws], up(x))
    assert rel(y.cpu().numpy(), ref) <= TOL[dt]
    assert rel(plan.inverse(y).cpu().numpy(), up(x)) <= 2 * TOL[dt]


def test_mixed_integer_arithmetic_is_exact(g):
    """int32 factors with arithmetic mod 2^32; small values keep every partial
    sum exact in FP64, so the oracle's result is the exact integer."""
    rng = np.random.default_rng(10200)
    radices = [3, 2, 5, 4]
    Ws = [rng.integers(-3, 4, size=(b, b)).astype(np.int32) for b in radices]
    x = rng.integers(-50, 51, size=(2, int(np.prod(radices)))).astype(np.int32)
    y = g.Plan.mixed(Ws, "i32", 2).forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.modes_mixed([W.astype(np.float64) for W in Ws], x.astype(np.float64))
    np.testing.assert_array_equal(y.astype(np.int64), np.rint(ref).astype(np.int64))


@pytest.mark.parametrize("radices", [[3, 2, 5, 4], [2, 2, 2, 2, 3], [16, 7, 2, 8], [4, 4, 3],
                                     [16, 3, 5, 7, 9, 11]])
def test_mixed_integer_wraps_modulo_2_32(g, radices):
    """int32 factors and data over the whole 32-bit range, so products and sums
    overflow: bit-exact against the oracle's mod-2^32 heterogeneous loop,
    including passes that apply several adjacent factors as their Kronecker
    product (formed modulo 2^32 on the host)."""
    rng = np.random.default_rng(10250 + sum(radices))
    Ws = [rng.integers(-2 ** 31, 2 ** 31, size=(b, b)).astype(np.int32) for b in radices]
    N = int(np.prod(radices))
    x = rng.integers(-2 ** 31, 2 ** 31, size=(3, N)).astype(np.int32)
    plan = g.Plan.mixed(Ws, "i32", 3)
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.modes_mixed_u32(Ws, x)
    np.testing.assert_array_equal(y.view(np.uint32), ref)
    # the adjoint of an integer factor is its transpose
    yi = plan.inverse(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(yi.view(np.uint32), oracle.modes_mixed_u32([W.T for W in Ws], x))


def test_mixed_set_w_filter_and_codec(g):
    rng = np.random.default_rng(10300)
    radices = [5, 4, 3, 8]
    Ws, x = make(radices, 2, "c128", rng)
    N = int(np.prod(radices))
    plan = g.Plan.mixed(Ws, "c128", 2)
    Ws2, _ = make(radices, 1, "c128", rng)
    plan.set_w(Ws2)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.modes_mixed(Ws2, x)
    assert rel(plan.forward(xd).cpu().numpy(), ref) <= 1e-12
    # natural-order low-pass at N / 3 on the mixed spectrum
    adj = [W.conj().T for W in Ws2]
    keep = np.arange(N) < N // 3
    want = oracle.modes_mixed(adj, np.where(keep, ref, 0))
    assert rel(plan.filter(xd, N // 3, True).cpu().numpy(), want) <= 1e-12
    # top-k codec: the kept pairs and their reconstruction
    idx, val = plan.compress(xd, 50)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    np.testing.assert_allclose(val, np.take_along_axis(ref, idx, axis=1), atol=1e-12)
    spec = np.zeros_like(ref)
    np.put_along_axis(spec, idx, val, axis=1)
    rec = plan.decompress(torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda()).cpu().numpy()
    assert rel(rec, oracle.modes_mixed(adj, spec)) <= 1e-12


def test_mixed_set_w_on_multi_factor_passes(g):
    """New factors through gtt_plan_set_w reach every stage of every
    multi-factor pass (forward and adjoint), without rebuilding the plan."""
    rng = np.random.default_rng(10350)
    radices = [16, 3, 9, 5, 7, 2, 2, 4, 11]
    Ws, x = make(radices, 1, "c64", rng)
    plan = g.Plan.mixed(Ws, "c64", 1)
    assert len(plan.describe()["passes"]) == 3
    Ws2, _ = make(radices, 1, "c64", rng)
    plan.set_w(Ws2)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    ref = oracle.modes_mixed([up(W) for W in Ws2], up(x))
    assert rel(y.cpu().numpy(), ref) <= TOL["c64"]
    assert rel(plan.inverse(y).cpu().numpy(), up(x)) <= 2 * TOL["c64"]


def test_mixed_plan_rejections(g):
    rng = np.random.default_rng(10400)
    Ws, x = make([2, 3], 1, "f32", rng)
    plan = g.Plan.mixed(Ws, "f32", 1)
    xd = torch.from_numpy(x).cuda()
    for call in (lambda: plan.backward(xd, xd), lambda: plan.set_passes([1, 1], [1, 1]),
                 lambda: plan.autotune(4), lambda: plan.set_schedule(4096, 64)):
        with pytest.raises(g.GTTError) as ei:
            call()
        assert ei.value.status == 2
    with pytest.raises(g.GTTError) as ei:
        g.Plan.mixed([np.eye(17, dtype=np.float32), np.eye(2, dtype=np.float32)], "f32", 1)
    assert ei.value.status == 1
