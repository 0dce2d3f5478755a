"""GPU parity of gtt_forward / gtt_inverse against the FP64 oracle.

Every comparison runs the CUDA path through the C ABI (via the thin binding)
and the oracle on the same seeded inputs.  Floating-point results are compared
by relative L2 error with the tolerances stated per workload; integer results
bit-exactly.
"""
import ctypes

import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu

DT = {"f64": (np.float64, False), "f32": (np.float32, False), "c64": (np.complex64, True),
      "c128": (np.complex128, True)}
# rel-L2 bounds for unitary / orthogonal W on the small sweeps
TOL = {"f64": 1e-13, "c128": 1e-13, "f32": 2e-6, "c64": 2e-6}


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


def rel_l2(a, ref):
    ref = np.asarray(ref)
    return float(np.linalg.norm(np.asarray(a, dtype=ref.dtype) - ref) / max(np.linalg.norm(ref), 1e-300))


def make_inputs(b, n, batch, dt, rng):
    npdt, cplx = DT[dt]
    if cplx:
        W = gi.haar_unitary(b, rng).astype(npdt)
        x = gi.complex_normal_x((batch, b ** n), rng, npdt)
    else:
        W = gi.haar_orthogonal(b, rng).astype(npdt)
        x = gi.normal_x((batch, b ** n), rng, npdt)
    return W, x


def up(a):
    a = np.asarray(a)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def gpu_fwd_inv(g, W, x, n, dt, sched=None):
    batch = x.shape[0]
    plan = g.Plan(W, n, dt, batch)
    if sched is not None:
        plan.set_schedule(*sched)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    return y.cpu().numpy(), xr.cpu().numpy(), plan


def n_for(b, target_log2=14):
    n = 1
    while b ** (n + 1) <= 2 ** target_log2:
        n += 1
    return n


# ------------------------------------------------------------- sweeps

@pytest.mark.parametrize("dt", ["f64", "f32", "c64", "c128"])
@pytest.mark.parametrize("b", list(range(2, 17)))
def test_forward_inverse_all_bases(g, dt, b):
    rng = np.random.default_rng(1000 + b)
    n = n_for(b)
    W, x = make_inputs(b, n, 3, dt, rng)
    y, xr, _ = gpu_fwd_inv(g, W, x, n, dt)
    ref = oracle.modes(up(W), up(x))
    assert rel_l2(y, ref) <= TOL[dt], rel_l2(y, ref)
    ref_inv = oracle.adjoint(up(W), up(y))
    assert rel_l2(xr, ref_inv) <= TOL[dt]
    assert rel_l2(xr, up(x)) <= 2 * TOL[dt]


@pytest.mark.parametrize("sched", [(64, 0), (256, 16), (2048, 32), (16384, 128), (65536, 256),
                                   (98304, 64), (200000, 512)])
@pytest.mark.parametrize("b,n,dt", [(2, 17, "f32"), (3, 10, "c64"), (4, 8, "f64"), (5, 7, "f32"),
                                    (7, 6, "c128"), (8, 5, "c64"), (16, 4, "f32")])
def test_schedule_sweep(g, sched, b, n, dt):
    """Every tile / run geometry the planner can emit gives the same transform."""
    rng = np.random.default_rng(2000 + b)
    W, x = make_inputs(b, n, 2, dt, rng)
    y, xr, plan = gpu_fwd_inv(g, W, x, n, dt, sched)
    ref = oracle.modes(up(W), up(x))
    assert rel_l2(y, ref) <= TOL[dt], (plan.describe(), rel_l2(y, ref))
    assert rel_l2(xr, up(x)) <= 2 * TOL[dt]


# ------------------------------------------------- the stated workloads

def test_b2_n12_f64_against_dense_oracle(g):
    """b=2, n=12, FP64, W = H/sqrt(2): forward and inverse vs the naive O(N^2)
    dense oracle, rel-L2 <= 1e-13."""
    W, x = gi.workload_inputs("b2_n12_f64")
    y, xr, _ = gpu_fwd_inv(g, W, x, 12, "f64")
    ref = oracle.dense(W, x[0]).real
    assert rel_l2(y[0], ref) <= 1e-13
    assert rel_l2(xr[0], oracle.dense(W.T.conj(), y[0]).real) <= 1e-13
    assert rel_l2(xr, x) <= 1e-13


def test_small_fp64_plan_spreads_over_many_ctas(g):
    """A small FP64 transform is split into passes of at most 3 digits with
    runs of 1 (FP64 runs at a small fraction of the FP32 rate, so one CTA per
    pass would bind): b = 2, n = 12 takes 4 passes of 512 tiles, and a
    complex128 b = 4, n = 6 plan (batch 1) 2 passes of 64 tiles; both against the dense
    oracle."""
    W, x = gi.workload_inputs("b2_n12_f64")
    plan = g.Plan(W, 12, "f64", 1)
    d = plan.describe()
    assert len(d["passes"]) == 4 and all(p["grid"] >= 256 for p in d["passes"]), d
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_l2(y[0], oracle.dense(W, x[0]).real) <= 1e-13
    rng = np.random.default_rng(7300)
    W4, x4 = make_inputs(4, 6, 1, "c128", rng)
    p4 = g.Plan(W4, 6, "c128", 1)
    assert len(p4.describe()["passes"]) == 2
    y4 = p4.forward(torch.from_numpy(x4).cuda()).cpu().numpy()
    assert rel_l2(y4, oracle.modes(W4, x4)) <= 1e-13


@pytest.mark.parametrize("n,batch,passes", [(4, 3, None), (5, 3, None), (6, 2, None), (7, 1, None), (8, 1, None),
                                             (7, 2, ([3, 4], [8, 1])), (7, 2, ([2, 2, 3], [64, 64, 8])),
                                             (6, 3, ([1, 5], [512, 1]))])
def test_b8_f32_tile_kernel_forward_and_adjoint(g, n, batch, passes):
    """FP32, b = 8: passes on 4096-element tiles run the compile-time tile
    kernel (top digits over runs of 8^(4-g), or the bottom digits of
    consecutive blocks on the first pass).  Forward and adjoint of a
    non-orthogonal W against the oracle, in place as well; other passes of
    an explicit schedule keep their kernels."""
    rng = np.random.default_rng(7200 + 10 * n + batch)
    W = (rng.standard_normal((8, 8)) * 0.4).astype(np.float32)
    x = gi.normal_x((batch, 8 ** n), rng, np.float32)
    plan = g.Plan(W, n, "f32", batch)
    if passes:
        plan.set_passes(*passes)
    d = plan.describe()
    names = [p["kernel"] for p in d["passes"]]
    assert any("gtt_forward_b8_kernel" in k for k in names), names
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    z = plan.inverse(xd)
    w = xd.clone()
    plan.forward(w, out=w)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(w, y)
    assert rel_l2(y.cpu().numpy(), oracle.modes(up(W), up(x))) <= TOL["f32"], names
    assert rel_l2(z.cpu().numpy(), oracle.adjoint(up(W), up(x))) <= TOL["f32"], names


def test_b4_n13_c64_full_size(g):
    """b=4, n=13 (N = 2^26), complex64, Haar W, in the default launch
    configuration: forward rel-L2 <= 1e-5, inverse(forward) vs x <= 2e-5,
    norm preserved."""
    W, x = gi.workload_inputs("b4_n13_c64")
    y, xr, plan = gpu_fwd_inv(g, W, x, 13, "c64")
    ref = oracle.modes(up(W), up(x))
    e = rel_l2(y, ref)
    print("b4_n13_c64 forward rel-L2", e, plan.describe())
    assert e <= 1e-5
    assert rel_l2(xr, up(x)) <= 2e-5
    assert abs(np.linalg.norm(up(y)) / np.linalg.norm(up(x)) - 1) <= 1e-5


def test_b16_n6_batch64_f32_full_size_sampled(g):
    """b=16, n=6, batch 64, FP32 CUDA-core path: the whole batch runs on the
    GPU; items 0, 21, 42, 63 are checked against the oracle (rel-L2 <= 1e-6)."""
    W, x = gi.workload_inputs("b16_n6_batch64_f32")
    plan = g.Plan(W, 6, "f32", 64)
    plan.set_precision(g.PREC_FP32)
    xd = torch.from_numpy(x).cuda()
    y = plan.forward(xd)
    torch.cuda.synchronize()
    for item in (0, 21, 42, 63):
        ref = oracle.modes(up(W), up(x[item]))
        e = rel_l2(y[item].cpu().numpy(), ref)
        assert e <= 1e-6, (item, e)


def test_b8_n7_batch32_f32_forward_sampled(g):
    """b=8, n=7, batch 32, FP32: forward rel-L2 <= 1e-5 on sampled items."""
    W, x = gi.workload_inputs("b8_n7_batch32_f32")
    plan = g.Plan(W, 7, "f32", 32)
    y = plan.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    for item in (0, 31):
        ref = oracle.modes(up(W), up(x[item]))
        assert rel_l2(y[item].cpu().numpy(), ref) <= 1e-5


# ------------------------------------------------------------- integers

def _i32_run(g, W, x, n):
    plan = g.Plan(np.asarray(W, dtype=np.int64).astype(np.int32), n, "i32", x.shape[0])
    xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.int64).astype(np.uint32).view(np.int32))).cuda()
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    return y.cpu().numpy().view(np.uint32), xr.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("amp", [2 ** 15, 2 ** 31 - 1])
def test_integer_hadamard_bit_exact(g, amp):
    """Unnormalised +-1 Hadamard on int32 (arithmetic mod 2^32), N = 2^12:
    bit-exact against the oracle; inverse(forward(x)) = 2^n x mod 2^32."""
    rng = np.random.default_rng(3000)
    n = 12
    x = rng.integers(-amp, amp, size=(2, 2 ** n), endpoint=True)
    W = np.array([[1, 1], [1, -1]])
    y, xr = _i32_run(g, W, x, n)
    np.testing.assert_array_equal(y, oracle.modes_u32(W, x))
    np.testing.assert_array_equal(xr, ((x.astype(np.int64) << n) & 0xFFFFFFFF).astype(np.uint32))


@pytest.mark.parametrize("b,n", [(3, 8), (5, 5), (16, 3), (2, 20)])
def test_integer_general_w_bit_exact(g, b, n):
    rng = np.random.default_rng(3100 + b)
    W = rng.integers(-9, 10, size=(b, b))
    x = rng.integers(-2 ** 30, 2 ** 30, size=(2, b ** n))
    y, _ = _i32_run(g, W, x, n)
    np.testing.assert_array_equal(y, oracle.modes_u32(W, x))


# ----------------------------------------------------------- edge cases

@pytest.mark.parametrize("b", [2, 3, 7, 16])
def test_single_digit_and_tiny_vectors_large_batch(g, b):
    rng = np.random.default_rng(4000 + b)
    for n, batch in ((1, 4097), (2, 1), (1, 1)):
        W, x = make_inputs(b, n, batch, "f32", rng)
        y, xr, _ = gpu_fwd_inv(g, W, x, n, "f32")
        assert rel_l2(y, oracle.modes(up(W), up(x))) <= TOL["f32"]


def test_in_place(g):
    rng = np.random.default_rng(4100)
    W, x = make_inputs(4, 9, 2, "c64", rng)
    plan = g.Plan(W, 9, "c64", 2)
    xd = torch.from_numpy(x).cuda()
    plan.forward(xd, out=xd)
    torch.cuda.synchronize()
    assert rel_l2(xd.cpu().numpy(), oracle.modes(up(W), up(x))) <= TOL["c64"]


def test_non_unitary_w_inverse_is_adjoint(g):
    """gtt_inverse is the W^H transform for any W (not G^-1)."""
    rng = np.random.default_rng(4200)
    W = (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))).astype(np.complex128) * 0.6
    x = gi.complex_normal_x((1, 3 ** 7), rng, np.complex128)
    y, xr, _ = gpu_fwd_inv(g, W, x, 7, "c128")
    assert rel_l2(y, oracle.modes(W, x)) <= 1e-13
    assert rel_l2(xr, oracle.adjoint(W, y)) <= 1e-13


def test_host_buffer_calls_match_device_calls(g):
    rng = np.random.default_rng(4300)
    W, x = make_inputs(4, 10, 2, "c64", rng)
    plan = g.Plan(W, 10, "c64", 2)
    yh = plan.forward_host(x)
    yd = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(yh, yd)
    xh = plan.inverse_host(yh)
    assert rel_l2(xh, up(x)) <= 2 * TOL["c64"]


def test_repeatable_bits(g):
    rng = np.random.default_rng(4400)
    W, x = make_inputs(8, 6, 3, "f32", rng)
    plan = g.Plan(W, 6, "f32", 3)
    xd = torch.from_numpy(x).cuda()
    a = plan.forward(xd).cpu().numpy()
    b = plan.forward(xd).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_misaligned_and_null_pointers_rejected(g):
    from paper_2507_02420_gb300 import _lib
    lib = _lib.load()
    W = np.eye(2, dtype=np.float32)
    plan = g.Plan(W, 4, "f32", 1)
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    st = lib.gtt_forward(plan._h, buf.data_ptr() + 4, buf.data_ptr(), None)
    assert st == 1
    st = lib.gtt_forward(plan._h, None, buf.data_ptr(), None)
    assert st == 1
    assert b"aligned" in lib.gtt_last_error() or lib.gtt_last_error()


# ------------------------------------------------- TMA-pipelined passes

@pytest.mark.parametrize("nbuf", [1, 2, 3, 4])
@pytest.mark.parametrize("b,n,dt,sched", [(4, 10, "c64", (32768, 128)), (2, 18, "f32", (16384, 128)),
                                          (8, 6, "f64", (32768, 128)), (16, 4, "f32", (16384, 1024)),
                                          (4, 9, "c128", (65536, 128)), (2, 16, "f32", (131072, 256)),
                                          (16, 5, "c64", (65536, 2048))])
def test_tma_pipeline_matches_oracle(g, nbuf, b, n, dt, sched):
    """TMA-staged passes (1..4 buffers) give the oracle's result; the plan's
    bounded-wait flag stays clear."""
    rng = np.random.default_rng(7000 + b + nbuf)
    W, x = make_inputs(b, n, 3, dt, rng)
    plan = g.Plan(W, n, dt, 3)
    plan.set_schedule(*sched)
    plan.set_pipeline(True, nbuf)
    d = plan.describe()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = plan.forward(xd)
    xr = plan.inverse(y)
    torch.cuda.synchronize()
    plan.check()
    ref = oracle.modes(up(W), up(x))
    assert rel_l2(y.cpu().numpy(), ref) <= TOL[dt], d
    assert rel_l2(xr.cpu().numpy(), up(x)) <= 2 * TOL[dt]
    # the same schedule without TMA gives bitwise identical results
    plan.set_pipeline(False, nbuf)
    y2 = plan.forward(xd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), y2.cpu().numpy())


def test_tma_used_for_power_of_two_bases(g):
    rng = np.random.default_rng(7100)
    W, x = make_inputs(4, 13, 1, "c64", rng)
    plan = g.Plan(W, 13, "c64", 1)
    plan.set_precision(g.PREC_FP32)  # the CUDA-core schedule (AUTO takes the tensor cores here)
    assert all(p["tma"] for p in plan.describe()["passes"])
