"""gtt_filter: natural-order spectral filtering (Sec. 4.3.2) on the GPU against
the paper's printed E10 values and the oracle's filter route."""
import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-6, "c64": 2e-6, "f64": 1e-12, "c128": 1e-12}


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


def make(b, n, batch, dt, rng):
    if dt in ("c64", "c128"):
        W = gi.haar_unitary(b, rng)
        x = gi.complex_normal_x((batch, b ** n), rng, np.complex128)
        cast = np.complex64 if dt == "c64" else np.complex128
    else:
        W = gi.haar_orthogonal(b, rng)
        x = gi.normal_x((batch, b ** n), rng, np.float64)
        cast = np.float32 if dt == "f32" else np.float64
    return W.astype(cast), x.astype(cast)


def test_e10_printed_values_through_the_gpu(g, golden):
    """Sec. 4.3.2: U3(pi/4, 0, pi), N = 16, cutoff 4; the low- and high-pass
    outputs printed to 4 decimals, complex128 on the GPU."""
    e = golden("e10_filter_u3_n4.txt")
    W = gi.u3(*e["theta_phi_lambda"]).astype(np.complex128)
    psi = (e["Psi"] / np.linalg.norm(e["Psi"])).astype(np.complex128)[None, :]
    c = int(e["cutoff"][0])
    plan = g.Plan(W, 4, "c128", 1)
    xd = torch.from_numpy(psi).cuda()
    low = plan.filter(xd, c, True).cpu().numpy()
    high = plan.filter(xd, c, False).cpu().numpy()
    torch.cuda.synchronize()
    np.testing.assert_allclose(low[0].real, e["low"], atol=5.1e-5)
    np.testing.assert_allclose(high[0].real, e["high"], atol=5.1e-5)
    np.testing.assert_allclose(low, oracle.filter(W, psi, c, True), atol=1e-13)
    np.testing.assert_allclose(high, oracle.filter(W, psi, c, False), atol=1e-13)


@pytest.mark.parametrize("b,n,dt,batch", [(2, 14, "f32", 3), (4, 8, "c64", 2), (16, 4, "f32", 3),
                                          (3, 7, "f64", 2), (8, 5, "c128", 2), (16, 3, "c64", 2)])
def test_filter_matches_oracle(g, b, n, dt, batch):
    rng = np.random.default_rng(9600 + b)
    W, x = make(b, n, batch, dt, rng)
    N = b ** n
    plan = g.Plan(W, n, dt, batch)
    xd = torch.from_numpy(x).cuda()
    for cut in (0, 1, N // 3, N // 2, N - 1, N):   # 1, N // 3: unaligned edges (4-byte zeroing)
        for keep_low in (True, False):
            y = plan.filter(xd, cut, keep_low).cpu().numpy()
            ref = oracle.filter(up(W), up(x), cut, keep_low)
            if (keep_low and cut == 0) or (not keep_low and cut == N):
                assert not np.any(y), (cut, keep_low)   # everything masked: exactly zero
                continue
            err = np.linalg.norm(up(y) - ref) / np.linalg.norm(ref)
            assert err <= TOL[dt], (b, n, dt, cut, keep_low, err)
    plan.check()


@pytest.mark.parametrize("b,n,dt,batch,prec", [(4, 10, "c64", 3, None), (2, 16, "f32", 1, None), (16, 4, "f32", 2, "bf16x3"),
                                               (8, 6, "f64", 2, None), (3, 8, "c64", 2, None)])
def test_filter_equals_forward_mask_inverse(g, b, n, dt, batch, prec):
    """The adjoint's first pass skips the tiles inside the zeroed range; every
    value must still equal forward -> mask -> inverse through the plain calls
    (exact comparison; +0 and -0 compare equal), for tile-aligned and
    unaligned cuts, both masks and several vectors."""
    rng = np.random.default_rng(9650 + b + n)
    W, x = make(b, n, batch, dt, rng)
    N = b ** n
    plan = g.Plan(W, n, dt, batch)
    if prec == "bf16x3":
        plan.set_precision(g.PREC_BF16X3)
    xd = torch.from_numpy(x).cuda()
    spec = plan.forward(xd)
    for cut in (1, N // 3, N // 2, N - 5):
        for keep_low in (True, False):
            y = plan.filter(xd, cut, keep_low).cpu().numpy()
            m = spec.clone()
            if keep_low:
                m[:, cut:] = 0
            else:
                m[:, :cut] = 0
            want = plan.inverse(m).cpu().numpy()
            np.testing.assert_array_equal(y, want, err_msg=f"cut {cut} keep_low {keep_low}")
    plan.check()


def test_filter_in_place_and_partition(g):
    """y == x is allowed; low + high recovers x for unitary W."""
    rng = np.random.default_rng(9700)
    W, x = make(4, 9, 2, "c64", rng)
    plan = g.Plan(W, 9, "c64", 2)
    cut = 4 ** 9 // 5
    lo = plan.filter(torch.from_numpy(x).cuda(), cut, True)
    xd = torch.from_numpy(x).cuda()
    plan.filter(xd, cut, False, out=xd)
    torch.cuda.synchronize()
    total = up(lo.cpu().numpy()) + up(xd.cpu().numpy())
    assert np.linalg.norm(total - up(x)) / np.linalg.norm(up(x)) <= 4e-6


def test_filter_rejects_bad_cut(g):
    rng = np.random.default_rng(9800)
    W, x = make(2, 6, 1, "f32", rng)
    plan = g.Plan(W, 6, "f32", 1)
    xd = torch.from_numpy(x).cuda()
    for cut in (-1, 2 ** 6 + 1):
        with pytest.raises(g.GTTError) as ei:
            plan.filter(xd, cut)
        assert ei.value.status == 1


def test_filter_full_size_bandwidth_workload(g):
    """b = 4, n = 13, complex64: low-pass at N / 3 against the oracle's filter."""
    W, x = gi.workload_inputs("b4_n13_c64")
    N = 4 ** 13
    plan = g.Plan(W, 13, "c64", 1)
    y = plan.filter(torch.from_numpy(x).cuda(), N // 3, True).cpu().numpy()
    ref = oracle.filter(up(W), up(x), N // 3, True)
    assert np.linalg.norm(up(y) - ref) / np.linalg.norm(ref) <= 1e-5
