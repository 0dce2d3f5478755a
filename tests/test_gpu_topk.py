"""gtt_compress / gtt_decompress: the top-k compression codec of Sec. 4.1.5.

The selection is an integer decision taken from floating-point magnitudes, so
it is checked bit-exactly against the same decision taken on the host from
the GPU's own spectrum in the same precision (|c|^2 with separately rounded
products and sum; larger index first between equal magnitudes); the spectrum
and the reconstruction are checked against the oracle within tolerance."""
import math

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


def host_select(spec, k):
    """Top-k indices per row of `spec` (a numpy array in the GPU's precision):
    |c|^2 descending (nonnegative, so value order is bit order), then the
    larger index first."""
    if np.iscomplexobj(spec):
        mag = spec.real * spec.real + spec.imag * spec.imag   # separately rounded, same precision
    else:
        mag = spec * spec
    N = spec.shape[-1]
    out = []
    for m in mag:
        if N > (1 << 16):   # keep the candidates at or above the k-th largest magnitude
            thr = np.partition(m, N - k)[N - k]
            cand = np.nonzero(m >= thr)[0]
        else:
            cand = np.arange(N)
        out.append(cand[np.lexsort((-cand, -m[cand]))][:k])
    return np.stack(out)


def make(b, n, batch, dt, rng):
    if dt in ("c64", "c128"):
        W = gi.haar_unitary(b, rng)
        x = gi.complex_normal_x((batch, b ** n), rng, np.complex128)
    else:
        W = gi.haar_orthogonal(b, rng)
        x = gi.normal_x((batch, b ** n), rng, np.float64)
    return W.astype(NP[dt]), x.astype(NP[dt])


def test_printed_compression_examples_through_the_gpu(g, golden):
    """Sec. 4.1.5, k = 2, complex128: the kept index sets [0 3] (GTT) and
    [7 6] (Hadamard, S2 and S3) and the printed fidelities."""
    g1 = golden("e3_compression_u3_n3.txt")
    ge = golden("e3_e5_compression_fidelity_k2.txt")
    W = gi.u3(*g1["theta_phi_lambda"])
    H = gi.hadamard_w(True).astype(np.complex128)
    for row, s in enumerate([g1["S1"], ge["S2"], ge["S3"]]):
        s = (s / np.linalg.norm(s)).astype(np.complex128)[None, :]
        for T, col, squared in ((W, "gtt_fidelity", True), (H, "hadamard_fidelity", False)):
            plan = g.Plan(T, 3, "c128", 1)
            idx, val = plan.compress(torch.from_numpy(s).cuda(), 2)
            idx, val = idx.cpu().numpy(), val.cpu().numpy()
            F = float(np.sum(np.abs(val) ** 2))
            assert abs((F * F if squared else F) - ge[col][row]) <= 1e-3
            if col == "gtt_fidelity" or row > 0:
                want = ge["S1_gtt_indices"] if col == "gtt_fidelity" else ge["S1_hadamard_indices"]
                np.testing.assert_array_equal(idx[0], want.astype(int))
            rec = plan.decompress(torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda()).cpu().numpy()[0]
            np.testing.assert_allclose(rec, oracle.reconstruct(T, idx, val, 8)[0], atol=1e-13)
            assert abs(abs(np.vdot(s[0], rec / np.linalg.norm(rec))) ** 2 - F) <= 1e-12


@pytest.mark.parametrize("b,n,dt,batch,k", [(2, 12, "f32", 3, 37), (4, 7, "c64", 2, 1000), (16, 3, "f32", 2, 4096),
                                            (3, 8, "f64", 2, 100), (8, 4, "c128", 3, 7), (4, 9, "c64", 1, 1)])
def test_selection_is_exact_and_reconstruction_matches_oracle(g, b, n, dt, batch, k):
    rng = np.random.default_rng(9900 + b + k)
    W, x = make(b, n, batch, dt, rng)
    N = b ** n
    plan = g.Plan(W, n, dt, batch)
    spec_d = torch.empty(batch, N, dtype=plan.torch_dtype, device="cuda")
    idx, val = plan.compress(torch.from_numpy(x).cuda(), k, spectrum=spec_d)
    spec = spec_d.cpu().numpy()
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    # the decision, repeated on the host in the same precision
    np.testing.assert_array_equal(idx, host_select(spec, k))
    np.testing.assert_array_equal(val, np.take_along_axis(spec, idx, axis=1))
    # the spectrum and the reconstruction against the oracle
    ref = oracle.modes(up(W), up(x))
    assert np.linalg.norm(up(spec) - ref) / np.linalg.norm(ref) <= TOL[dt]
    rec = plan.decompress(torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda()).cpu().numpy()
    rref = oracle.reconstruct(up(W), idx, up(val), N)
    assert np.linalg.norm(up(rec) - rref) / np.linalg.norm(rref) <= TOL[dt]
    plan.check()


def test_all_ties_keep_the_largest_indices(g):
    """H/sqrt(2) on a basis vector: every coefficient has the same magnitude."""
    W = gi.hadamard_w(True).astype(np.float32)
    x = np.zeros((2, 2 ** 10), np.float32)
    x[0, 0] = 1.0
    x[1, 5] = 1.0
    plan = g.Plan(W, 10, "f32", 2)
    idx, _ = plan.compress(torch.from_numpy(x).cuda(), 6)
    want = np.arange(1023, 1017, -1)
    np.testing.assert_array_equal(idx.cpu().numpy(), np.stack([want, want]))


@pytest.mark.parametrize("b,n,dt,batch,k", [(4, 10, "c64", 3, 4096), (2, 21, "f32", 2, 700), (8, 7, "f64", 2, 33)])
def test_candidate_prepass_selection_is_exact(g, b, n, dt, batch, k):
    """Vectors of 2^20 elements or more go through the 12-bit bucket pre-pass
    and a candidate list; the selection must still equal the host's."""
    rng = np.random.default_rng(9930 + b + n)
    W, x = make(b, n, batch, dt, rng)
    plan = g.Plan(W, n, dt, batch)
    spec_d = torch.empty(batch, b ** n, dtype=plan.torch_dtype, device="cuda")
    idx, val = plan.compress(torch.from_numpy(x).cuda(), k, spectrum=spec_d)
    spec = spec_d.cpu().numpy()
    np.testing.assert_array_equal(idx.cpu().numpy(), host_select(spec, k))
    np.testing.assert_array_equal(val.cpu().numpy(), np.take_along_axis(spec, idx.cpu().numpy(), axis=1))
    plan.check()


def test_estimate_above_the_kth_key_collects_again(g):
    """The threshold estimate samples every 32nd coefficient.  Vector 0 has
    100 large coefficients, all at sampled indices, so the estimate lands on
    their bucket although the 1024th largest key lies far below it: the exact
    histogram catches this and the vector collects again from the exact
    bucket.  Vector 1 has none and takes the estimate.  Both selections must
    equal the host's.  (W = I, so the spectrum is x.)"""
    rng = np.random.default_rng(9960)
    n, k = 10, 1024
    x = gi.complex_normal_x((2, 4 ** n), rng, np.complex64).astype(np.complex64)
    x[0, 32 * np.arange(100)] = 100.0 + 50.0j
    plan = g.Plan(np.eye(4, dtype=np.complex64), n, "c64", 2)
    spec_d = torch.empty(2, 4 ** n, dtype=plan.torch_dtype, device="cuda")
    idx, val = plan.compress(torch.from_numpy(x).cuda(), k, spectrum=spec_d)
    spec = spec_d.cpu().numpy()
    np.testing.assert_array_equal(spec, x)
    np.testing.assert_array_equal(idx.cpu().numpy(), host_select(spec, k))
    np.testing.assert_array_equal(val.cpu().numpy(), np.take_along_axis(spec, idx.cpu().numpy(), axis=1))
    assert set(32 * np.arange(100)) <= set(idx.cpu().numpy()[0].tolist())
    plan.check()


def test_candidate_overflow_falls_back_to_the_spectrum(g):
    """2^20 equal magnitudes: every coefficient lands in one bucket, the
    candidate list overflows, and the selection reads the spectrum: the
    largest indices, in descending order."""
    W = gi.hadamard_w(True).astype(np.float32)
    n = 20
    x = np.zeros((2, 2 ** n), np.float32)
    x[0, 0] = 1.0
    x[1, 12345] = 1.0
    plan = g.Plan(W, n, "f32", 2)
    idx, _ = plan.compress(torch.from_numpy(x).cuda(), 100)
    want = np.arange(2 ** n - 1, 2 ** n - 101, -1)
    np.testing.assert_array_equal(idx.cpu().numpy(), np.stack([want, want]))


def test_keeping_everything_reconstructs_x(g):
    rng = np.random.default_rng(9910)
    W, x = make(4, 5, 2, "c64", rng)   # N = 1024 <= 4096
    plan = g.Plan(W, 5, "c64", 2)
    idx, val = plan.compress(torch.from_numpy(x).cuda(), 1024)
    rec = plan.decompress(idx, val).cpu().numpy()
    assert np.linalg.norm(up(rec) - up(x)) / np.linalg.norm(up(x)) <= 4e-6


@pytest.mark.parametrize("b,n,dt,batch,k,layout", [(4, 10, "c64", 2, 1024, "random"), (2, 20, "f32", 1, 700, "random"),
                                                    (8, 7, "f64", 3, 33, "one_tile"), (16, 5, "c128", 2, 100, "random"),
                                                    (4, 13, "c64", 1, 4096, "clustered"), (2, 12, "f32", 2, 1, "random")])
def test_decompress_first_pass_on_kept_pairs_equals_the_dense_inverse(g, b, n, dt, batch, k, layout):
    """gtt_decompress runs its first pass only on the tiles that hold kept
    pairs (after zero-filling y); every value must equal the plain inverse
    of the zero-filled spectrum with the pairs scattered into it (exact
    comparison; +0 and -0 compare equal).  Indices outside [0, N) are
    skipped."""
    rng = np.random.default_rng(9970 + b + n + k)
    W, _ = make(b, 1, 1, dt, rng)
    N = b ** n
    if layout == "one_tile":
        idx = np.stack([rng.choice(64, size=k, replace=False) + 1000 for _ in range(batch)])
    elif layout == "clustered":
        idx = np.stack([rng.choice(N // 64, size=k, replace=False) * 7 % N for _ in range(batch)])
    else:
        idx = np.stack([rng.choice(N, size=k, replace=False) for _ in range(batch)])
    idx = idx.astype(np.int64)
    if k > 2:
        idx[0, 0], idx[0, 1] = -1, N   # skipped
    cplx = dt in ("c64", "c128")
    val = (rng.standard_normal((batch, k)) + (1j * rng.standard_normal((batch, k)) if cplx else 0)).astype(NP[dt])
    plan = g.Plan(W, n, dt, batch)
    y = plan.decompress(torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda()).cpu().numpy()
    spec = np.zeros((batch, N), NP[dt])
    for v in range(batch):
        ok = (idx[v] >= 0) & (idx[v] < N)
        spec[v, idx[v][ok]] = val[v][ok]
    want = plan.inverse(torch.from_numpy(spec).cuda()).cpu().numpy()
    np.testing.assert_array_equal(y, want)
    plan.check()


def test_codec_rejects_bad_arguments(g):
    rng = np.random.default_rng(9920)
    W, x = make(2, 6, 1, "f32", rng)
    plan = g.Plan(W, 6, "f32", 1)
    xd = torch.from_numpy(x).cuda()
    for k in (0, 65, 5000):
        with pytest.raises(g.GTTError) as ei:
            plan.compress(xd, k)
        assert ei.value.status == 1
    ip = g.Plan(np.array([[1, 1], [1, -1]], dtype=np.int32), 6, "i32", 1)
    with pytest.raises(g.GTTError) as ei:
        ip.compress(torch.zeros(1, 64, dtype=torch.int32, device="cuda"), 4)
    assert ei.value.status == 2


def test_full_size_bandwidth_workload(g):
    """b = 4, n = 13, complex64, k = 1024: exact selection from the GPU spectrum."""
    W, x = gi.workload_inputs("b4_n13_c64")
    plan = g.Plan(W, 13, "c64", 1)
    spec_d = torch.empty(1, 4 ** 13, dtype=torch.complex64, device="cuda")
    idx, val = plan.compress(torch.from_numpy(x).cuda(), 1024, spectrum=spec_d)
    spec = spec_d.cpu().numpy()
    np.testing.assert_array_equal(idx.cpu().numpy(), host_select(spec, 1024))
    rec = plan.decompress(idx, val).cpu().numpy()
    F = float(np.sum(np.abs(val.cpu().numpy().astype(np.complex128)) ** 2) / np.linalg.norm(up(x)) ** 2)
    assert abs(np.vdot(up(x)[0], up(rec)[0]).real / np.linalg.norm(up(x)) ** 2 - F) <= 1e-5
    assert 0 < F < 1
    assert math.isfinite(F)
