"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a route against a
different statement (the Kronecker definition through numpy's kron, the
recursive basis functions, closed forms, the paper's printed worked examples,
invariants, finite differences).  The last test plants plausible mistakes in
the oracle's use and checks that the pins catch them.
"""
import math

import numpy as np
import pytest

import gtt_inputs as gi
import oracle

BASES = (2, 3, 4, 5, 8, 16)


def kron_power(W, n):
    """Def. 2.3: G_N = W^{(x)n}, through numpy's Kronecker product."""
    G = np.array(W, dtype=np.complex128)
    for _ in range(n - 1):
        G = np.kron(G, W)
    return G


def rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def small_n(b):
    return {2: 8, 3: 5, 4: 4, 5: 3, 8: 3, 16: 2}[b]


# ---------------------------------------------------------------- routes

@pytest.mark.parametrize("b", BASES)
def test_dense_matches_kronecker_definition(b):
    """O1 (element product form, Sec. 2.6) equals Def. 2.3 (W^{(x)n} via kron)."""
    rng = np.random.default_rng(10 + b)
    n = small_n(b)
    W = rand_c(rng, (b, b))  # a general, non-unitary, non-symmetric W
    x = rand_c(rng, b ** n)
    G = kron_power(W, n)
    np.testing.assert_allclose(oracle.dense_matrix(W, n), G, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.dense(W, x), G @ x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("b", BASES)
def test_basis_function_route_equals_dense(b):
    """O2: sampling the recursive basis functions f_q at the midpoints x_p
    (Eq. defGNOne with Eq. gtt_recursive_general_b_main) gives the same matrix."""
    rng = np.random.default_rng(20 + b)
    n = 2 if b == 16 else 3
    W = rand_c(rng, (b, b))
    np.testing.assert_allclose(oracle.basis_matrix(W, n), kron_power(W, n), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("b", BASES)
def test_alg1_and_mode_loop_equal_definition(b):
    """O3 (Algorithm 1) and O4 (mode loop) reproduce G_N x for general W."""
    rng = np.random.default_rng(30 + b)
    n = small_n(b)
    W = rand_c(rng, (b, b))
    x = rand_c(rng, (3, b ** n))
    ref = x @ kron_power(W, n).T
    np.testing.assert_allclose(oracle.alg1(W, x[1]), ref[1], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.modes(W, x, threads=3), ref, rtol=1e-12, atol=1e-12)
    Wr = rng.standard_normal((b, b))
    xr = rng.standard_normal((2, b ** n))
    np.testing.assert_allclose(oracle.modes(Wr, xr), xr @ kron_power(Wr, n).real.T,
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("b", (2, 3, 4))
def test_single_mode_pass_is_one_kronecker_factor(b):
    """O4's building block: one mode-k pass applies W to digit k only, i.e. it is
    the matrix I_{b^(n-1-k)} (x) W (x) I_{b^k} (Def. 2.3 with every other
    factor the identity; digit k has stride b^k).  Composing the passes for
    k = 0..n-1 gives W^{(x)n}.  A swapped digit (k <-> n-1-k), an off-by-one k,
    or a transposed W fails."""
    rng = np.random.default_rng(40 + b)
    n = 4
    N = b ** n
    W = rand_c(rng, (b, b))          # general, non-unitary, non-symmetric
    x = rand_c(rng, N)
    cur = x
    for k in range(n):
        F = np.kron(np.kron(np.eye(b ** (n - 1 - k)), W), np.eye(b ** k))
        y = oracle.mode_pass(W, x, k, threads=2)
        np.testing.assert_allclose(y, F @ x, rtol=1e-12, atol=1e-12)
        # the wrong digits give something else
        for kk in {n - 1 - k, (k + 1) % n} - {k}:
            Fk = np.kron(np.kron(np.eye(b ** (n - 1 - kk)), W), np.eye(b ** kk))
            assert not np.allclose(y, Fk @ x, atol=1e-6)
        Ft = np.kron(np.kron(np.eye(b ** (n - 1 - k)), W.T), np.eye(b ** k))
        assert not np.allclose(y, Ft @ x, atol=1e-6)
        cur = oracle.mode_pass(W, cur, k, threads=1)
    np.testing.assert_allclose(cur, kron_power(W, n) @ x, rtol=1e-12, atol=1e-12)
    with pytest.raises(RuntimeError):
        oracle.mode_pass(W, x, n)


def test_hadamard_closed_form():
    """Sec. 2.6: for W = H/sqrt(2), G_N(p,q) = (-1)^{p.q} / sqrt(N)."""
    n = 10
    N = 2 ** n
    p = np.arange(N)[:, None]
    q = np.arange(N)[None, :]
    pq = p & q
    parity = np.zeros_like(pq)
    for k in range(n):
        parity ^= (pq >> k) & 1
    Gclosed = np.where(parity == 1, -1.0, 1.0) / math.sqrt(N)
    x = np.random.default_rng(0).uniform(-1, 1, N)
    y = oracle.modes(gi.hadamard_w(True), x)
    np.testing.assert_allclose(y, Gclosed @ x, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.dense_matrix(gi.hadamard_w(True), 6).real,
                               Gclosed[:64, :64] * math.sqrt(N) / 8.0, atol=1e-15)


# ------------------------------------------------------ worked examples

def test_e2_fourier_series_adjoint(golden):
    """Sec. 2.5.1: C = N^{-1/2} G^H g with W = [[1,i],[1,-i]]/sqrt(2) is (1/2, -i/2)."""
    g = golden("e2_fourier_series_b2_n1.txt")
    W = np.vstack([g["W_row0"], g["W_row1"]]).astype(np.complex128)
    C = oracle.adjoint(W, g["g"].astype(np.complex128)) / math.sqrt(2.0)
    np.testing.assert_allclose(C, g["C"], atol=1e-15)


def test_e3_compression_example(golden):
    """Sec. 4.1.5: U3(pi/4, pi/3, pi/6); the printed W, G_N (8x8) and G_N |S1>."""
    g = golden("e3_compression_u3_n3.txt")
    W = gi.u3(*g["theta_phi_lambda"])
    # re and im are each rounded to 3 decimals: |error| <= 0.5e-3 * sqrt(2)
    tol3 = 0.5e-3 * math.sqrt(2) + 1e-12
    np.testing.assert_allclose(W, np.vstack([g["W_row0"], g["W_row1"]]), atol=tol3)
    G_printed = np.vstack([g[f"G_row{i}"] for i in range(8)])
    np.testing.assert_allclose(oracle.dense_matrix(W, 3), G_printed, atol=tol3)
    # G S1 from the 3-decimal S1: rounding of S1 moves the result by < 2.5e-3
    np.testing.assert_allclose(oracle.modes(W, g["S1"]), g["G_S1"], atol=2.5e-3)
    np.testing.assert_allclose(oracle.alg1(W, g["S1"]), g["G_S1"], atol=2.5e-3)
    np.testing.assert_allclose(oracle.modes(gi.hadamard_w(True), g["S1"]), g["H_S1"], atol=2.5e-3)


def test_e3_e5_topk_compression(golden):
    """Sec. 4.1.5, k = 2: the retained index sets and the fidelity table.  The
    re-normalised truncation has fidelity F = sum over the kept |c|^2; the
    printed Hadamard column is F and the printed GTT column is F^2 (the table
    is inconsistent; both are pinned as printed).  The inputs are printed to 3
    decimals, so the fidelities agree to 1e-3."""
    g1 = golden("e3_compression_u3_n3.txt")
    g = golden("e3_e5_compression_fidelity_k2.txt")
    W = gi.u3(*g1["theta_phi_lambda"])
    H = gi.hadamard_w(True)
    states = [g1["S1"], g["S2"], g["S3"]]
    for row, s in enumerate(states):
        s = s / np.linalg.norm(s)
        for T, col, squared in ((W, "gtt_fidelity", True), (H, "hadamard_fidelity", False)):
            idx, val = oracle.topk(T, s, 2)
            F = float(np.sum(np.abs(val) ** 2))
            assert abs((F * F if squared else F) - g[col][row]) <= 1e-3, (row, col, F)
            # the reconstruction from the kept pair, re-normalised, has fidelity F
            rec = oracle.reconstruct(T, idx, val, 8)[0]
            rec = rec / np.linalg.norm(rec)
            assert abs(abs(np.vdot(s, rec)) ** 2 - F) <= 1e-12
        if row == 0:
            np.testing.assert_array_equal(oracle.topk(W, s, 2)[0][0], g["S1_gtt_indices"].astype(int))
        else:   # S2, S3: the Hadamard spectrum has no ties among its top two
            np.testing.assert_array_equal(oracle.topk(H, s, 2)[0][0], g["S1_hadamard_indices"].astype(int))
            np.testing.assert_array_equal(oracle.topk(W, s, 2)[0][0], g["S1_gtt_indices"].astype(int))


def test_topk_order_and_tie_break():
    """Largest |c| first; equal magnitudes keep the larger index first (the
    printed Hadamard choice [7 6] for S1 where indices 5 and 6 tie exactly)."""
    # H/sqrt(2) on e_0: every coefficient has magnitude 2^(-n/2): all ties
    idx, val = oracle.topk(gi.hadamard_w(True), np.eye(16)[0], 5)
    np.testing.assert_array_equal(idx[0], [15, 14, 13, 12, 11])
    rng = np.random.default_rng(77)
    W = gi.haar_unitary(3, rng)
    x = gi.complex_normal_x((2, 81), rng, np.complex128)
    idx, val = oracle.topk(W, x, 81)
    c = oracle.modes(W, x)
    for b in range(2):
        mags = np.abs(val[b])
        assert np.all(np.diff(mags) <= 1e-15)
        np.testing.assert_array_equal(np.sort(idx[b]), np.arange(81))   # k = N keeps everything
    np.testing.assert_allclose(oracle.reconstruct(W, idx, val, 81), x, atol=1e-13)
    np.testing.assert_allclose(np.take_along_axis(c, idx, axis=1), val)


def test_e10_natural_order_filter(golden):
    """Sec. 4.3.2: spectrum of the normalised signal under U3(pi/4, 0, pi), and
    the low/high outputs G^dagger(mask * spectrum) with cutoff c = 4."""
    g = golden("e10_filter_u3_n4.txt")
    W = gi.u3(*g["theta_phi_lambda"])
    psi = g["Psi"] / np.linalg.norm(g["Psi"])
    spec = oracle.modes(W, psi)
    np.testing.assert_allclose(spec.imag, 0, atol=1e-15)
    np.testing.assert_allclose(spec.real, g["spectrum"], atol=5.1e-5)
    c = int(g["cutoff"][0])
    idx = np.arange(16)
    low = oracle.adjoint(W, np.where(idx < c, spec, 0))
    high = oracle.adjoint(W, np.where(idx >= c, spec, 0))
    np.testing.assert_allclose(low.real, g["low"], atol=5.1e-5)
    np.testing.assert_allclose(high.real, g["high"], atol=5.1e-5)
    # the oracle's filter route gives the printed outputs too
    np.testing.assert_allclose(oracle.filter(W, psi, c, True).real, g["low"], atol=5.1e-5)
    np.testing.assert_allclose(oracle.filter(W, psi, c, False).real, g["high"], atol=5.1e-5)
    # low + high = G^dagger G psi = psi for unitary W (the masks partition the spectrum)
    np.testing.assert_allclose(oracle.filter(W, psi, c, True) + oracle.filter(W, psi, c, False), psi,
                               atol=1e-14)
    # Sec. 4.3.2 also transforms the outputs back: the masks are recovered
    np.testing.assert_allclose(oracle.modes(W, low), np.where(idx < c, spec, 0), atol=1e-14)


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("b", BASES)
def test_unitary_norm_and_adjoint_roundtrip(b):
    """Thm. thm_unitary_G_N: for unitary W, ||G x|| = ||x|| and G^H G x = x."""
    rng = np.random.default_rng(40 + b)
    n = small_n(b) + (2 if b <= 4 else 1)
    W = gi.haar_unitary(b, rng)
    x = rand_c(rng, (2, b ** n))
    y = oracle.modes(W, x)
    np.testing.assert_allclose(np.linalg.norm(y, axis=1), np.linalg.norm(x, axis=1), rtol=1e-13)
    np.testing.assert_allclose(oracle.adjoint(W, y), x, rtol=1e-12, atol=1e-12)
    Wr = gi.haar_orthogonal(b, rng)
    xr = rng.standard_normal(b ** n)
    np.testing.assert_allclose(oracle.adjoint(Wr, oracle.modes(Wr, xr)), xr, atol=1e-12)


@pytest.mark.parametrize("b", BASES)
def test_basis_vector_maps_to_kron_of_columns(b):
    """Def. 2.3 closed form: G e_q = W[:, q_{n-1}] (x) ... (x) W[:, q_0]
    (the leftmost Kronecker factor carries the most significant digit)."""
    rng = np.random.default_rng(50 + b)
    n = small_n(b)
    N = b ** n
    W = rand_c(rng, (b, b))
    for q in rng.integers(0, N, size=4):
        digits = [(int(q) // b ** k) % b for k in range(n)]
        ref = np.array([1.0 + 0j])
        for k in reversed(range(n)):
            ref = np.kron(ref, W[:, digits[k]])
        e = np.zeros(N, dtype=np.complex128)
        e[q] = 1
        np.testing.assert_allclose(oracle.modes(W, e), ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("b", BASES)
def test_separable_input_maps_factorwise(b):
    """G (u_{n-1} (x) ... (x) u_0) = (W u_{n-1}) (x) ... (x) (W u_0) with
    distinct u_k (distinct factors expose any digit-order mistake)."""
    rng = np.random.default_rng(60 + b)
    n = small_n(b) + 1
    W = rand_c(rng, (b, b))
    us = [rand_c(rng, b) for _ in range(n)]
    x = np.array([1.0 + 0j])
    ref = np.array([1.0 + 0j])
    for k in reversed(range(n)):
        x = np.kron(x, us[k])
        ref = np.kron(ref, W @ us[k])
    np.testing.assert_allclose(oracle.modes(W, x), ref, rtol=1e-11, atol=1e-12)


# ------------------------------------------------------------- integers

def _hadamard_pm1_bigint(x):
    """y[p] = sum_q (-1)^{popcount(p & q)} x[q] exactly, then mod 2^32."""
    N = len(x)
    n = N.bit_length() - 1
    p = np.arange(N)[:, None]
    q = np.arange(N)[None, :]
    pq = p & q
    parity = np.zeros_like(pq)
    for k in range(n):
        parity ^= (pq >> k) & 1
    S = np.where(parity == 1, -1, 1).astype(np.int64)
    y = S @ np.asarray(x, dtype=np.int64)    # |y| <= N * 2^31 < 2^63
    return (y % (1 << 32)).astype(np.uint32)


@pytest.mark.parametrize("amp", [2 ** 15, 2 ** 31 - 1])
def test_integer_hadamard_bit_exact(amp):
    """Unnormalised +-1 Hadamard (Sec. 2.3, b=2 case) on integers, N = 2^12:
    the uint32 mode loop equals the exact sum reduced mod 2^32 (amp = 2^31-1
    makes partial sums overflow, so the wrap-around itself is pinned)."""
    rng = np.random.default_rng(70)
    N = 2 ** 12
    x = rng.integers(-amp, amp, size=N, endpoint=True)
    W = np.array([[1, 1], [1, -1]])
    ref = _hadamard_pm1_bigint(x)
    np.testing.assert_array_equal(oracle.modes_u32(W, x), ref)
    np.testing.assert_array_equal(oracle.dense_u32(W, x[:256]), _hadamard_pm1_bigint(x[:256]))


def test_integer_general_w_wraps_like_python_ints():
    """uint32 mode loop for a general integer 3x3 W equals exact big-integer
    arithmetic mod 2^32 (Python ints, Kronecker definition)."""
    rng = np.random.default_rng(71)
    b, n = 3, 4
    W = rng.integers(-7, 8, size=(b, b))
    x = rng.integers(-2 ** 20, 2 ** 20, size=b ** n)
    G = np.array([[1]], dtype=object)
    for _ in range(n):
        G = np.kron(G, W.astype(object))
    y = [(int(v) % (1 << 32)) for v in G.dot(x.astype(object))]
    np.testing.assert_array_equal(oracle.modes_u32(W, x), np.array(y, dtype=np.uint32))


# ------------------------------------------------------------- gradient

def test_gradient_matches_finite_differences_real():
    """O6 vs FP64 central differences of L = sum(m * y^2) at b=2, n=6, for a
    non-orthogonal W (a trained W is no longer unitary)."""
    rng = np.random.default_rng(80)
    b, n = 2, 6
    W = gi.haar_orthogonal(b, rng) + 0.3 * rng.standard_normal((b, b))
    x = rng.standard_normal((2, b ** n))
    m = rng.uniform(0, 1, (2, b ** n))
    y = oracle.modes(W, x)
    dx, dW = oracle.grad(W, x, 2 * m * y)
    fdx, fdW = oracle.fd_grad_real(W, x, m)
    assert np.linalg.norm(dx - fdx) <= 1e-7 * np.linalg.norm(fdx)
    assert np.linalg.norm(dW - fdW) <= 1e-7 * np.linalg.norm(fdW)


def test_gradient_complex_conjugate_convention():
    """Complex W, x: dx and dW follow dL/dRe + i dL/dIm (PyTorch's
    convention), checked by central differences of each real coordinate."""
    rng = np.random.default_rng(81)
    b, n = 3, 3
    W = rand_c(rng, (b, b)) * 0.5
    x = rand_c(rng, b ** n)
    m = rng.uniform(0, 1, b ** n)

    def loss(W_, x_):
        return float(np.sum(m * np.abs(oracle.modes(W_, x_)) ** 2))

    y = oracle.modes(W, x)
    dx, dW = oracle.grad(W, x, 2 * m * y)
    h = 1e-6
    fdW = np.zeros_like(W)
    for idx in np.ndindex(b, b):
        for unit in (1.0, 1j):
            Wp = W.copy(); Wp[idx] += h * unit
            Wm = W.copy(); Wm[idx] -= h * unit
            fdW[idx] += unit * (loss(Wp, x) - loss(Wm, x)) / (2 * h)
    fdx = np.zeros_like(x)
    for i in range(b ** n):
        for unit in (1.0, 1j):
            xp = x.copy(); xp[i] += h * unit
            xm = x.copy(); xm[i] -= h * unit
            fdx[i] += unit * (loss(W, xp) - loss(W, xm)) / (2 * h)
    assert np.linalg.norm(dW - fdW) <= 1e-7 * np.linalg.norm(fdW)
    assert np.linalg.norm(dx - fdx) <= 1e-7 * np.linalg.norm(fdx)


def test_adjoint_identity():
    """<G x, g> = <x, G^H g> for a general complex W."""
    rng = np.random.default_rng(82)
    W = rand_c(rng, (4, 4))
    x = rand_c(rng, 4 ** 5)
    g = rand_c(rng, 4 ** 5)
    lhs = np.vdot(g, oracle.modes(W, x))
    rhs = np.vdot(oracle.adjoint(W, g), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ----------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(golden):
    """Each plausible mistake, planted in the oracle's use on the CPU, is
    caught by at least one of the pins above."""
    g3 = golden("e3_compression_u3_n3.txt")
    W3 = gi.u3(*g3["theta_phi_lambda"])
    Gp = np.vstack([g3[f"G_row{i}"] for i in range(8)])

    def close(a, b, tol):
        return np.allclose(a, b, atol=tol)

    # transposed W (Y = X W instead of X W^T in Algorithm 1)
    tol3 = 0.5e-3 * math.sqrt(2) + 1e-12
    assert not close(oracle.dense_matrix(W3.T, 3), Gp, tol3)
    # conjugated W
    assert not close(oracle.dense_matrix(W3.conj(), 3), Gp, tol3)
    # forward used where the adjoint is meant (E2)
    g2 = golden("e2_fourier_series_b2_n1.txt")
    W2 = np.vstack([g2["W_row0"], g2["W_row1"]]).astype(np.complex128)
    assert not close(oracle.modes(W2, g2["g"].astype(complex)) / math.sqrt(2), g2["C"], 1e-6)
    # digit-reversed output ordering (separable test with distinct factors)
    rng = np.random.default_rng(90)
    b, n = 3, 4
    W = rand_c(rng, (b, b))
    us = [rand_c(rng, b) for _ in range(n)]
    x = np.array([1.0 + 0j])
    ref = np.array([1.0 + 0j])
    for k in reversed(range(n)):
        x = np.kron(x, us[k])
        ref = np.kron(ref, W @ us[k])
    y = oracle.modes(W, x).reshape([b] * n)
    y_rev = np.transpose(y, axes=list(reversed(range(n)))).reshape(-1)
    assert not close(y_rev, ref, 1e-8)
    # a dropped mode (n-1 passes) breaks the E10 spectrum
    g10 = golden("e10_filter_u3_n4.txt")
    Wf = gi.u3(*g10["theta_phi_lambda"])
    psi = g10["Psi"] / np.linalg.norm(g10["Psi"])
    short = oracle.modes(Wf, psi.reshape(2, 8))   # two length-8 transforms
    assert not close(short.reshape(-1).real, g10["spectrum"], 5.1e-5)
    # sign error in the integer Hadamard breaks bit-exactness
    xi = np.random.default_rng(91).integers(-2 ** 15, 2 ** 15, size=2 ** 12)
    bad = oracle.modes_u32(np.array([[1, 1], [-1, 1]]), xi)
    assert not np.array_equal(bad, _hadamard_pm1_bigint(xi))


# ------------------------------------------------ heterogeneous transform

def test_mixed_mode_loop_is_the_kronecker_product():
    """Remark after Def. 2.3: G = W_0 (x) ... (x) W_{n-1} with b_k x b_k
    factors.  The mode loop equals numpy's Kronecker product for unequal
    radices (a transposed factor or a reversed factor order fails), reduces to
    the homogeneous transform for equal factors, and keeps norms for unitary
    factors."""
    rng = np.random.default_rng(31)
    for radices in ([2, 3], [3, 2, 5], [4, 2, 3, 2], [5, 7]):
        Ws = [gi.haar_unitary(b, rng) for b in radices]
        N = int(np.prod(radices))
        x = gi.complex_normal_x((3, N), rng, np.complex128)
        ref = oracle.kron_dense(Ws, x)
        np.testing.assert_allclose(oracle.modes_mixed(Ws, x), ref, atol=1e-12)
        assert not np.allclose(oracle.modes_mixed(Ws[::-1], x), ref, atol=1e-6)
        assert not np.allclose(oracle.modes_mixed([W.T for W in Ws], x), ref, atol=1e-6)
        np.testing.assert_allclose(np.linalg.norm(ref, axis=1), np.linalg.norm(x, axis=1), rtol=1e-12)
    W = gi.haar_unitary(3, rng)
    x = gi.complex_normal_x((2, 3 ** 5), rng, np.complex128)
    np.testing.assert_allclose(oracle.modes_mixed([W] * 5, x), oracle.modes(W, x), atol=1e-12)


def test_mixed_integer_route_wraps_like_python_ints():
    """The uint32 heterogeneous loop equals exact big-integer arithmetic with
    the Kronecker definition (remark after Def. 2.3), reduced mod 2^32, for
    values whose partial sums overflow 32 bits.  A reversed factor order and a
    transposed factor fail."""
    rng = np.random.default_rng(72)
    for radices in ([3, 2, 5, 4], [2, 2, 2, 2, 3], [7, 3]):
        Ws = [rng.integers(-2 ** 31, 2 ** 31, size=(b, b)) for b in radices]
        N = int(np.prod(radices))
        x = rng.integers(-2 ** 31, 2 ** 31, size=(2, N))
        G = np.array([[1]], dtype=object)
        for W in Ws:
            G = np.kron(G, W.astype(object))
        ref = np.array([[int(v) % (1 << 32) for v in G.dot(xv.astype(object))] for xv in x],
                       dtype=np.uint32)
        got = oracle.modes_mixed_u32(Ws, x)
        np.testing.assert_array_equal(got, ref)
        assert not np.array_equal(oracle.modes_mixed_u32(Ws[::-1], x), ref)
        assert not np.array_equal(oracle.modes_mixed_u32([Ws[0].T] + Ws[1:], x), ref)
    # equal factors reduce to the single-base integer loop
    W = rng.integers(-9, 10, size=(3, 3))
    x = rng.integers(-2 ** 31, 2 ** 31, size=3 ** 5)
    np.testing.assert_array_equal(oracle.modes_mixed_u32([W] * 5, x)[0], oracle.modes_u32(W, x))
