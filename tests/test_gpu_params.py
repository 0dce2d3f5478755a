"""Tuning W = U3(theta, phi, lambda) through the hand-written backward
(Sec. 4.2, function encoding): the parameter gradient of the retained-set
energy against FP64 central finite differences of the oracle, and gradient
ascent of the compression fidelity from the Hadamard point."""
import math

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


def oracle_energy(params, x, support):
    c = oracle.modes(gi.u3(*params), x.astype(np.complex128))
    return float(sum(np.sum(np.abs(c[b, support[b]]) ** 2) for b in range(x.shape[0])))


@pytest.mark.parametrize("n,k", [(4, 4), (8, 16), (10, 3)])
def test_parameter_gradient_matches_finite_differences(g, n, k):
    rng = np.random.default_rng(9950 + n)
    x = np.stack([gi.function_encoding_signal(n),
                  gi.complex_normal_x((2 ** n,), rng, np.complex128)]).astype(np.complex128)
    x[1] /= np.linalg.norm(x[1])
    p0 = (0.7, 0.4, 2.3)
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    W = g.params.u3(t[0], t[1], t[2])
    plan = g.Plan(W.detach(), n, "c128", 2)
    xd = torch.from_numpy(x).cuda()
    support, _ = plan.compress(xd, k)
    E = g.params.support_energy(xd, W, n, support).sum()
    (grad,) = torch.autograd.grad(E, t)
    sup = support.cpu().numpy()
    assert abs(float(E.detach()) - oracle_energy(p0, x, sup)) <= 1e-12
    h = 1e-6
    for i in range(3):
        lo, hi = list(p0), list(p0)
        lo[i] -= h
        hi[i] += h
        fd = (oracle_energy(hi, x, sup) - oracle_energy(lo, x, sup)) / (2 * h)
        assert abs(float(grad[i]) - fd) <= 1e-7 + 1e-6 * abs(fd), (i, float(grad[i]), fd)


def test_fidelity_ascent_from_the_hadamard_point(g):
    """U3(pi/2, 0, pi) is the Hadamard matrix; ascent from there with the
    retained set updated every step ends at least as high."""
    n, k = 6, 4
    x = torch.from_numpy(gi.function_encoding_signal(n).astype(np.complex128)[None, :]).cuda()
    H = torch.tensor(gi.hadamard_w(True), dtype=torch.complex128)
    assert torch.allclose(g.params.u3(*[torch.tensor(v, dtype=torch.float64) for v in (math.pi / 2, 0.0, math.pi)]),
                          H, atol=1e-15)
    params, hist = g.params.fit_u3(x, n, k, steps=40, lr=0.5)
    hplan = g.Plan(H, n, "c128", 1)
    _, hv = hplan.compress(x, k)
    F_h = float((hv.abs() ** 2).sum())
    assert abs(hist[0] - F_h) <= 1e-12
    assert hist[-1] >= F_h - 1e-12 and max(hist) > F_h + 1e-3
    assert all(math.isfinite(v) for v in hist)
    assert all(0.0 < v <= 1.0 + 1e-12 for v in hist)
