"""Tunable parameterisations of W and the function-encoding objective.

The function-encoding section of the paper (Sec. 4.2) tunes the GTT through
the parameters of W = U3(theta, phi, lambda) (b = 2) so that a discretised
signal becomes sparse in the transformed domain.  With the retained index set
S (the k largest coefficients) and the truncated spectrum re-normalised before
the inverse transform, as in the compression protocol of Sec. 4.1.5, the
reconstruction fidelity for unitary G and normalised psi is
F = sum_{j in S} |(G psi)_j|^2 (this reproduces the printed Hadamard
fidelities there; the printed GTT fidelities are F^2).  For a fixed S, F is
smooth in the parameters; its gradient runs through the library's forward and
hand-written backward (GTTFunction), and torch's autograd takes dL/dW to the
parameters.
"""
from __future__ import annotations

import math

import torch

from .api import Plan
from .autograd import gtt


def u3(theta: torch.Tensor, phi: torch.Tensor, lam: torch.Tensor, dtype=torch.complex128) -> torch.Tensor:
    """U3(theta, phi, lambda), the general 2x2 unitary of the paper's Eq. U3:
    [[cos(t/2), -e^{i l} sin(t/2)], [e^{i p} sin(t/2), e^{i(p+l)} cos(t/2)]].
    Differentiable in the three (real, 0-dimensional) parameters."""
    c, s = torch.cos(theta / 2), torch.sin(theta / 2)
    el, ep = torch.exp(1j * lam), torch.exp(1j * phi)
    row0 = torch.stack([c.to(dtype), (-el * s).to(dtype)])
    row1 = torch.stack([(ep * s).to(dtype), (ep * el * c).to(dtype)])
    return torch.stack([row0, row1])


def support_energy(x: torch.Tensor, W: torch.Tensor, n: int, support: torch.Tensor) -> torch.Tensor:
    """sum over j in `support` of |(G_N x)_j|^2 for every vector of x ([batch, N],
    CUDA); `support` is a [batch, k] index tensor.  With unitary W and unit
    vectors x this is the compression fidelity F of the retained set."""
    c = gtt(x, W.to(x.device), n)
    kept = torch.gather(c, 1, support.to(x.device))
    return (kept.abs() ** 2).sum(dim=1)


def fit_u3(x: torch.Tensor, n: int, k: int, steps: int = 40, lr: float = 0.5,
           init=(math.pi / 2, 0.0, math.pi)):
    """Gradient ascent of the compression fidelity over (theta, phi, lambda)
    for b = 2 (step 5 of the function-encoding procedure, Sec. 4.2, with a
    gradient method in place of a bounded quasi-Newton search).  Every step
    takes the retained set S from gtt_compress at the current parameters and
    the gradient of F = sum_{j in S} |(G_N x)_j|^2 from the library's backward.
    x: [batch, 2^n] complex128 CUDA tensor of unit vectors.  The default start
    U3(pi/2, 0, pi) is the Hadamard matrix.  Returns (parameters, fidelity of
    every step); the fidelities are summed over the batch."""
    t = torch.tensor(init, dtype=torch.float64, requires_grad=True)
    plan = Plan(u3(*t.detach()), n, "c128", int(x.shape[0]))
    history = []
    for _ in range(steps):
        W = u3(t[0], t[1], t[2])
        plan.set_w(W.detach())
        support, _ = plan.compress(x, k)
        F = support_energy(x, W, n, support).sum()
        history.append(float(F.detach()))
        (grad,) = torch.autograd.grad(F, t)
        with torch.no_grad():
            t += lr * grad
    return t.detach(), history
