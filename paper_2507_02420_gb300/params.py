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

import torch

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
