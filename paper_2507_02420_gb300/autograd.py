"""torch.autograd wrapper: y = G_N x with the library's hand-written adjoint.

GTTFunction.apply(x, W, n) takes x of shape [batch, N] on a CUDA device and a
b x b W (trainable).  The forward calls gtt_forward; the backward calls
gtt_backward, which returns dL/dx = (W^H)^{(x)n} dL/dy and dL/dW as a per-mode
reduction of fibre outer products (PyTorch's conjugate convention for complex
types).  W's values are copied to the host on every forward (the kernels read
W from their constant bank).
"""
from __future__ import annotations

import threading

import torch

from .api import Plan, dtype_code

_cache: dict = {}
_lock = threading.Lock()


def _plan_for(W: torch.Tensor, n: int, x: torch.Tensor) -> Plan:
    key = (int(W.shape[0]), int(n), x.dtype, int(x.shape[0]), x.device.index)
    with _lock:
        plan = _cache.get(key)
        if plan is None:
            plan = Plan(W.detach().cpu(), n, dtype_code(x.dtype), int(x.shape[0]))
            _cache[key] = plan
        else:
            plan.set_w(W.detach().cpu())
    return plan


class GTTFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, W, n):
        if x.dim() != 2:
            raise ValueError("x must have shape [batch, N]")
        x = x.contiguous()
        plan = _plan_for(W, n, x)
        y = plan.forward(x)
        ctx.save_for_backward(x, W)
        ctx.n = n
        return y

    @staticmethod
    def backward(ctx, gy):
        x, W = ctx.saved_tensors
        plan = _plan_for(W, ctx.n, x)
        need_dx, need_dW = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dx, dW = plan.backward(x, gy.contiguous(), need_dx=need_dx, need_dW=need_dW)
        if dW is not None:
            dW = dW.to(W.device, W.dtype)
        return dx, dW, None


def gtt(x: torch.Tensor, W: torch.Tensor, n: int) -> torch.Tensor:
    """Differentiable y = (W (x) ... (x) W) x along the last dimension."""
    return GTTFunction.apply(x, W, n)
