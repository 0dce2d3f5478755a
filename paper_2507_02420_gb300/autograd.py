"""torch.autograd wrapper: y = G_N x with the library's hand-written adjoint.

GTTFunction.apply(x, W, n) takes x of shape [batch, N] on a CUDA device and a
b x b W (trainable).  The forward calls gtt_forward_saving where the plan's
schedules allow it (keeping the activation the backward would otherwise
recompute, one vector-sized buffer held until the backward), else
gtt_forward; the backward calls gtt_backward_saved or gtt_backward, which
return dL/dx = (W^H)^{(x)n} dL/dy and dL/dW as a per-mode reduction of fibre
outer products (PyTorch's conjugate convention for complex types).  The kernels read W from their constant bank, so its values have to
be on the host when a kernel is launched: the wrapper copies W to the host only
when it may differ from the last copy the plan took.  The plan's cache keeps a
detached alias of the W it copied (so that storage cannot be freed and reused
by another tensor) and the version counter it had; W is copied again when it
lives in another storage or when an in-place update has bumped the counter (an
optimizer step does).  A forward or backward with an unchanged W therefore
neither copies W nor waits for the device.  Changes that bypass the version
counter (writes through ``W.data``) are not seen: pass a fresh tensor instead
(``W.clone()``), as a finite-difference gradient check must.
"""
from __future__ import annotations

import threading

import torch

from ._lib import GTTError
from .api import Plan, dtype_code

_cache: dict = {}
_lock = threading.Lock()


def _plan_for(W: torch.Tensor, n: int, x: torch.Tensor) -> Plan:
    key = (int(W.shape[0]), int(n), x.dtype, int(x.shape[0]), x.device.index)
    with _lock:
        entry = _cache.get(key)
        if entry is None:
            plan = Plan(W.detach().cpu(), n, dtype_code(x.dtype), int(x.shape[0]))
            _cache[key] = [plan, W.detach(), W._version]
            return plan
        plan, held, version = entry
        if W.data_ptr() != held.data_ptr() or W.dtype != held.dtype or W._version != version:
            plan.set_w(W.detach().cpu())
            entry[1], entry[2] = W.detach(), W._version
    return plan


class GTTFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, W, n):
        if x.dim() != 2:
            raise ValueError("x must have shape [batch, N]")
        x = x.contiguous()
        plan = _plan_for(W, n, x)
        ckpt = None
        # keep the checkpoint only when a backward can follow
        if (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]) and getattr(plan, "_saving", True):
            try:
                y, ckpt = plan.forward_saving(x)
            except GTTError as e:
                if e.status != 2:  # GTT_ERR_UNSUPPORTED: this plan keeps no checkpoint
                    raise
                plan._saving = False
        if ckpt is None:
            y = plan.forward(x)
            ckpt = x.new_empty(0)
        ctx.save_for_backward(x, W, ckpt)
        ctx.n = n
        return y

    @staticmethod
    def backward(ctx, gy):
        x, W, ckpt = ctx.saved_tensors
        plan = _plan_for(W, ctx.n, x)
        need_dx, need_dW = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if ckpt.numel():
            dx, dW = plan.backward_saved(x, ckpt, gy.contiguous(), need_dx=need_dx, need_dW=need_dW)
        else:
            dx, dW = plan.backward(x, gy.contiguous(), need_dx=need_dx, need_dW=need_dW)
        if dW is not None:
            dW = dW.to(W.device, W.dtype)
        return dx, dW, None


def gtt(x: torch.Tensor, W: torch.Tensor, n: int) -> torch.Tensor:
    """Differentiable y = (W (x) ... (x) W) x along the last dimension."""
    return GTTFunction.apply(x, W, n)
