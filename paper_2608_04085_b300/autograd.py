"""torch.autograd wrapper: forward -> rt_forward, backward -> rt_gradient.

Argument marshalling only; both directions run in the CUDA library. The
perturbation tensor must be a contiguous CUDA float64 tensor in the
concatenated [instance][component][ny][nx] layout of the context.
"""
from __future__ import annotations

import torch

from . import Context


class CnopObjective(torch.autograd.Function):
    """J(v0) for every instance of a Context (Sec. 3.1, Eq. objective)."""

    @staticmethod
    def forward(ctx, v0: torch.Tensor, rt: Context):
        J, _, _ = rt.forward(v0)
        ctx.save_for_backward(v0)
        ctx.rt = rt
        return torch.as_tensor(J, dtype=torch.float64, device=v0.device)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        (v0,) = ctx.saved_tensors
        rt: Context = ctx.rt
        _, g, _ = rt.gradient(v0.detach())
        scale = torch.empty_like(g)
        for i, (off, n) in enumerate(zip(rt.offsets, rt.sizes)):
            scale[off:off + n] = gJ[i]
        return g * scale, None


def objective(v0: torch.Tensor, rt: Context) -> torch.Tensor:
    return CnopObjective.apply(v0, rt)
