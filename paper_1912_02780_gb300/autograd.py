"""torch.autograd wrappers over the C ABI.

``lnz(T0, plan)`` returns ln Z / N of the HOTRG network built from the site
tensor T0 (a CUDA float64 tensor of shape (d0,)*4); its backward is the
library's hand-written reverse pass (SM Sec. B recursion / SM Sec. E chain
rule, plus the adjoint of the truncated eigensolve), which recomputes the
stage intermediates of every step from the checkpoints the forward kept.

``lnz_ising(beta, plan, J, h)`` does the same for the square-lattice Ising
model, differentiable in beta (a 0-dim tensor): the site tensor and its beta
derivative are built on the device by the library.

PyTorch supplies only device memory, the stream and the autograd graph; all
arithmetic runs in the CUDA library.  A plan holds the checkpoints of its
last forward, so each forward must be followed by its backward before the
same plan runs another forward.
"""
from __future__ import annotations

import torch

from . import Plan

__all__ = ["HotrgFunction", "IsingFunction", "lnz", "lnz_ising", "make_plan"]


def make_plan(d0: int, d_cut: int, n_steps: int, precision: str = "fp64", split_from_step: int = 1,
              fixed_w_grad: bool = False, device=None) -> Plan:
    """A plan bound to the current CUDA stream of ``device``."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    stream = torch.cuda.current_stream(dev).cuda_stream
    return Plan(d0, d_cut, n_steps, precision, split_from_step=split_from_step, want_grad=True,
                fixed_w_grad=fixed_w_grad, stream=stream)


class HotrgFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T0: torch.Tensor, plan: Plan):
        if T0.dtype != torch.float64 or not T0.is_cuda or T0.shape != (plan.d0,) * 4:
            raise ValueError("T0 must be a CUDA float64 tensor of shape (d0, d0, d0, d0)")
        T0c = T0.contiguous()
        out = torch.empty(plan.n_steps + 2, dtype=torch.float64, device=T0.device)
        plan.forward_device(T0c.data_ptr(), out.data_ptr())
        plan.sync()
        ctx.plan = plan
        ctx.shape = T0.shape
        ctx.device = T0.device
        return out[0].clone()

    @staticmethod
    def backward(ctx, grad_out):
        g = torch.empty(ctx.shape, dtype=torch.float64, device=ctx.device)
        ctx.plan.backward_device(g.data_ptr())
        ctx.plan.sync()
        return grad_out * g, None


class IsingFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta: torch.Tensor, plan: Plan, J: float, h: float):
        lnz_value, _, _ = plan.forward_ising(float(beta), J, h)
        ctx.plan = plan
        return torch.tensor(lnz_value, dtype=torch.float64, device=beta.device)

    @staticmethod
    def backward(ctx, grad_out):
        _, dbeta = ctx.plan.backward(want_dbeta=True)
        return grad_out * dbeta, None, None, None


def lnz(T0: torch.Tensor, plan: Plan) -> torch.Tensor:
    return HotrgFunction.apply(T0, plan)


def lnz_ising(beta: torch.Tensor, plan: Plan, J: float = 1.0, h: float = 0.0) -> torch.Tensor:
    return IsingFunction.apply(beta, plan, J, h)
