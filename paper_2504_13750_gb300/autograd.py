"""torch.autograd.Function around the discrete adjoint of the C ABI.

``trajectory_loss(grid, T0, p, u, v, Y, n_steps, dt, ckpt_every)`` loads the
initial state from primitive fields (device tensors) with the temperature
field T0 as the differentiable input, runs n fixed-dt steps and returns the
time-integrated mean end-wall pressure sum_n dt mean_j p(nx-1, j)^{n+1}.
When T0 requires a gradient the forward call runs janc_step_adjoint, whose
checkpoint-and-recompute reverse sweep yields dL/dU^0; janc_primitive_T_vjp
maps it to dL/dT0, which backward() scales by the incoming gradient. All
arithmetic runs in libjanc.so.
"""
from __future__ import annotations

import torch

from . import janc


class JancTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T0, grid, p, u, v, Y, n_steps, dt, ckpt_every):
        for t in (T0, p, u, v, Y):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("inputs must be contiguous float64 CUDA tensors")
        T0d = T0.detach()
        janc.janc_set_state_primitive(grid.handle, T0d, p, u, v, Y)
        if ctx.needs_input_grad[0]:
            dLdU0 = torch.empty((grid.nv, grid.ny, grid.nx), dtype=torch.float64, device=T0.device)
            loss = janc.janc_step_adjoint(grid.handle, n_steps, dt, ckpt_every, janc.LOSS_ENDWALL_P, None, dLdU0)
            dLdT = torch.empty_like(T0d)
            janc.janc_primitive_T_vjp(grid.handle, T0d, p, u, v, Y, dLdU0, dLdT)
            ctx.save_for_backward(dLdT)
        else:
            loss = janc.janc_step_adjoint(grid.handle, n_steps, dt, ckpt_every, janc.LOSS_ENDWALL_P, None, None)
        return torch.tensor(loss, dtype=torch.float64, device=T0.device)

    @staticmethod
    def backward(ctx, g):
        (dLdT,) = ctx.saved_tensors
        return g * dLdT, None, None, None, None, None, None, None, None


def trajectory_loss(grid, T0, p, u, v, Y, n_steps, dt, ckpt_every=50):
    return JancTrajectory.apply(T0, grid, p, u, v, Y, n_steps, dt, ckpt_every)
