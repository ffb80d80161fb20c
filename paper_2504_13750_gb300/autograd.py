"""torch.autograd.Function wrappers around the discrete adjoint of the C ABI.

``rollout(grid, U0, n_steps, dt, ckpt_every)`` maps the initial conserved
state U^0 (a device tensor [nv, ny, nx]) to U^N after n fixed-dt steps. Its
forward runs janc_adjoint_forward (checkpoints kept on the device); its
backward receives dL/dU^N from whatever loss follows and runs
janc_adjoint_reverse, so any torch expression of U^N is differentiable with
respect to U^0. One rollout may be pending per grid at a time.

Both take ``store_faces`` to choose the adjoint mode (the forward's
linearisation kept in the segment stores, or recomputed in the reverse).

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


def _set_mode(grid, store_faces):
    if store_faces is not None:
        janc.janc_set_adjoint_mode(grid.handle, janc.ADJ_STORE_FACES if store_faces else janc.ADJ_RECOMPUTE)


def trajectory_loss(grid, T0, p, u, v, Y, n_steps, dt, ckpt_every=50, store_faces=None):
    """store_faces: True / False sets the grid's adjoint mode
    (janc_set_adjoint_mode: keep the forward's linearisation in the segment
    stores, or recompute it); None leaves the grid's mode as it is."""
    _set_mode(grid, store_faces)
    return JancTrajectory.apply(T0, grid, p, u, v, Y, n_steps, dt, ckpt_every)


class JancRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, grid, n_steps, dt, ckpt_every):
        if not (U0.is_cuda and U0.dtype == torch.float64 and U0.is_contiguous()):
            raise ValueError("U0 must be a contiguous float64 CUDA tensor")
        janc.janc_set_state(grid.handle, U0.detach())
        janc.janc_adjoint_forward(grid.handle, n_steps, dt, ckpt_every, janc.LOSS_SEEDED)
        UN = torch.empty_like(U0)
        janc.janc_get_state(grid.handle, UN, None)
        ctx.grid = grid
        return UN

    @staticmethod
    def backward(ctx, gUN):
        gU0 = torch.empty_like(gUN)
        janc.janc_adjoint_reverse(ctx.grid.handle, gUN.contiguous(), gU0)
        return gU0, None, None, None, None


def rollout(grid, U0, n_steps, dt, ckpt_every=50, store_faces=None):
    """store_faces: as for trajectory_loss."""
    _set_mode(grid, store_faces)
    return JancRollout.apply(U0, grid, n_steps, dt, ckpt_every)
