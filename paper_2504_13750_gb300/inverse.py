"""Inverse problem of Sec. 6.2 in a synthetic form: recover the equivalence
ratio of the fresh propellant from two flow-field snapshots of a reacting
channel with a periodic circumferential direction, by gradient descent
(Adam) on the relative-error loss of Eq. 6.6 through the discrete adjoint.

Setting (the paper's injection model and its parameters are not printed, so
this stands in for them): x periodic (the unrolled circumference), a wall at
the bottom and a zero-gradient outlet at the top, the one-step global H2-O2
reaction on a gamma = 1.29 gas as an explicit source (JANC_CHEM_EXPLICIT).
A reacting front is developed from a hot igniter column at phi = 1; in that
snapshot the fresh-gas cells (water mass fraction below 1e-3) take the
mixture of equivalence ratio theta at the same T, p and velocity, which gives
U_0(theta). The loss compares U_n(theta) after n fixed-dt steps with
U_n(1.0):  L = ||U_n(theta) - U_n(1)|| / ||U_n(1)||. Its gradient is
<dL/dU_0, dU_0/dtheta>: dL/dU_0 from janc_adjoint_forward (which leaves U_n
for the loss) and janc_adjoint_reverse with the cotangent dL/dU_n, dU_0/dtheta
by a central difference of the (smooth) state set-up.

Everything runs through the C ABI (janc_*); torch holds device buffers and
runs the optimiser.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, janc

MECH = "global_h2o2_g129"
RU = 8.314472


def _h2o2_Y(mech, phi):
    """H2-O2 mass fractions at equivalence ratio phi (moles H2 : O2 = 2 phi : 1)."""
    M = dict(zip(mech["species"], mech["M"]))
    return inputs.premix_Y(mech, {"H2": 2.0 * phi * M["H2"], "O2": M["O2"]})


class ChannelInverse:
    def __init__(self, nx=250, ny=100, Lx=0.10, Ly=0.04, n_steps=100, dev_steps=400, ckpt_every=None, seed=0,
                 store_faces=True):
        """ckpt_every=None keeps the whole trajectory on the device (one
        segment: the reverse sweep recomputes nothing); about
        (4 n_steps + 2) x 16 x nx x ny x 8 bytes. store_faces also keeps the
        face derivatives of every stage (janc_set_adjoint_mode
        ADJ_STORE_FACES): 24 nv ((nx+1) ny + (ny+1) nx) x 8 bytes more per
        step, and a reverse sweep that does not recompute them."""
        import torch

        self.torch = torch
        self.mech = inputs.load_mechanism(MECH)
        ckpt_every = n_steps if ckpt_every is None else ckpt_every
        self.nx, self.ny, self.n_steps, self.ckpt = nx, ny, n_steps, ckpt_every
        dx, dy = Lx / nx, Ly / ny
        self.grid = inputs.grid_dict(nx, ny, dx, dy, [2, 2, 0, 1])
        self.g = janc.Grid.from_grid_dict(self.mech, self.grid, chemistry=janc.CHEM_EXPLICIT)
        self.nv = self.g.nv
        # developed reacting state at phi = 1 from a hot igniter column
        rng = np.random.default_rng(seed)
        x = (np.arange(nx) + 0.5) * dx
        y = (np.arange(ny) + 0.5) * dy
        X, Yg = np.meshgrid(x, y)
        T = np.full((ny, nx), 300.0)
        p = np.full((ny, nx), inputs.ATM)
        hot = X < 0.05 * Lx
        T[hot] = 2000.0
        p[hot] = 20.0 * inputs.ATM
        T *= 1.0 + 0.01 * rng.standard_normal((ny, nx)) * ~hot
        Y1 = _h2o2_Y(self.mech, 1.0)
        Yf = np.repeat(np.repeat(Y1[:, None, None], ny, 1), nx, 2)
        z = np.zeros((ny, nx))
        self.g.set_primitive(T, p, z, z, np.ascontiguousarray(Yf))
        self.g.step(dev_steps, cfl=0.5)
        U, T = self.g.get_state()
        rho = U[0]
        Yc = U[4:] / rho                      # carried mass fractions
        Yall = np.concatenate([Yc, 1.0 - Yc.sum(0, keepdims=True)])
        W = np.tensordot(1.0 / np.asarray(self.mech["M"]), Yall, axes=1)
        self.T0 = T
        self.p0 = rho * RU * W * T
        self.u0 = U[1] / rho
        self.v0 = U[2] / rho
        self.Y0 = Yall
        self.fresh = Yall[-1] < 1e-3
        # the snapshot's fields stay on the device; only Y(theta) changes
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        self._dT0, self._dp0, self._du0, self._dv0 = (dev(a) for a in (self.T0, self.p0, self.u0, self.v0))
        self._dY0 = dev(Yall)
        self._dfresh = dev(self.fresh)
        # fixed dt: the CFL dt of the snapshot
        self.set_theta(1.0)
        _, self.dt = self.g.step(1, cfl=0.5, want_time=True)
        self.set_theta(1.0)
        self.target = self._forward()
        self.tnorm = float(self.torch.linalg.vector_norm(self.target))
        janc.janc_set_adjoint_mode(self.g.handle, janc.ADJ_STORE_FACES if store_faces else janc.ADJ_RECOMPUTE)
        nbytes = janc.janc_adjoint_workspace_bytes(self.g.handle, n_steps, ckpt_every)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self.wp = (self.ws.data_ptr() + 255) & ~255
        self.nbytes = nbytes

    def set_theta(self, theta):
        """Loads U_0(theta): the snapshot with the fresh-gas cells at
        equivalence ratio theta (fields on the device, no host copies)."""
        Yth = self.torch.from_numpy(_h2o2_Y(self.mech, theta)).cuda()
        Y = self.torch.where(self._dfresh[None], Yth[:, None, None], self._dY0).contiguous()
        janc.janc_set_state_primitive(self.g.handle, self._dT0, self._dp0, self._du0, self._dv0, Y)

    def state(self):
        U = self.torch.empty((self.nv, self.ny, self.nx), dtype=self.torch.float64, device="cuda")
        janc.janc_get_state(self.g.handle, U, None)
        return U

    def _forward(self):
        self.g.step(self.n_steps, dt=self.dt)
        return self.state()

    def loss_and_grad(self, theta):
        """L(theta) and dL/dtheta: one checkpointed forward (janc_adjoint_forward),
        the loss and its cotangent dL/dU_n from U_n, one reverse sweep
        (janc_adjoint_reverse), then the contraction with dU_0/dtheta."""
        torch = self.torch
        self.set_theta(theta)
        janc.janc_adjoint_forward(self.g.handle, self.n_steps, self.dt, self.ckpt, janc.LOSS_SEEDED, self.wp,
                                  self.nbytes)
        Un = self.state()
        diff = Un - self.target
        dn = float(torch.linalg.vector_norm(diff))
        L = dn / self.tnorm
        seed = (diff / (dn * self.tnorm)).contiguous() if dn > 0 else torch.zeros_like(diff)
        gU0 = torch.empty_like(Un)
        janc.janc_adjoint_reverse(self.g.handle, seed, gU0)
        h = 1e-4
        self.set_theta(theta + h)
        Up = self.state()
        self.set_theta(theta - h)
        Um = self.state()
        dU0 = (Up - Um) / (2.0 * h)
        return L, float(torch.sum(gU0 * dU0))

    def optimize(self, theta0, iters=100, lr=0.01):
        """Adam on theta; returns the history [(theta, L)] and the wall time."""
        torch = self.torch
        th = torch.tensor([float(theta0)], dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([th], lr=lr)
        hist = []
        t0 = time.perf_counter()
        for _ in range(iters):
            L, gth = self.loss_and_grad(float(th.detach()))
            hist.append((float(th.detach()), L))
            opt.zero_grad()
            th.grad = torch.tensor([gth], dtype=torch.float64)
            opt.step()
        torch.cuda.synchronize()
        return hist, time.perf_counter() - t0

    def close(self):
        self.g.close()
        self.ws = None
