"""One x-slab of a domain per rank (arXiv 2504.13750, Sec. 4.4, Fig. 3).

A ``Slab`` is the C ABI's stand-alone slab (``janc_slab_create``): the rank's
columns of the domain as a grid whose step calls back into Python after every
state-producing phase. The callback moves the packed edge columns to the
neighbouring ranks and takes the max of the LF speeds over all ranks through
an exchanger; ``TorchExchange`` does both with torch.distributed (NCCL for
CUDA tensors, gloo for host tensors). This module only marshals: the packing,
the halo reads and every step of the method run in libjanc.so.
"""
from __future__ import annotations

from . import janc


def partition(nx: int, world: int):
    """[(x0, nx_local)] of every rank: contiguous column ranges, the first
    nx % world ranks one column wider (janc_slab_partition)."""
    return [janc.janc_slab_partition(nx, world, k) for k in range(world)]


def neighbours(rank: int, world: int, periodic: bool):
    """(low, high) neighbour ranks of `rank`, None where the side is the
    domain's physical boundary; a periodic x axis joins the ends."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return lo, hi


class TorchExchange:
    """Halo exchange and LF-speed max of one rank through torch.distributed.

    exchange(): the low neighbour's send_hi arrives in recv_lo and the high
    neighbour's send_lo in recv_hi. Per neighbour the messages are posted in
    the order (send_hi, recv_lo, send_lo, recv_hi), so that when both
    neighbours are the same rank (two ranks on a periodic axis) the two
    messages between them still pair up correctly under in-order matching.
    A single rank on a periodic axis exchanges with itself by copies.

    allreduce_max(): the LF speeds travel as the int64 view of the bit
    patterns of non-negative doubles, whose integer order is their order as
    doubles, so the max is exact.
    """

    def __init__(self, rank: int, world: int, periodic: bool, group=None):
        self.rank, self.world, self.group = int(rank), int(world), group
        self.lo, self.hi = neighbours(self.rank, self.world, bool(periodic))

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch.distributed as dist

        if self.world == 1:
            if self.lo is not None:
                recv_lo.copy_(send_hi)
                recv_hi.copy_(send_lo)
            return
        ops = []
        if self.hi is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, self.hi, self.group))
        if self.lo is not None:
            ops.append(dist.P2POp(dist.irecv, recv_lo, self.lo, self.group))
        if self.lo is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, self.lo, self.group))
        if self.hi is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, self.hi, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()

    def allreduce_max(self, alpha2):
        import torch.distributed as dist

        if self.world > 1:
            dist.all_reduce(alpha2, op=dist.ReduceOp.MAX, group=self.group)


class Slab:
    """This rank's slab of the domain `grid` (a grid dict: nx, ny, dx, dy, bc,
    ...) on the current CUDA device and stream, exchanging through `comm`
    (a TorchExchange, or any object with the same two methods). The buffers
    the callback moves are CUDA tensors owned here."""

    def __init__(self, mech: dict, grid: dict, rank: int, world: int, comm, chemistry=True, stream=None):
        import torch

        self.mech = janc.Mechanism(mech)
        self.nv = self.mech.ns + 3
        self.desc = janc.make_desc(grid["nx"], grid["ny"], grid["dx"], grid["dy"], grid["bc"], chemistry=chemistry,
                                   weno_eps=grid.get("weno_eps", 1e-6), newton_tol=grid.get("newton_tol", 1e-12),
                                   newton_maxit=grid.get("newton_maxit", 50))
        self.x0, self.nx = partition(grid["nx"], world)[rank]
        self.ny = int(grid["ny"])
        self.comm = comm
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = janc.janc_slab_halo_doubles(self.desc, self.mech)
        f64 = dict(dtype=torch.float64, device="cuda")
        self.send_lo, self.send_hi = torch.zeros(h, **f64), torch.zeros(h, **f64)
        self.recv_lo, self.recv_hi = torch.zeros(h, **f64), torch.zeros(h, **f64)
        self.alpha2 = torch.zeros(2, dtype=torch.int64, device="cuda")
        self._errors = []
        self._fn = janc.JANC_EXCHANGE_FN(self._exchange)
        self._x = janc.janc_slab_exchange(self.send_lo.data_ptr(), self.send_hi.data_ptr(), self.recv_lo.data_ptr(),
                                          self.recv_hi.data_ptr(), self.alpha2.data_ptr(), self._fn, None)
        local = janc.make_desc(self.nx, self.ny, grid["dx"], grid["dy"], grid["bc"], chemistry=chemistry)
        nbytes = janc.janc_workspace_bytes(local, self.mech)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self.workspace.data_ptr() + 255) & ~255
        with torch.cuda.stream(self.stream):
            self.handle = janc.janc_slab_create(self.desc, self.mech, self.x0, self.nx, self._x, aligned, nbytes,
                                                self.stream.cuda_stream)

    def _exchange(self, user, stream):
        try:
            self.comm.exchange(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi)
            self.comm.allreduce_max(self.alpha2)
            return 0
        except Exception as e:  # reported through JANC_E_EXCHANGE
            self._errors.append(e)
            return 1

    def _call(self, f, *a, **k):
        import torch

        with torch.cuda.stream(self.stream):
            try:
                return f(*a, **k)
            except janc.JancError:
                if self._errors:
                    raise self._errors[-1]
                raise

    def set_primitive(self, T, p, u, v, Y):
        """This slab's columns of the primitive fields (its own arrays)."""
        self._call(janc.janc_set_state_primitive, self.handle, T, p, u, v, Y)

    def set_state(self, U, T0=None):
        self._call(janc.janc_set_state, self.handle, U, T0)

    def step(self, n, dt=0.0, cfl=0.0, want_time=False):
        return self._call(janc.janc_step, self.handle, n, dt=dt, cfl=cfl, want_time=want_time)

    def get_state(self, check=True):
        import numpy as np

        U = np.zeros((self.nv, self.ny, self.nx))
        T = np.zeros((self.ny, self.nx))
        self._call(janc.janc_get_state, self.handle, U, T, check=check)
        return U, T

    def columns(self):
        return self.x0, self.nx

    def status(self):
        return janc.janc_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            janc.janc_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
