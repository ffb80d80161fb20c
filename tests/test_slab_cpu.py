"""The multi-rank x-slab path on CPU ranks (gloo): the partition, the halo
exchange and the all-reduce max of the LF speeds of paper_2504_13750_gb300.slab
(the code a rank runs around janc_slab_create), checked with host buffers.

Each rank takes its columns of one state (slab.partition), exchanges its 3
edge columns with its neighbours (TorchExchange.exchange) and the max of its
LF speeds (TorchExchange.allreduce_max), then evaluates the right-hand side of
Eq. 4.10 on its columns with the oracle's ghosted form, the x ghosts taken
from what it received. Put together, the ranks' L must equal the oracle's
whole-domain L bit for bit, as the paper's N-device runs equal one device:
any wrong neighbour, column order, side or missed max fails it. World sizes
2 and 3, walls and a periodic x axis (where, with 2 ranks, both neighbours of
a rank are the same rank). No GPU is involved."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NX, NY = 24, 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _state(bc):
    import oracle as orc
    from paper_2504_13750_gb300 import inputs

    mech = inputs.load_mechanism("h2air_synth")
    st = inputs.tube(mech, NX, NY, Lx=0.05 * NX / 256, perturb_seed=3, aspect=1.4)
    rng = np.random.default_rng(9)
    st["T"] = st["T"] + rng.normal(0.0, 5.0, st["T"].shape)
    st["u"] = rng.normal(0.0, 90.0, (NY, NX))
    st["v"] = rng.normal(0.0, 90.0, (NY, NX))
    st["grid"]["bc"] = list(bc)
    U = orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])
    return mech, st, U


def _ghosted(U, T, lo, hi, bc):
    """The rank's columns with 3 ghost layers: x ghosts from the received
    halos (planes U..., T) or the physical boundary, y ghosts physical (slip
    walls: mirror with the normal momentum negated)."""
    nv, ny, w = U.shape
    P = np.full((nv, ny + 6, w + 6), np.nan)
    PT = np.full((ny + 6, w + 6), np.nan)
    P[:, 3:3 + ny, 3:3 + w], PT[3:3 + ny, 3:3 + w] = U, T
    for side, recv in ((0, lo), (1, hi)):
        cols = slice(0, 3) if side == 0 else slice(w + 3, w + 6)
        if recv is not None:
            H = recv.reshape(nv + 1, ny, 3)
            P[:, 3:3 + ny, cols], PT[3:3 + ny, cols] = H[:nv], H[nv]
        else:
            assert bc[side] == 0
            src = np.array([2, 1, 0]) if side == 0 else np.array([w - 1, w - 2, w - 3])
            P[:, 3:3 + ny, cols], PT[3:3 + ny, cols] = U[:, :, src], T[:, src]
            P[1, 3:3 + ny, cols] *= -1.0
    assert bc[2] == 0 and bc[3] == 0
    for rows, src in ((slice(0, 3), np.array([2, 1, 0])), (slice(ny + 3, ny + 6), np.array([ny - 1, ny - 2, ny - 3]))):
        P[:, rows, 3:3 + w], PT[rows, 3:3 + w] = U[:, src, :], T[src, :]
        P[2, rows, 3:3 + w] *= -1.0
    return P, PT


def _rank(rank, world, port, bc, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle as orc
    from paper_2504_13750_gb300 import slab

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mech, st, U = _state(bc)
        x0, w = slab.partition(NX, world)[rank]
        comm = slab.TorchExchange(rank, world, periodic=bc[0] == 2)
        Ul = np.ascontiguousarray(U[:, :, x0:x0 + w])
        Tl = np.ascontiguousarray(st["T"][:, x0:x0 + w])
        planes = np.concatenate([Ul, Tl[None]])  # the halo layout [plane][ny][3]
        send_lo = torch.from_numpy(np.ascontiguousarray(planes[:, :, :3]).ravel())
        send_hi = torch.from_numpy(np.ascontiguousarray(planes[:, :, w - 3:]).ravel())
        recv_lo = torch.full_like(send_lo, float("nan"))
        recv_hi = torch.full_like(send_hi, float("nan"))
        comm.exchange(send_lo, send_hi, recv_lo, recv_hi)
        bits = np.asarray(orc.lf_alpha(mech, Ul, Tl), dtype=np.float64).view(np.int64).copy()
        a2 = torch.from_numpy(bits)
        comm.allreduce_max(a2)
        alpha = a2.numpy().view(np.float64)
        P, PT = _ghosted(Ul, Tl, recv_lo.numpy() if comm.lo is not None else None,
                         recv_hi.numpy() if comm.hi is not None else None, bc)
        g = st["grid"]
        L = orc.rhs_ghosted(mech, w, NY, g["dx"], g["dy"], P, PT, alpha)
        out[rank] = (x0, L, alpha.copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,bc", [(2, (0, 0, 0, 0)), (2, (2, 2, 0, 0)), (3, (0, 0, 0, 0)), (3, (2, 2, 0, 0))])
def test_ranks_exchange_halos_and_alpha_like_one_domain(world, bc):
    import oracle as orc

    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, bc, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    mech, st, U = _state(bc)
    L0, _, _, al0 = orc.rhs(mech, st["grid"], U, st["T"])
    L = np.concatenate([res[r][1] for r in range(world)], axis=2)
    assert [res[r][0] for r in range(world)] == sorted(res[r][0] for r in range(world))
    for r in range(world):
        assert np.array_equal(res[r][2], al0)
    assert np.array_equal(L, L0)


def test_partition_and_neighbours():
    from paper_2504_13750_gb300 import janc, slab

    for nx, world in ((4096, 3), (100, 7), (9, 3), (24, 1)):
        parts = slab.partition(nx, world)
        assert parts[0][0] == 0 and sum(w for _, w in parts) == nx
        assert all(a + w == b for (a, w), (b, _) in zip(parts, parts[1:]))
        assert max(w for _, w in parts) - min(w for _, w in parts) <= 1
        assert [w for _, w in parts] == sorted((w for _, w in parts), reverse=True)
    with pytest.raises(janc.JancError):
        slab.partition(11, 4)  # a slab of 2 columns cannot hold a neighbour's halo
    assert slab.neighbours(0, 3, False) == (None, 1)
    assert slab.neighbours(2, 3, False) == (1, None)
    assert slab.neighbours(0, 3, True) == (2, 1)
    assert slab.neighbours(0, 2, True) == (1, 1)
    assert slab.neighbours(0, 1, True) == (0, 0)
    assert slab.neighbours(0, 1, False) == (None, None)


def test_single_rank_periodic_exchanges_with_itself():
    from paper_2504_13750_gb300 import slab

    comm = slab.TorchExchange(0, 1, periodic=True)
    a, b = torch.arange(6.0), torch.arange(6.0) + 10
    ra, rb = torch.zeros(6), torch.zeros(6)
    comm.exchange(a, b, ra, rb)
    assert torch.equal(ra, b) and torch.equal(rb, a)
    x = torch.tensor([3, 5])
    comm.allreduce_max(x)
    assert x.tolist() == [3, 5]
