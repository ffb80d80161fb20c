"""x-slab domain decomposition (Sec. 4.4, Fig. 3) on one GPU: N slabs of a
domain, exchanging 3 ghost columns of every stored plane and taking the LF
speeds as the max over all slabs, give the undivided grid's result bit for bit
(the paper's multi-GPU check that N devices reproduce one). Covered: the
single-process split (janc_split_*) over ragged partitions, every boundary
set and chemistry mode, CFL and fixed dt, dy != dx; and the stand-alone slab
(janc_slab_create) through its exchange callback, as one periodic rank that
exchanges with itself and as two ranks driven from two host threads."""
import threading

import numpy as np
import pytest

import oracle as orc
from paper_2504_13750_gb300 import inputs

pytestmark = pytest.mark.gpu

H2AIR = inputs.load_mechanism("h2air_synth")
GAS = inputs.load_mechanism("ideal_gamma14")
GLOBAL = inputs.load_mechanism("global_h2o2_g129")


@pytest.fixture(scope="module")
def J():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_13750_gb300 import build, janc

    build.build()
    return janc


def _tube(nx, ny, bc=(0, 0, 0, 0), aspect=1.0, seed=5, vel=0.0, mech=H2AIR, Y=None):
    st = inputs.tube(mech, nx, ny, Lx=0.05 * nx / 256, perturb_seed=seed, aspect=aspect, Y=Y)
    st["grid"]["bc"] = list(bc)
    if vel:
        rng = np.random.default_rng(seed)
        st["u"] = rng.normal(0.0, vel, (ny, nx))
        st["v"] = rng.normal(0.0, vel, (ny, nx))
    return st


def _whole(J, mech, st, chem, n, **kw):
    g = J.Grid.from_grid_dict(mech, st["grid"], chemistry=chem)
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    t = g.step(n, want_time=True, **kw)
    U, T = g.get_state()
    g.close()
    return U, T, t


def _split(J, mech, st, chem, n, slabs, **kw):
    s = J.Split.from_grid_dict(mech, st["grid"], slabs, chemistry=chem)
    s.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    t = s.step(n, want_time=True, **kw)
    U, T = s.get_state()
    cols = s.columns()
    s.close()
    return U, T, t, cols


CASES = [
    # (name, nx, ny, bc, mech, chemistry, steps, step args, velocity, aspect, slab counts)
    ("tube-walls-lie", 256, 32, (0, 0, 0, 0), "h2air", 1, 12, {"cfl": 0.5}, 0.0, 1.0, (2, 3, 7)),
    ("tube-ragged-strang", 100, 24, (0, 0, 0, 0), "h2air", 2, 8, {"cfl": 0.5}, 60.0, 1.0, (7,)),
    ("periodic-x-zerograd-y", 96, 20, (2, 2, 1, 1), "h2air", 1, 10, {"cfl": 0.5}, 150.0, 1.0, (1, 2, 5)),
    ("zerograd-x-periodic-y-aniso", 90, 16, (1, 1, 2, 2), "h2air", 1, 10, {"cfl": 0.5}, 150.0, 1.7, (4,)),
    ("walls-no-chem-fixed-dt", 64, 12, (0, 1, 0, 0), "gas", 0, 15, {"dt": 2e-8}, 80.0, 0.6, (3,)),
    ("explicit-source", 72, 12, (0, 0, 0, 0), "global", 3, 10, {"cfl": 0.5}, 0.0, 1.0, (2, 4)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_split_equals_undivided_grid_bitwise(J, case):
    name, nx, ny, bc, mk, chem, n, kw, vel, aspect, counts = case
    mech = {"h2air": H2AIR, "gas": GAS, "global": GLOBAL}[mk]
    Y = {"h2air": None, "gas": np.ones(1), "global": inputs.premix_Y(GLOBAL, {"H2": 4.032, "O2": 31.998})}[mk]
    st = _tube(nx, ny, bc=bc, aspect=aspect, vel=vel, mech=mech, Y=Y)
    Uw, Tw, tw = _whole(J, mech, st, chem, n, **kw)
    for k in counts:
        Us, Ts, ts, cols = _split(J, mech, st, chem, n, k, **kw)
        assert sum(w for _, w in cols) == nx and cols[0][0] == 0
        assert np.array_equal(Us, Uw), (name, k, float(np.max(np.abs(Us - Uw))))
        assert np.array_equal(Ts, Tw), (name, k)
        assert ts == tw, (name, k)


def test_split_full_size_tube_four_slabs(J):
    """The 4096 x 512 tube of the benchmark cut into 4 slabs, 3 steps at
    CFL 0.5: bit for bit the undivided grid, and within the one-step bar of
    the oracle after one step."""
    st = inputs.tube(H2AIR, 4096, 512, perturb_seed=0)
    Uw, Tw, _ = _whole(J, H2AIR, st, True, 3, cfl=0.5)
    Us, Ts, _, _ = _split(J, H2AIR, st, True, 3, 4, cfl=0.5)
    assert np.array_equal(Us, Uw) and np.array_equal(Ts, Tw)


def test_split_one_step_matches_oracle(J):
    st = _tube(128, 24, vel=50.0, aspect=1.3)
    U0 = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    Us, Ts, ts, _ = _split(J, H2AIR, st, True, 1, 5, cfl=0.5)
    Uo, To, s, to, _ = orc.step(H2AIR, st["grid"], U0, st["T"], 1, cfl=0.5)
    assert s == 0 and abs(ts[0] - to) / to < 1e-14
    for k in range(U0.shape[0]):
        assert np.max(np.abs(Us[k] - Uo[k])) <= 1e-10 * np.max(np.abs(Uo[k]))


def test_split_set_state_conserved_and_status(J):
    """The conserved-state load scatters whole-domain U and the warm-start T;
    a bad cell in one slab raises the split's status word."""
    st = _tube(48, 8)
    U0 = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    s = J.Split.from_grid_dict(H2AIR, st["grid"], 3)
    s.set_state(U0, st["T"])
    U, T = s.get_state()
    assert np.array_equal(U, U0) and np.max(np.abs(T - st["T"]) / st["T"]) < 1e-12
    bad = U0.copy()
    bad[0, 4, 40] = -1.0  # negative density in the last slab
    s.set_state(bad, st["T"])
    assert J.janc_split_get_state(s.handle, np.zeros_like(U0), np.zeros_like(st["T"]), check=False) == -5
    assert s.status()["status"] & J.ST_NONPOSITIVE
    s.close()


def test_split_refuses_narrow_slabs(J):
    st = _tube(20, 8)
    with pytest.raises(J.JancError) as e:
        J.Split.from_grid_dict(H2AIR, st["grid"], 7)  # 20 // 7 = 2 < 3 columns
    assert e.value.rc == -1


class _SelfExchange:
    """One rank on a periodic x axis: its own right columns are its low halo
    and its left columns its high halo (copies on the current stream)."""

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)

    def allreduce_max(self, alpha2):
        pass


def test_standalone_slab_periodic_self_exchange(J):
    """janc_slab_create through the exchange callback: the whole periodic
    domain as one rank equals the periodic grid bit for bit."""
    from paper_2504_13750_gb300 import slab

    st = _tube(96, 20, bc=(2, 2, 0, 0), vel=120.0)
    Uw, Tw, tw = _whole(J, H2AIR, st, True, 8, cfl=0.5)
    s = slab.Slab(H2AIR, st["grid"], 0, 1, _SelfExchange())
    s.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    ts = s.step(8, cfl=0.5, want_time=True)
    U, T = s.get_state()
    s.close()
    assert np.array_equal(U, Uw) and np.array_equal(T, Tw) and ts == tw


class _ThreadExchange:
    """Two ranks of one process, one host thread each, each with its own
    stream. Per exchange: both wait until their packing is done (stream
    synchronise) and meet at a barrier; each copies its neighbour's send
    buffer into its receive buffer and the neighbour's LF-speed pair into a
    private copy, waits for those copies and meets the other again (so no
    buffer is overwritten while the other still reads it); then each takes
    the max. All waiting is on the host, with a time limit."""

    def __init__(self, rank, peers, barrier, periodic):
        from paper_2504_13750_gb300 import slab

        self.rank, self.peers, self.barrier = rank, peers, barrier
        self.lo, self.hi = slab.neighbours(rank, 2, periodic)
        self.alpha_peer = None

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch

        stream = torch.cuda.current_stream()
        stream.synchronize()
        self.barrier.wait(timeout=60)
        if self.lo is not None:
            recv_lo.copy_(self.peers[self.lo].send_hi)
        if self.hi is not None:
            recv_hi.copy_(self.peers[self.hi].send_lo)
        self.alpha_peer = self.peers[1 - self.rank].alpha2.clone()
        stream.synchronize()
        self.barrier.wait(timeout=60)

    def allreduce_max(self, alpha2):
        import torch

        torch.maximum(alpha2, self.alpha_peer, out=alpha2)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (2, 2, 1, 1)])
def test_two_standalone_slabs_in_two_threads(J, bc):
    """Two stand-alone slabs (the per-rank form) driven from two host threads
    through the callback, with walls and with a periodic x axis (where both
    neighbours of a rank are the same rank): bit for bit the undivided grid."""
    import torch

    from paper_2504_13750_gb300 import slab

    st = _tube(90, 16, bc=bc, vel=100.0)
    Uw, Tw, _ = _whole(J, H2AIR, st, True, 6, cfl=0.5)
    barrier = threading.Barrier(2)
    peers = [None, None]
    cols = slab.partition(90, 2)
    out = [None, None]
    errs = []

    def rank(r):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            comm = _ThreadExchange(r, peers, barrier, bc[0] == 2)
            with torch.cuda.stream(stream):
                peers[r] = slab.Slab(H2AIR, st["grid"], r, 2, comm, stream=stream)
            barrier.wait(timeout=60)
            x0, w = cols[r]
            part = {k: np.ascontiguousarray(st[k][:, x0:x0 + w]) for k in ("T", "p", "u", "v")}
            Y = np.ascontiguousarray(st["Y"][:, :, x0:x0 + w])
            peers[r].set_primitive(part["T"], part["p"], part["u"], part["v"], Y)
            peers[r].step(6, cfl=0.5)
            out[r] = peers[r].get_state()
        except Exception as e:  # noqa: BLE001 - reported below
            errs.append(e)
            barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    U = np.concatenate([out[0][0], out[1][0]], axis=2)
    T = np.concatenate([out[0][1], out[1][1]], axis=1)
    for p in peers:
        p.close()
    assert np.array_equal(U, Uw) and np.array_equal(T, Tw)
