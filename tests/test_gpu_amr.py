"""Block-structured AMR on the GPU (janc_amr_*) against the AMR oracle
(oracle/amr.py): the same block lists (bit-exact), the base layer and every
refined layer within the per-step floating-point tolerance, on a reacting
tube with walls and on a Riemann problem with zero-gradient and periodic
sides."""
import numpy as np
import pytest

import oracle as orc
from amr import EXTERNAL, PHYSICAL, AMROracle, Layer
from paper_2504_13750_gb300 import inputs

pytestmark = pytest.mark.gpu

H2AIR = inputs.load_mechanism("h2air_synth")
GAS = inputs.load_mechanism("ideal_gamma14")


@pytest.fixture(scope="module")
def J():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_13750_gb300 import build, janc

    build.build()
    return janc


def rel_err(a, b):
    out = 0.0
    for k in range(a.shape[0]):
        s = max(float(np.max(np.abs(b[k]))), 1e-300)
        out = max(out, float(np.max(np.abs(a[k] - b[k])) / s))
    return out


def _margin_ok(o: AMROracle):
    """No cell of a parent layer sits within 1e-9 (relative) of the threshold,
    so both sides take the same refinement decisions."""
    for i in range(1, o.levels + 1):
        dx, dy = o.h(i - 1)
        T, valid = o.layer_T(i - 1)
        x = o.grad_T(T, dx, dy, valid)[valid]
        if x.size and np.min(np.abs(x - o.threshold)) <= 1e-9 * o.threshold:
            return False
    return True


def _compare(J, mech, st, chem, levels, thr, nbuf, every, nsteps, cfl=0.5, dt=0.0, tol_step=1e-10, sync=False):
    if dt > 0.0:
        cfl = 0.0
    U = orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])
    o = AMROracle(mech, st["grid"], U, st["T"], levels=levels, threshold=thr, n_buffer=nbuf, regrid_every=every,
                  chem=chem, synchronous=sync)
    a = J.Amr(mech, st["grid"], chemistry=chem, levels=levels, threshold=thr, n_buffer=nbuf, regrid_every=every,
              synchronous=sync)
    a.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    for n in range(nsteps):
        if n % every == 0:
            assert _margin_ok(o), "a gradient sits on the threshold: pick another"
        t_o = o.step(dt=dt, cfl=cfl)
        t_g = a.step(1, dt=dt, cfl=cfl)
        assert abs(t_g - t_o) <= 1e-12 * t_o, (n, t_g, t_o)
        tol = tol_step * (n + 1)
        Ub, Tb = a.base()
        assert rel_err(Ub, o.U0) < tol, (n, rel_err(Ub, o.U0))
        assert rel_err(Tb[None], o.T0[None]) < tol
        for i in range(1, levels + 1):
            pos, UL, TL = a.layer(i)
            assert [tuple(p) for p in pos] == o.layers[i].pos, (n, i)
            if len(pos):
                # the bound is per step of that layer: 2^i steps per base step under crossover
                tol_i = tol * (1 if sync else 2 ** i)
                assert rel_err(UL.transpose(1, 0, 2, 3), o.layers[i].U.transpose(1, 0, 2, 3)) < tol_i, (n, i)
                assert np.max(np.abs(TL - o.layers[i].T) / o.layers[i].T) < tol_i
    assert a.status() == 0
    assert a.cell_updates() == o.cell_updates_per_step()
    return a, o


@pytest.mark.parametrize("sync,levels,aspect", [(False, 2, 1.0), (True, 2, 1.0), (False, 3, 1.0), (False, 2, 1.7)])
def test_amr_reacting_tube_with_walls(J, sync, levels, aspect):
    """Crossover (Fig. 2a) and synchronous (Fig. 2b) advance; three layers
    exercise a refined layer whose parent is itself refined; the last case has
    dy = 1.7 dx on every layer."""
    st = inputs.tube(H2AIR, 64, 16, Lx=0.05 * 64 / 256, perturb_seed=3, aspect=aspect)
    dx = st["grid"]["dx"]
    a, o = _compare(J, H2AIR, st, True, levels=levels, thr=100.0 / dx, nbuf=2, every=2, nsteps=5, sync=sync)
    assert all(o.layers[i].pos for i in range(1, levels + 1))
    a.close()


def test_amr_riemann_zero_gradient_and_periodic(J):
    nx, ny = 128, 16
    st = inputs.sod(GAS, nx)
    for k in ("T", "p", "u", "v"):
        st[k] = np.repeat(st[k][:1], ny, 0)
    st["Y"] = np.repeat(st["Y"][:, :1], ny, 1)
    # a transverse wave so that the y direction does work
    y = (np.arange(ny) + 0.5) / ny
    st["v"] = st["v"] + 20.0 * np.sin(2 * np.pi * y)[:, None]
    st["grid"].update(ny=ny, dy=st["grid"]["dx"], bc=[1, 1, 2, 2])
    dt = 0.2 * st["grid"]["dx"] / 420.0
    a, o = _compare(J, GAS, st, False, levels=2, thr=5.0 / st["grid"]["dx"], nbuf=3, every=3, nsteps=7, dt=dt)
    assert len(o.layers[2].pos) > 2
    a.close()


def test_amr_without_refinement_is_the_grid_step(J):
    st = inputs.tube(H2AIR, 64, 16, Lx=0.05 * 64 / 256, perturb_seed=3)
    a = J.Amr(H2AIR, st["grid"], chemistry=True, levels=2, threshold=1e300, n_buffer=2, regrid_every=2)
    a.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    g = J.Grid.from_grid_dict(H2AIR, st["grid"])
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    a.step(4, cfl=0.5)
    g.step(4, cfl=0.5)
    Ua, Ta = a.base()
    Ug, Tg = g.get_state()
    assert np.array_equal(Ua, Ug) and np.array_equal(Ta, Tg)
    assert J.janc_amr_layer_blocks(a.handle, 1) == 0
    a.close()
    g.close()


def test_full_layer_is_a_decomposed_fine_grid(J):
    """Domain decomposition is exact: with every layer-1 block present (a
    threshold every cell exceeds), layer 1 is the 2x-finer grid cut into
    16 x 16 blocks that exchange 3 ghost columns per side every RK stage.
    From the same one-to-four start it must step like one undecomposed fine
    grid with dt/2 (the single-GPU form of the "N subdomains = 1 domain"
    parity), to rounding. The two start apart at the rounding level: the
    layer copies its parent's T while the fine grid's set_state recovers T
    from U by Newton, and the stiff chemistry amplifies that difference in
    the radical planes, so the bound is 1e-11 per step."""
    st = inputs.tube(H2AIR, 64, 16, Lx=0.05 * 64 / 256, perturb_seed=3)
    a = J.Amr(H2AIR, st["grid"], chemistry=True, levels=1, threshold=-1.0, n_buffer=0, regrid_every=1000)
    a.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    U0, T0 = a.base()
    gf = dict(st["grid"], nx=128, ny=32, dx=st["grid"]["dx"] / 2, dy=st["grid"]["dy"] / 2)
    f = J.Grid.from_grid_dict(H2AIR, gf)
    f.set_state(np.ascontiguousarray(np.repeat(np.repeat(U0, 2, 1), 2, 2)),
                np.ascontiguousarray(np.repeat(np.repeat(T0, 2, 0), 2, 1)))
    dt = 2e-8
    for n in range(1, 5):
        a.step(1, dt=dt)
        f.step(2, dt=dt / 2)
        pos, UL, TL = a.layer(1)
        assert len(pos) == (128 // 16) * (32 // 16)
        Ug = np.zeros((UL.shape[1], 32, 128))
        Tg = np.zeros((32, 128))
        for k, (bx, by) in enumerate(pos):
            Ug[:, by * 16:(by + 1) * 16, bx * 16:(bx + 1) * 16] = UL[k]
            Tg[by * 16:(by + 1) * 16, bx * 16:(bx + 1) * 16] = TL[k]
        Uf, Tf = f.get_state()
        assert rel_err(Ug, Uf) < 1e-11 * n, (n, rel_err(Ug, Uf))
        assert np.max(np.abs(Tg - Tf) / Tf) < 1e-11 * n
    assert a.status() == 0
    a.close()
    f.close()


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (2, 2, 0, 0), (1, 1, 2, 2), (2, 2, 2, 2), (0, 1, 1, 0)])
def test_device_block_lists_match_the_oracle_layer(J, bc):
    """The regrid's block lists, built on the device from refinement flags
    (janc_amr_block_lists: the compaction and neighbour kernels of the
    regrid), against the AMR oracle's definition: blocks in (by, bx) order,
    the position map, and the neighbours across every side (periodic partner,
    physical side, external side), for random flag patterns."""
    rng = np.random.default_rng(sum(bc) + 7)
    for nbx, nby in [(1, 1), (2, 3), (8, 4), (13, 5), (256, 64), (1024, 128)]:
        for density in (0.0, 0.3, 0.7, 1.0):
            flags = (rng.random((nby, nbx)) < density).astype(np.uint8)
            pos, mp, nbr = J.janc_amr_block_lists(flags, bc)
            opos = [(bx, by) for by in range(nby) for bx in range(nbx) if flags[by, bx]]
            assert [tuple(p) for p in pos] == opos
            want_map = -np.ones((nby, nbx), dtype=np.int32)
            for k, (bx, by) in enumerate(opos):
                want_map[by, bx] = k
            assert np.array_equal(mp, want_map)
            if nbx * nby <= 4096:  # the oracle's neighbour walk is plain Python
                lay = Layer(1, opos, None, None, nbx, nby, bc)
                for k in range(len(opos)):
                    assert tuple(nbr[k]) == lay.neighbours(k), (nbx, nby, k)
    assert EXTERNAL == -1 and PHYSICAL == -2   # the codes the kernels use


def test_regrid_every_step_matches_the_oracle(J):
    """A regrid before every base step of the reacting tube: each regrid
    builds the lists on the device, refills the state into the layer's spare
    buffer (growing the buffers only when the layer outgrows them) and swaps
    it in; the layers and the base still match the AMR oracle step by step."""
    st = inputs.tube(H2AIR, 64, 16, Lx=0.05 * 64 / 256, perturb_seed=3)
    dx = st["grid"]["dx"]
    a, o = _compare(J, H2AIR, st, True, levels=2, thr=100.0 / dx, nbuf=2, every=1, nsteps=6)
    assert all(o.layers[i].pos for i in range(1, 3))
    a.close()
