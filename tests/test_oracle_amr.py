"""Pins of the AMR oracle (oracle/amr.py) against what the paper and the
mathematics fix: the crossover order of Algorithm 2, the exactness of
one-to-four refinement followed by four-to-one coarsening, ghost blocks that
reproduce a uniform fine array, the external-boundary band, the refinement
criterion against a brute-force definition, reduction to the base step when
nothing is refined, and the accuracy gain on a Riemann problem."""
import numpy as np
import pytest

import oracle as orc
from amr import AMROracle, NG
from paper_2504_13750_gb300 import inputs

H2AIR = inputs.load_mechanism("h2air_synth")
GAS = inputs.load_mechanism("ideal_gamma14")


def _tube(nx, ny, seed=3):
    st = inputs.tube(H2AIR, nx, ny, Lx=0.05 * nx / 256, perturb_seed=seed)
    U = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    return st, U


def test_no_refinement_is_the_base_step():
    st, U = _tube(32, 16)
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=2, threshold=np.inf)
    Ub, Tb = U.copy(), st["T"].copy()
    for _ in range(3):
        dt = a.step(cfl=0.5)
        Ub, Tb, s, _, _ = orc.step(H2AIR, st["grid"], Ub, Tb, 1, dt=dt)
        assert s == 0
    assert not a.layers[1].pos
    assert np.array_equal(a.U0, Ub) and np.array_equal(a.T0, Tb)


def test_crossover_order_of_algorithm_2():
    st, U = _tube(32, 16)
    force = {1: {(0, 0), (1, 0)}, 2: {(0, 0), (1, 1)}}
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=2, force_blocks=force, chem=False)
    dt = 1e-8
    a.step(dt=dt)
    assert a.trace == [(2, dt / 4), (2, dt / 4), (1, dt / 2), (2, dt / 4), (2, dt / 4), (1, dt / 2), (0, dt)]


def test_synchronous_order_of_algorithm_2():
    """Fig. 2b: every layer takes the same dt, deepest first, once per step."""
    st, U = _tube(32, 16)
    force = {1: {(0, 0), (1, 0)}, 2: {(0, 0), (1, 1)}}
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=2, force_blocks=force, chem=False, synchronous=True)
    dt = 1e-8
    a.step(dt=dt)
    assert a.trace == [(2, dt), (1, dt), (0, dt)]
    assert a.cell_updates_per_step() == 32 * 16 + (2 + 2) * 256


def test_synchronous_and_crossover_agree_to_high_order():
    """Both strategies integrate the same equations with third-order RK3
    steps. On a smooth acoustic wave without chemistry, after the same
    simulated time, their base layers differ by far less than the change over
    that time. (With split chemistry the base layer's own dt enters the
    first-order splitting error, so the two differ at O(dt) there.)"""
    st, U = _tube(32, 16)
    x = np.arange(32) / 32
    st["T"] = 1150.0 + 50.0 * np.sin(2 * np.pi * x)[None, :] * np.ones((16, 1))
    st["p"] = inputs.ATM * (1 + 0.05 * np.cos(2 * np.pi * x))[None, :] * np.ones((16, 1))
    U = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    force = {1: {(2, 0), (3, 0), (2, 1), (3, 1)}}
    dt = 2e-8
    c = AMROracle(H2AIR, st["grid"], U, st["T"], levels=1, force_blocks=force, regrid_every=100, chem=False)
    y = AMROracle(H2AIR, st["grid"], U, st["T"], levels=1, force_blocks=force, regrid_every=100, chem=False,
                  synchronous=True)
    for _ in range(4):
        c.step(dt=dt)
    for _ in range(8):
        y.step(dt=dt / 2)
    moved = 0
    for k in range(4):
        change = np.max(np.abs(c.U0[k] - U[k]))
        if change > 0:
            moved += 1
            assert np.max(np.abs(c.U0[k] - y.U0[k])) < 0.02 * change, k
    assert moved == 3


def test_fine_to_coarse_skips_the_external_band():
    """The four-to-one mean writes the parent cells whose four children the
    fine solver computed; parent cells with a child in the external band
    (a copy of the parent) keep their own value, so that region evolves on
    the parent layer instead of freezing."""
    st, U = _tube(32, 16)
    force = {1: {(2, 0)}}                      # one block: every side external or physical
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=1, force_blocks=force, chem=False)
    a.regrid()
    L = a.layers[1]
    rng = np.random.default_rng(3)
    L.U = L.U * (1 + 1e-3 * rng.standard_normal(L.U.shape))
    U_before = a.U0.copy()
    a.fine_to_coarse()
    band = a.external_band(L, 0)
    keep = band[0::2, 0::2] | band[0::2, 1::2] | band[1::2, 0::2] | band[1::2, 1::2]
    f = L.U[0]
    mean = 0.25 * ((f[:, 0::2, 0::2] + f[:, 0::2, 1::2]) + (f[:, 1::2, 0::2] + f[:, 1::2, 1::2]))
    region = a.U0[:, 0:8, 16:24]
    assert keep.any() and not keep.all()
    assert np.array_equal(region[:, keep], U_before[:, 0:8, 16:24][:, keep])
    assert np.array_equal(region[:, ~keep], mean[:, ~keep])


def test_refine_then_coarsen_returns_the_parent():
    st, U = _tube(32, 16)
    force = {1: {(1, 0), (2, 1), (3, 1)}, 2: {(2, 1), (5, 2)}}
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=2, force_blocks=force, chem=False)
    a.regrid()
    U0, T0 = a.U0.copy(), a.T0.copy()
    U1 = a.layers[1].U.copy()
    a.fine_to_coarse()
    assert np.array_equal(a.U0, U0)            # four-to-one of a one-to-four copy is exact
    assert np.max(np.abs(a.T0 - T0) / T0) < 1e-12
    assert np.array_equal(a.layers[1].U, U1)
    # layer-2 block (5, 2) sits in layer-1 block (2, 1): it holds layer-1 values one-to-four
    L2 = a.layers[2]
    k = L2.index[(5, 2)]
    P = a.layers[1]
    kp = P.index[(2, 1)]
    quad = P.U[kp][:, 0:8, 8:16]              # (by % 2, bx % 2) = (0, 1)
    assert np.array_equal(L2.U[k][:, 0::2, 0::2], quad) and np.array_equal(L2.U[k][:, 1::2, 1::2], quad)


@pytest.mark.parametrize("bc", [[0, 0, 0, 0], [1, 1, 2, 2], [2, 2, 0, 1]])
def test_ghost_blocks_reproduce_the_fine_array(bc):
    """Every layer-1 block present: each block's right-hand side from its ghost
    block (neighbours, periodic partners and physical ghosts) equals, bit for
    bit, the right-hand side of the whole layer-1 array as one grid with the
    domain's boundaries and the same LF speeds."""
    st, U = _tube(32, 16)
    st["grid"]["bc"] = bc
    rng = np.random.default_rng(2)
    st["u"] = rng.normal(0, 80.0, st["T"].shape)
    st["v"] = rng.normal(0, 80.0, st["T"].shape)
    U = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    nbx, nby = 32 * 2 // 16, 16 * 2 // 16
    force = {1: {(bx, by) for bx in range(nbx) for by in range(nby)}}
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=1, force_blocks=force)
    a.regrid()
    L = a.layers[1]
    # perturb the fine data so that blocks are not piecewise constant
    L.U = L.U * (1 + 1e-3 * rng.standard_normal(L.U.shape))
    L.T = np.stack([orc.newton(H2AIR, st["grid"], L.U[k], L.T[k])[0] for k in range(len(L.pos))])
    B = 16
    Ug = np.zeros((a.nv, 32, 64))
    Tg = np.zeros((32, 64))
    for k, (bx, by) in enumerate(L.pos):
        Ug[:, by * B:(by + 1) * B, bx * B:(bx + 1) * B] = L.U[k]
        Tg[by * B:(by + 1) * B, bx * B:(bx + 1) * B] = L.T[k]
    dx, dy = a.h(1)
    gfine = dict(st["grid"], nx=64, ny=32, dx=dx, dy=dy)
    Lg, _, _, alpha = orc.rhs(H2AIR, gfine, Ug, Tg)
    assert np.array_equal(alpha, orc.lf_alpha(H2AIR, Ug, Tg))
    for k, (bx, by) in enumerate(L.pos):
        assert not a.external_band(L, k).any()
        P, PT = a.ghost_block(L, L.U, L.T, k)
        Lk = orc.rhs_ghosted(H2AIR, B, B, dx, dy, P, PT, alpha)
        assert np.array_equal(Lk, Lg[:, by * B:(by + 1) * B, bx * B:(bx + 1) * B]), (bx, by)


def test_external_band_takes_the_parent_and_stops_the_nan_ghosts():
    st, U = _tube(32, 16)
    force = {1: {(1, 0), (2, 0), (2, 1)}}
    a = AMROracle(H2AIR, st["grid"], U, st["T"], levels=1, force_blocks=force, chem=False)
    a.regrid()
    L = a.layers[1]
    rng = np.random.default_rng(5)
    L.U = L.U * (1 + 1e-3 * rng.standard_normal(L.U.shape))
    L.T = np.stack([orc.newton(H2AIR, st["grid"], L.U[k], L.T[k])[0] for k in range(len(L.pos))])
    parents = [a.parent_copy(1, bx, by) for (bx, by) in L.pos]
    a.solve_layer(1, 2e-9)
    for k in range(len(L.pos)):
        band = a.external_band(L, k)
        assert band.any() and not band.all()
        assert np.array_equal(L.U[k][:, band], parents[k][0][:, band])
        assert np.array_equal(L.T[k][band], parents[k][1][band])
        assert np.all(np.isfinite(L.U[k])) and np.all(np.isfinite(L.T[k]))
        assert not np.array_equal(L.U[k][:, ~band], parents[k][0][:, ~band])


def test_refinement_flags_match_brute_force():
    st, U = _tube(32, 16)
    rng = np.random.default_rng(9)
    T = 300.0 + 50.0 * rng.random((16, 32))
    T[6:9, 10:13] += 1500.0
    U = orc.prim_to_cons(H2AIR, T, st["p"], st["u"], st["v"], st["Y"])
    dx = st["grid"]["dx"]
    thr = 1500.0 / dx * 0.4
    a = AMROracle(H2AIR, st["grid"], U, T, levels=1, threshold=thr, n_buffer=2)
    got = set(a.refinement_block_mask(1))
    # brute force: cell gradients by their definition, then every candidate block
    marked = []
    for j in range(16):
        for i in range(32):
            ip, im = min(i + 1, 31), max(i - 1, 0)
            jp, jm = min(j + 1, 15), max(j - 1, 0)
            gx = (T[j, ip] - T[j, im]) / ((ip - im) * dx)
            gy = (T[jp, i] - T[jm, i]) / ((jp - jm) * st["grid"]["dy"])
            if np.hypot(gx, gy) > thr:
                marked.append((i, j))
    want = set()
    for by in range(2):
        for bx in range(4):
            x0, y0 = bx * 8, by * 8
            for (i, j) in marked:
                dxc = max(x0 - i, 0, i - (x0 + 7))
                dyc = max(y0 - j, 0, j - (y0 + 7))
                if max(dxc, dyc) <= 2:
                    want.add((bx, by))
    assert got == want and 0 < len(got) < 8


def test_amr_sharpens_a_riemann_problem():
    """Sod's problem along x: the two-layer AMR solution, averaged to the base
    grid, is closer to a uniform 4x finer solution than the base grid alone."""
    nx, ny = 128, 8
    st = inputs.sod(GAS, nx)
    st2 = inputs.sod(GAS, nx)
    st["grid"]["ny"] = ny
    for k in ("T", "p", "u", "v"):
        st[k] = np.repeat(st[k][:1], ny, 0)
    st["Y"] = np.repeat(st["Y"][:, :1], ny, 1)
    st["grid"]["dy"] = st["grid"]["dx"]
    st["grid"]["bc"] = [1, 1, 1, 1]
    U = orc.prim_to_cons(GAS, st["T"], st["p"], st["u"], st["v"], st["Y"])
    # uniform reference at 4x resolution
    nf = nx * 4
    x = np.repeat(np.repeat(st["T"], 4, 0), 4, 1)
    Tf = x
    pf = np.repeat(np.repeat(st["p"], 4, 0), 4, 1)
    zf = np.zeros_like(Tf)
    Yf = np.repeat(np.repeat(st["Y"], 4, 1), 4, 2)
    gf = dict(st["grid"], nx=nf, ny=ny * 4, dx=st["grid"]["dx"] / 4, dy=st["grid"]["dy"] / 4)
    Uf = orc.prim_to_cons(GAS, Tf, pf, zf, zf, Yf)
    dt = 0.2 * st["grid"]["dx"] / 420.0
    a = AMROracle(GAS, st["grid"], U, st["T"], levels=2, threshold=5.0 / st["grid"]["dx"], n_buffer=3,
                  regrid_every=4, chem=False)
    Uc, Tc = U.copy(), st["T"].copy()
    nsteps = 40
    for _ in range(nsteps):
        a.step(dt=dt)
        Uc, Tc, _, _, _ = orc.step(GAS, st["grid"], Uc, Tc, 1, dt=dt, chem=False)
    Uf, Tf, s, _, _ = orc.step(GAS, gf, Uf, Tf, 4 * nsteps, dt=dt / 4, chem=False)
    assert s == 0
    ref = Uf[0].reshape(ny, 4, nx, 4).mean(axis=(1, 3))
    e_amr = np.abs(a.U0[0] - ref).mean()
    e_base = np.abs(Uc[0] - ref).mean()
    assert a.layers[2].pos, "no layer-2 blocks"
    assert e_amr < 0.5 * e_base, (e_amr, e_base)
    assert np.allclose(a.U0[0], a.U0[0][:1])   # stays one-dimensional
