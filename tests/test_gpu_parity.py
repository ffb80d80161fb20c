"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Metric per conserved plane q (and T): max|q_gpu - q_oracle| / max|q_oracle|
(norm-wise relative, since pointwise relative error is ill-posed for
rho v ~ 0 and radical mass fractions ~ 1e-20). Bars: 1e-12 for one right-hand
side, 1e-10 after one step, 1e-8 after 200 steps (all FP64).
"""
import numpy as np
import pytest

import mech_variants
import oracle as orc
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
    """Per-plane norm-wise relative error, max over planes."""
    a = np.asarray(a).reshape(a.shape[0], -1) if np.ndim(a) > 2 else np.asarray(a).reshape(1, -1)
    b = np.asarray(b).reshape(a.shape)
    out = 0.0
    for k in range(a.shape[0]):
        s = np.max(np.abs(b[k]))
        if s == 0.0:
            s = 1.0
        out = max(out, float(np.max(np.abs(a[k] - b[k])) / s))
    return out


def _cons(mech, st):
    return orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])


def _grid(J, mech, st, chem=True):
    return J.Grid.from_grid_dict(mech, st["grid"], chemistry=chem)


def test_reciprocal_within_one_ulp(J):
    rng = np.random.default_rng(0)
    x = 10.0 ** rng.uniform(-250, 250, 200000) * rng.uniform(1, 2, 200000)
    assert J.janc_selfcheck_rcp(x) <= 1


def test_set_state_matches_oracle_eos(J):
    st = inputs.tube(H2AIR, 37, 11, perturb_seed=3)
    g = _grid(J, H2AIR, st)
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], st["Y"])
    U, T = g.get_state()
    assert rel_err(U, _cons(H2AIR, st)) < 1e-14
    assert np.array_equal(T, st["T"])
    # conserved input + cold Newton start reproduces T
    g.set_state(_cons(H2AIR, st))
    U2, T2 = g.get_state()
    assert np.max(np.abs(T2 - st["T"]) / st["T"]) < 1e-12


@pytest.mark.parametrize("nx,ny,bc,aspect", [(256, 32, [0, 0, 0, 0], 1.0), (37, 11, [0, 0, 0, 0], 1.0),
                                             (45, 7, [2, 2, 1, 1], 1.0), (33, 9, [1, 1, 0, 0], 1.0),
                                             (3, 3, [0, 0, 0, 0], 1.0), (1, 1, [1, 1, 1, 1], 1.0),
                                             (45, 7, [0, 0, 0, 0], 1.7), (33, 9, [2, 2, 1, 1], 0.6)])
def test_face_fluxes_and_rhs(J, nx, ny, bc, aspect):
    """Face fluxes, L and alpha of one state; the last two grids have dy != dx
    (Eq. 4.10 divides the x-flux difference by dx and the y one by dy)."""
    st = inputs.tube(H2AIR, nx, ny, perturb_seed=5, aspect=aspect)
    st["grid"]["bc"] = bc
    rng = np.random.default_rng(nx * 100 + ny)
    st["u"] = rng.normal(0, 200.0, (ny, nx))
    st["v"] = rng.normal(0, 200.0, (ny, nx))
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    L, Fx, Gy, al = g.rhs()
    L0, Fx0, Gy0, al0 = orc.rhs(H2AIR, st["grid"], U, st["T"])
    assert np.max(np.abs(al - al0) / al0) < 1e-13
    assert rel_err(Fx, Fx0) < 1e-12
    assert rel_err(Gy, Gy0) < 1e-12
    assert rel_err(L, L0) < 1e-10


@pytest.mark.parametrize("nx,ny,aspect", [(256, 32, 1.0), (512, 96, 1.0), (1024, 96, 1.0), (256, 64, 1.7),
                                          (256, 64, 0.6)])
def test_one_step_tube(J, nx, ny, aspect):
    """One step against the oracle at sizes that take each launch shape the
    grid kernels choose by size: 256 x 32 (8-face flux tiles, 32 x 1 update
    blocks, 32-thread chemistry blocks), 512 x 96 (16-face tiles, 32 x 2,
    64 threads), 1024 x 96 (16-face tiles, 32 x 4, 128 threads); the
    4096 x 512 bench grid (32-face tiles, 32 x 8) is covered by
    test_full_size_config2_two_steps. The 256 x 64 tubes have dy = 1.7 dx and
    dy = 0.6 dx, so the CFL step takes dx in one and dy in the other."""
    st = inputs.tube(H2AIR, nx, ny, Lx=0.05 * nx / 256, perturb_seed=5, aspect=aspect)
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    t, dtl = g.step(1, cfl=0.5, want_time=True)
    Ug, Tg = g.get_state()
    Uo, To, s, to, dts = orc.step(H2AIR, st["grid"], U, st["T"], 1, cfl=0.5)
    assert s == 0
    assert abs(t - to) / to < 1e-14
    assert rel_err(Ug, Uo) < 1e-10
    assert rel_err(Tg[None], To[None]) < 1e-10


def test_200_steps_tube_config1(J):
    """256 x 32 detonation tube, chemistry on, CFL 0.5, 200 steps."""
    st = inputs.tube(H2AIR, 256, 32)
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    t, _ = g.step(200, cfl=0.5, want_time=True)
    Ug, Tg = g.get_state()
    Uo, To, s, to, _ = orc.step(H2AIR, st["grid"], U, st["T"], 200, cfl=0.5)
    assert s == 0
    assert abs(t - to) / to < 1e-12
    assert rel_err(Ug, Uo) < 1e-8
    assert rel_err(Tg[None], To[None]) < 1e-8
    # the GPU conserves mass and elements on its own to roundoff
    assert abs(Ug[0].sum() - U[0].sum()) / U[0].sum() < 1e-12


def test_200_steps_anisotropic_tube(J):
    """256 x 64 detonation tube with dy = 1.7 dx, chemistry on, CFL 0.5,
    200 steps (the 200-step bar on a grid whose two spacings differ)."""
    st = inputs.tube(H2AIR, 256, 64, perturb_seed=6, aspect=1.7)
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    t, _ = g.step(200, cfl=0.5, want_time=True)
    Ug, Tg = g.get_state()
    Uo, To, s, to, _ = orc.step(H2AIR, st["grid"], U, st["T"], 200, cfl=0.5)
    assert s == 0
    assert abs(t - to) / to < 1e-12
    assert rel_err(Ug, Uo) < 1e-8
    assert rel_err(Tg[None], To[None]) < 1e-8
    g.close()


@pytest.mark.parametrize("steps", [1, 60])
def test_strang_splitting_tube(J, steps):
    """The Strang order (chemistry dt/2, flux dt, chemistry dt/2) on a
    256 x 32 tube with a ragged 37-cell-wide igniting band, CFL 0.5."""
    st = inputs.tube(H2AIR, 256, 32, perturb_seed=4)
    st["T"][:, :37] = 1500.0
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st, chem=J.CHEM_STRANG)
    g.set_state(U, st["T"])
    t, _ = g.step(steps, cfl=0.5, want_time=True)
    Ug, Tg = g.get_state()
    Uo, To, s, to, _ = orc.step(H2AIR, st["grid"], U, st["T"], steps, cfl=0.5, chem=orc.CHEM_STRANG)
    assert s == 0
    tol = 1e-10 if steps == 1 else 1e-8
    assert abs(t - to) / to < 1e-12
    assert rel_err(Ug, Uo) < tol
    assert rel_err(Tg[None], To[None]) < tol
    # and it is not the Lie result
    Ul, _, _, _, _ = orc.step(H2AIR, st["grid"], U, st["T"], steps, cfl=0.5, chem=orc.CHEM_LIE)
    assert rel_err(Ug, Ul) > 1e3 * tol


def test_strang_rejected_by_server_and_adjoint(J):
    st = inputs.tube(H2AIR, 16, 8)
    g = _grid(J, H2AIR, st, chem=J.CHEM_STRANG)
    g.set_state(_cons(H2AIR, st), st["T"])
    with pytest.raises(RuntimeError):
        J.janc_step_adjoint(g.handle, 2, 1e-8, 1, J.LOSS_ENDWALL_P, None, None)
    with pytest.raises(RuntimeError):
        J.janc_server_create(J.Mechanism(H2AIR), chemistry=J.CHEM_STRANG)
    g.close()


GLOBAL = inputs.load_mechanism("global_h2o2_g129")


@pytest.mark.parametrize("steps", [1, 60])
def test_explicit_source_global_mechanism(J, steps):
    """JANC_CHEM_EXPLICIT (production rates as an RK3 source, no split
    chemistry) with the one-step global mechanism at gamma = 1.29: a 128 x 16
    stoichiometric H2-O2 tube with the 2000 K / 20 atm igniter."""
    Y = inputs.premix_Y(GLOBAL, {"H2": 4.032, "O2": 31.998})
    st = inputs.tube(GLOBAL, 128, 16, Lx=0.025, Y=Y, perturb_seed=1)
    U = _cons(GLOBAL, st)
    g = _grid(J, GLOBAL, st, chem=J.CHEM_EXPLICIT)
    g.set_state(U, st["T"])
    t, _ = g.step(steps, cfl=0.5, want_time=True)
    Ug, Tg = g.get_state()
    Uo, To, s, to, _ = orc.step(GLOBAL, st["grid"], U, st["T"], steps, cfl=0.5, chem=orc.CHEM_EXPLICIT)
    assert s == 0
    tol = 1e-10 if steps == 1 else 1e-8
    assert abs(t - to) / to < 1e-12
    assert rel_err(Ug, Uo) < tol
    assert rel_err(Tg[None], To[None]) < tol
    if steps > 1:  # the igniter has formed water (nothing is clipped: WENO may undershoot near 0)
        assert np.max(1.0 - (Ug[4] + Ug[5]) / Ug[0]) > 0.05
    g.close()


@pytest.mark.parametrize("nx,ny", [(8, 8), (4096, 512)])
def test_uniform_periodic_state_stays_uniform(J, nx, ny):
    """Freestream at any size, bit for bit: a uniform reacting state moving
    diagonally with periodic boundaries (WENO reproduces constant data
    exactly, the LF speeds are a max over identical cells, every cell reacts
    alike) stays uniform, and its cells equal those of an 8 x 8 grid."""
    Y = inputs.h2air_Y(H2AIR, 1.0)

    def run(nx, ny):
        g = J.Grid(H2AIR, nx, ny, 1e-4, 1e-4, [2, 2, 2, 2], chemistry=True)
        one = np.ones((ny, nx))
        g.set_primitive(1250.0 * one, 2 * inputs.ATM * one, 50.0 * one, -30.0 * one,
                        np.ascontiguousarray(Y[:, None, None] * one))
        g.step(3, dt=2e-8)
        U, T = g.get_state()
        g.close()
        return U, T

    U, T = run(nx, ny)
    assert np.all(U == U[:, :1, :1]) and np.all(T == T[0, 0])
    Us, Ts = run(8, 8)
    assert np.array_equal(U[:, 0, 0], Us[:, 0, 0]) and T[0, 0] == Ts[0, 0]
    assert U[4:, 0, 0].sum() < U[0, 0, 0]           # still a mixture; chemistry has run
    st = inputs.ignition_cell(H2AIR, T0=1250.0, p0=2 * inputs.ATM)
    U1 = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    assert not np.allclose(U[4:, 0, 0], U1[4:, 0, 0], rtol=1e-12, atol=0)  # it reacted


def test_sod_gpu(J):
    import ref_exact

    st = inputs.sod(GAS, 400)
    U = _cons(GAS, st)
    g = _grid(J, GAS, st, chem=False)
    g.set_state(U, st["T"])
    t, _ = g.step(690, cfl=0.2, want_time=True)
    Ug, Tg = g.get_state()
    Uo, To, s, to, _ = orc.step(GAS, st["grid"], U, st["T"], 690, cfl=0.2, chem=False)
    assert rel_err(Ug, Uo) < 1e-8
    ex = ref_exact.riemann_exact((1.0, 0.0, 1e5), (0.125, 0.0, 1e4), st["x"], t)
    assert np.mean(np.abs(Ug[0, 0] - ex[0])) / np.mean(np.abs(ex[0])) < 3.5e-3


def test_ignition_cell_gpu(J):
    st = inputs.ignition_cell(H2AIR, T0=1500.0)
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    g.step(4000, dt=5e-9)
    Ug, Tg = g.get_state()
    Uo, To, s, _, _ = orc.step(H2AIR, st["grid"], U, st["T"], 4000, dt=5e-9)
    assert rel_err(Ug, Uo) < 1e-9
    assert abs(Tg[0, 0] - To[0, 0]) / To[0, 0] < 1e-10


def test_linear_mechanism_three_species(J):
    from test_oracle_pins import _linear_mech

    m = _linear_mech(3.0e4)
    m["elements"] = {}
    nx, ny = 17, 5
    rng = np.random.default_rng(2)
    Y = rng.dirichlet(np.ones(3), (ny, nx)).transpose(2, 0, 1).copy()
    st = {"T": rng.uniform(900, 1300, (ny, nx)), "p": np.full((ny, nx), 1e5), "u": rng.normal(0, 50, (ny, nx)),
          "v": np.zeros((ny, nx)), "Y": Y, "grid": inputs.grid_dict(nx, ny, 1e-3, 1e-3, [0, 0, 0, 0])}
    U = _cons(m, st)
    g = _grid(J, m, st)
    g.set_state(U, st["T"])
    # dt = 5e-7 s keeps the acoustic CFL near 0.35 on this 1 mm grid
    g.step(20, dt=5e-7)
    Ug, _ = g.get_state()
    Uo, _, s, _, _ = orc.step(m, st["grid"], U, st["T"], 20, dt=5e-7)
    assert s == 0
    assert rel_err(Ug, Uo) < 1e-10


def test_full_size_config2_two_steps(J):
    """4096 x 512 tube in the benchmark's launch configuration: two steps
    against the oracle on the whole grid, element by element."""
    st = inputs.tube(H2AIR, 4096, 512, perturb_seed=0)
    U = _cons(H2AIR, st)
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    g.step(2, cfl=0.5)
    Ug, Tg = g.get_state()
    orc.set_threads(0)
    Uo, To, s, _, _ = orc.step(H2AIR, st["grid"], U, st["T"], 2, cfl=0.5)
    assert s == 0
    assert rel_err(Ug, Uo) < 1e-10
    assert rel_err(Tg[None], To[None]) < 1e-10


def test_status_word_reports_bad_state(J):
    st = inputs.tube(H2AIR, 16, 8)
    U = _cons(H2AIR, st)
    U[0, 3, 4] = -1.0  # negative density in one cell
    g = _grid(J, H2AIR, st)
    g.set_state(U, st["T"])
    rc = J.janc_get_state(g.handle, np.zeros_like(U), np.zeros(st["T"].shape), check=False)
    assert rc == -5
    assert g.status()["status"] & J.ST_NONPOSITIVE


def test_fp64_peak_probe(J):
    r = J.janc_fp64_peak(n_iter=2000)
    assert 1e11 < r < 1e13


def test_exponential_within_two_ulp(J):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-700, 700, 100000), rng.uniform(-40, 40, 100000), rng.normal(0, 1e-3, 10000),
                        np.linspace(-30, 30, 6001)])
    assert J.janc_selfcheck_exp(x) <= 2


def test_run_time_table_chemistry_kernels(J):
    """A 9-species table whose reaction structure differs from the compiled
    one (the shipped reactions in reverse order) runs the run-time-table
    chemistry kernels: one CFL step and 40 steps against the oracle on the same
    table, and the 40 steps against the compiled kernels on the shipped order
    (the same arithmetic up to the order of the sums over reactions)."""
    rev = mech_variants.reordered(H2AIR)
    st = inputs.tube(H2AIR, 256, 32, perturb_seed=5)
    U = _cons(H2AIR, st)
    g = _grid(J, rev, st)
    g.set_state(U, st["T"])
    g.step(1, cfl=0.5)
    Ug, Tg = g.get_state()
    Uo, To, s, _, _ = orc.step(rev, st["grid"], U, st["T"], 1, cfl=0.5)
    assert s == 0
    assert rel_err(Ug, Uo) < 1e-10 and rel_err(Tg[None], To[None]) < 1e-10
    g.step(39, cfl=0.5)
    Ug, Tg = g.get_state()
    Uo, To, s, _, _ = orc.step(rev, st["grid"], U, st["T"], 40, cfl=0.5)
    assert s == 0
    assert rel_err(Ug, Uo) < 1e-8 and rel_err(Tg[None], To[None]) < 1e-8
    gf = _grid(J, H2AIR, st)
    gf.set_state(U, st["T"])
    gf.step(40, cfl=0.5)
    Uf, Tf = gf.get_state()
    assert rel_err(Ug, Uf) < 1e-8 and rel_err(Tg[None], Tf[None]) < 1e-8
    g.close()
    gf.close()
