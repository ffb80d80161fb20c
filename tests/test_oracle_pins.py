"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a
first-principles derivation (WENO5), closed forms and invariants
(freestream, conservation, symmetry, element balance, backward Euler for a
linear source), convergence orders, the exact Riemann solution of the Sod
problem (Sec. 5.1(1)), thermodynamic equilibrium (for Eq. 4.9) and an
independent stiff integration of a constant-volume reactor (Sec. 5.1(2)).
"""
import os

import numpy as np
import pytest

import oracle as orc
import ref_exact
from paper_2504_13750_gb300 import inputs

H2AIR = inputs.load_mechanism("h2air_synth")
GAS = inputs.load_mechanism("ideal_gamma14")
R_GAS = 287.0


def _cons(mech, st):
    return orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])


# ----------------------------------------------------------------------------
# WENO5
# ----------------------------------------------------------------------------
def _weno_from_definition():
    """Candidate values, linear weights and smoothness indicators derived from
    their definitions (Jiang & Shu 1996): quadratics matching cell averages on
    each 3-cell substencil, the quartic on all 5 cells, and
    beta_k = sum_{l=1,2} int_cell (d^l p_k / dx^l)^2 dx (dx = 1)."""
    sp = pytest.importorskip("sympy")
    x = sp.Symbol("x")
    f = sp.symbols("f0:5")  # cell averages on cells -2..2 (centre cell 0)
    cells = [-2, -1, 0, 1, 2]

    def fit(idx, deg):
        c = sp.symbols(f"c0:{deg + 1}")
        P = sum(c[m] * x**m for m in range(deg + 1))
        eqs = [sp.integrate(P, (x, cells[j] - sp.Rational(1, 2), cells[j] + sp.Rational(1, 2))) - f[j] for j in idx]
        sol = sp.solve(eqs, c)
        return sp.expand(P.subs(sol))

    half = sp.Rational(1, 2)
    q, beta = [], []
    for k in range(3):
        P = fit([k, k + 1, k + 2], 2)
        q.append(sp.expand(P.subs(x, half)))
        beta.append(sp.expand(sum(sp.integrate(sp.diff(P, x, l) ** 2, (x, -half, half)) for l in (1, 2))))
    P5 = fit([0, 1, 2, 3, 4], 4).subs(x, half)
    d = sp.symbols("d0:3")
    resid = sp.expand(sum(d[k] * q[k] for k in range(3)) - P5)
    dsol = sp.solve([resid.coeff(fj) for fj in f], d)
    dv = [dsol[d[k]] for k in range(3)]
    return (sp.lambdify(f, q), sp.lambdify(f, beta), [float(v) for v in dv])


def test_weno5_matches_first_principles():
    qf, bf, d = _weno_from_definition()
    assert np.allclose(d, [0.1, 0.6, 0.3], rtol=0, atol=1e-15)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for trial in range(200):
        scale = 10.0 ** rng.uniform(-3, 6)
        fv = rng.normal(size=5) * scale
        if trial % 4 == 0:
            fv[3:] += 20 * scale  # a jump inside the stencil
        q = np.array(qf(*fv))
        b = np.array(bf(*fv))
        a = np.array(d) / (eps + b) ** 2
        ref = np.sum(a * q) / np.sum(a)
        got = orc.weno5(fv, eps)
        assert abs(got - ref) <= 1e-12 * (np.max(np.abs(fv)) + 1e-300), (fv, got, ref)


def test_weno5_special_cases():
    # polynomial data of degree <= 1: all smoothness indicators agree, the
    # weights are the linear ones and the face value is exact
    for c0, c1 in [(3.0, 0.0), (-2.0, 0.5), (1e5, -37.0)]:
        cells = np.arange(-2, 3)
        got = orc.weno5(c0 + c1 * cells, 1e-6)
        assert abs(got - (c0 + c1 * 0.5)) <= 1e-12 * abs(c0)
    # odd symmetry, bitwise
    rng = np.random.default_rng(1)
    for _ in range(50):
        fv = rng.normal(size=5) * 1e3
        assert orc.weno5(-fv, 1e-6) == -orc.weno5(fv, 1e-6)
    # essentially non-oscillatory: a jump between f3 and f4 leaves stencil 0/1
    # smooth; the face value stays within the smooth data range
    fv = np.array([1.0, 1.0, 1.0, 1.0, 100.0])
    assert abs(orc.weno5(fv, 1e-6) - 1.0) < 1e-6


# ----------------------------------------------------------------------------
# Semi-discretisation + RK3
# ----------------------------------------------------------------------------
def _advection(N, dt_of, tend=0.002, u0=100.0):
    """Contact-wave advection: rho = 1 + 0.2 sin(2 pi x), u, p constant,
    periodic in x. The exact solution is a translation."""
    dx = 1.0 / N
    x = (np.arange(N) + 0.5) * dx
    rho = 1 + 0.2 * np.sin(2 * np.pi * x)
    p = 1e5 * np.ones(N)
    T = p / (rho * R_GAS)
    g = inputs.grid_dict(N, 1, dx, dx, [inputs.BC_PERIODIC] * 2 + [inputs.BC_ZEROGRAD] * 2)
    U = orc.prim_to_cons(GAS, T[None], p[None], u0 * np.ones((1, N)), np.zeros((1, N)), np.ones((1, 1, N)))
    dt = dt_of(dx)
    n = int(np.ceil(tend / dt))
    U, Tt, st, t, _ = orc.step(GAS, g, U, T[None].copy(), n, dt=tend / n, chem=False)
    assert st == 0
    return U[0, 0], 1 + 0.2 * np.sin(2 * np.pi * (x - u0 * tend))


def test_space_order_five():
    errs = []
    for N in (20, 40, 80):
        rho, ex = _advection(N, lambda dx: 0.5 * dx ** (5 / 3) / 450.0)
        errs.append(np.mean(np.abs(rho - ex)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.7), orders


def test_time_order_three():
    # fixed grid; the error against a 16x finer dt isolates the RK3 error
    N = 40
    ref, _ = _advection(N, lambda dx: 0.05 * dx / 450.0)
    errs = []
    for cfl in (1.2, 0.6, 0.3):
        rho, _ = _advection(N, lambda dx: cfl * dx / 450.0)
        errs.append(np.max(np.abs(rho - ref)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 3.0) < 0.3), orders


def test_freestream_exact():
    st = inputs.tube(H2AIR, 24, 8, ign_frac=0.0)
    U = _cons(H2AIR, st)
    L, Fx, Gy, al = orc.rhs(H2AIR, st["grid"], U, st["T"])
    assert np.all(L == 0.0)


def test_sod_exact_riemann():
    gold = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "sod_star_state.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                gold[k] = float(v)
    ps, us = ref_exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - gold["p_star"]) < 1e-5 and abs(us - gold["u_star"]) < 1e-5
    errs = {}
    for N in (400, 800):
        st = inputs.sod(GAS, N)
        U, T = _cons(GAS, st), st["T"].copy()
        t, tend = 0.0, 0.01
        while t < tend - 1e-15:
            dt = min(orc.cfl_dt(GAS, st["grid"], U, T, 0.2), tend - t)
            U, T, s, tt, _ = orc.step(GAS, st["grid"], U, T, 1, dt=dt, chem=False)
            assert s == 0
            t += tt
        ex = ref_exact.riemann_exact((1.0, 0.0, 1e5), (0.125, 0.0, 1e4), st["x"], tend)
        rho = U[0, 0]
        u = U[1, 0] / rho
        p, _ = orc.primitives(GAS, U, T)
        errs[N] = [np.mean(np.abs(a - b)) / np.mean(np.abs(b)) for a, b in
                   ((rho, ex[0]), (p[0], ex[2]))] + [np.mean(np.abs(u - ex[1])) / us / np.sqrt(1e5)]
    # bounds frozen from the first run at 400 cells (L1(rho) = 3.1e-3)
    assert errs[400][0] < 3.5e-3 and errs[400][1] < 3.5e-3 and errs[400][2] < 1e-2, errs
    # first-order convergence across discontinuities
    assert all(errs[400][i] / errs[800][i] > 1.6 for i in range(3)), errs


# ----------------------------------------------------------------------------
# Thermodynamics and Newton recovery
# ----------------------------------------------------------------------------
def test_thermo_consistency():
    # Eq. 4.4 and 4.5 must integrate Eq. 4.3: dh/dT = cp, ds/dT = cp/T
    for k in range(H2AIR["ns"]):
        for T in (300.0, 900.0, 2000.0, 3500.0):
            h = 1e-5 * T
            cp, _, _ = orc.thermo(H2AIR, k, T)
            _, hp, sp_ = orc.thermo(H2AIR, k, T + h)
            _, hm, sm = orc.thermo(H2AIR, k, T - h)
            assert abs((hp - hm) / (2 * h) - cp) < 1e-8 * cp
            assert abs((sp_ - sm) / (2 * h) - cp / T) < 1e-8 * cp / T
    # anchors of the synthetic table: h(298.15) = formation enthalpy of H2O
    k = H2AIR["species"].index("H2O")
    _, h, _ = orc.thermo(H2AIR, k, 298.15)
    assert abs(h * 8.314472 - (-241.8e3)) < 1e-6 * 241.8e3


def test_newton_recovers_temperature():
    rng = np.random.default_rng(3)
    n = 200
    T = rng.uniform(250.0, 3500.0, n)
    p = rng.uniform(0.3, 80.0, n) * inputs.ATM
    Y = rng.dirichlet(np.ones(H2AIR["ns"]), n).T
    u, v = rng.normal(0, 500, n), rng.normal(0, 500, n)
    U = orc.prim_to_cons(H2AIR, T, p, u, v, Y)
    grid = inputs.grid_dict(n, 1, 1.0, 1.0, [1] * 4)
    for warm in (np.full(n, 1000.0), T * 1.3, T * 0.8):
        Tr, st = orc.newton(H2AIR, grid, U, warm)
        assert st == 0
        assert np.max(np.abs(Tr - T) / T) < 1e-12
    # calorically perfect gas: closed form T = e / cv
    Ug = orc.prim_to_cons(GAS, T, p, u, v, np.ones((1, n)))
    e = Ug[3] / Ug[0] - 0.5 * (Ug[1] ** 2 + Ug[2] ** 2) / Ug[0] ** 2
    Tr, st = orc.newton(GAS, grid, Ug, np.full(n, 500.0))
    assert np.max(np.abs(Tr - e / (2.5 * R_GAS)) / Tr) < 1e-12
    pg, cg = orc.primitives(GAS, Ug, Tr)
    assert np.max(np.abs(cg - np.sqrt(1.4 * R_GAS * Tr)) / cg) < 1e-12
    assert np.max(np.abs(pg - p) / p) < 1e-12


# ----------------------------------------------------------------------------
# Kinetics and point-implicit chemistry
# ----------------------------------------------------------------------------
def _elements_matrix(mech):
    el = mech["elements"]
    names = sorted({e for s in mech["species"] for e in el[s]})
    return np.array([[el[s].get(e, 0) for s in mech["species"]] for e in names], dtype=float)


def test_rates_conserve_mass_and_elements():
    E = _elements_matrix(H2AIR)
    M = H2AIR["M"]
    rng = np.random.default_rng(4)
    for _ in range(50):
        T = rng.uniform(500.0, 3500.0)
        X = 10.0 ** rng.uniform(-6, 2, H2AIR["ns"])
        w = orc.production_rates(H2AIR, T, X)
        scale = np.max(np.abs(w)) + 1e-300
        assert abs(np.sum(w)) <= 1e-12 * scale * H2AIR["ns"]
        assert np.all(np.abs(E @ (w / M)) <= 1e-12 * np.max(np.abs(w / M)) * H2AIR["ns"])
        assert w[-1] == 0.0  # N2 inert


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(5)
    st = inputs.ignition_cell(H2AIR, T0=2200.0, p0=10 * inputs.ATM)
    for trial in range(10):
        Y = rng.dirichlet(np.ones(H2AIR["ns"])) * 0.5 + 0.5 * st["Y"][:, 0, 0]
        U = orc.prim_to_cons(H2AIR, np.array([1500.0 + 200 * trial]), np.array([10 * inputs.ATM]),
                             np.zeros(1), np.zeros(1), Y[:, None])[:, 0]
        T = 1500.0 + 200 * trial
        S, J = orc.source_jacobian(H2AIR, U, T)
        nsp = H2AIR["ns"] - 1
        for l in range(nsp):
            h = 1e-6 * U[4 + l] + 1e-12
            up, um = U.copy(), U.copy()
            up[4 + l] += h
            um[4 + l] -= h
            Sp, _ = orc.source_jacobian(H2AIR, up, T)
            Sm, _ = orc.source_jacobian(H2AIR, um, T)
            fd = (Sp - Sm) / (2 * h)
            assert np.max(np.abs(fd - J[:, l])) <= 1e-6 * (np.max(np.abs(J)) + 1e-300), (trial, l)


def _linear_mech(kf, dh_R=1500.0, ds_R=0.7):
    """A <=> B with an inert carrier N; same heat capacity, offsets in the
    enthalpy and entropy constants so that K_c = exp(ds_R - dh_R / T)."""
    base = [3.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    nasa = np.array([base, base, base])
    nasa[1, 5] = dh_R
    nasa[1, 6] = ds_R
    return {"name": "linear", "species": ["A", "B", "N"], "ns": 3, "nr": 1,
            "M": np.array([0.03, 0.03, 0.028]), "nasa": nasa,
            "A": np.array([kf]), "b": np.zeros(1), "Ea": np.zeros(1),
            "nuf": np.array([[1, 0, 0]], dtype=np.int32), "nub": np.array([[0, 1, 0]], dtype=np.int32),
            "tb": np.zeros(1, dtype=np.int32), "eff": np.ones((1, 3)), "elements": {}}


def test_point_implicit_is_backward_euler_for_linear_source():
    kf, T, dt = 3.0e4, 1200.0, 2e-5
    m = _linear_mech(kf)
    Kc = np.exp(0.7 - 1500.0 / T)
    kb = kf / Kc
    MA, MB = 0.03, 0.03
    rhoA, rhoB, rhoN = 0.4, 0.1, 0.7
    u = np.array([rhoA + rhoB + rhoN, 0.0, 0.0, 1e5, rhoA, rhoB])
    # exact linear system in (rhoA, rhoB): d/dt = A (rhoA, rhoB)
    A = np.array([[-kf, kb], [kf, -kb]])  # equal molar masses
    expect = np.linalg.solve(np.eye(2) - dt * A, np.array([rhoA, rhoB]))
    got, st = orc.point_implicit(m, u[:, None], np.array([T]), dt)
    assert st == 0
    assert np.allclose(got[4:6, 0], expect, rtol=1e-13, atol=0)
    assert abs(got[4, 0] + got[5, 0] - (rhoA + rhoB)) < 1e-15
    _ = MA, MB


def test_point_implicit_reaches_gibbs_equilibrium():
    # repeated point-implicit updates at frozen T converge to S = 0; that
    # composition must minimise the Helmholtz energy (pins Eq. 4.9)
    T = 2600.0
    st = inputs.ignition_cell(H2AIR, T0=T, p0=5 * inputs.ATM)
    U = _cons(H2AIR, st)[:, 0, 0]
    for dt in [1e-9] * 200 + [1e-7] * 200 + [1e-5] * 400:
        U, s = orc.point_implicit(H2AIR, U[:, None], np.array([T]), dt)
        U = U[:, 0]
        assert s == 0
    M = H2AIR["M"]
    c = np.append(U[4:] / M[:-1], (U[0] - U[4:].sum()) / M[-1])
    ceq, res = ref_exact.gibbs_equilibrium(H2AIR, T, c, H2AIR["elements"])
    major = ceq > 1e-3 * ceq.max()
    assert np.max(np.abs(c[major] - ceq[major]) / ceq[major]) < 1e-4, (c, ceq)


def _crossing(t, T, level):
    """Time at which T first reaches ``level`` (linear interpolation)."""
    i = int(np.argmax(T >= level))
    assert i > 0
    return t[i - 1] + (level - T[i - 1]) * (t[i] - t[i - 1]) / (T[i] - T[i - 1])


def test_ignition_delay_matches_independent_stiff_integration():
    T0, p0 = 1500.0, 20 * inputs.ATM
    st = inputs.ignition_cell(H2AIR, T0=T0, p0=p0)
    U0 = _cons(H2AIR, st)
    rho = U0[0, 0, 0]
    Y0 = st["Y"][:, 0, 0]
    t_end = 2.0e-4
    t_eval = np.linspace(0, t_end, 20001)
    R = ref_exact.ConstantVolumeReactor(H2AIR)
    tr, Tr, _ = R.ignition(rho, Y0, T0, t_end, t_eval)
    tau_ref = _crossing(tr, Tr, T0 + 400.0)

    def oracle_run(dt):
        U, T = U0.copy(), st["T"].copy()
        ts, Ts = [0.0], [T0]
        chunk = max(1, int(round(1e-8 / dt)))
        for _ in range(int(round(t_end / dt)) // chunk):
            U, T, s, tt, _ = orc.step(H2AIR, st["grid"], U, T, chunk, dt=dt, chem=True)
            assert s == 0
            ts.append(ts[-1] + tt)
            Ts.append(T[0, 0])
        ts, Ts = np.array(ts), np.array(Ts)
        return _crossing(ts, Ts, T0 + 400.0), Ts[-1]

    tau5, Tend5 = oracle_run(5e-9)  # the paper's adopted dt (Sec. 5.1(2))
    tau10, _ = oracle_run(1e-8)
    assert abs(tau5 - tau_ref) / tau_ref < 0.01, (tau5, tau_ref)
    assert abs(Tend5 - Tr[-1]) / Tr[-1] < 1e-3
    # first order in dt: halving dt roughly halves the delay error
    e5, e10 = abs(tau5 - tau_ref), abs(tau10 - tau_ref)
    assert 1.6 < e10 / e5 < 2.5, (e5, e10, tau_ref)


# ----------------------------------------------------------------------------
# Whole-step invariants on the detonation tube
# ----------------------------------------------------------------------------
def test_tube_conserves_mass_elements_energy():
    st = inputs.tube(H2AIR, 64, 16)
    U = _cons(H2AIR, st)
    T = st["T"].copy()
    U1, T1, s, t, dts = orc.step(H2AIR, st["grid"], U, T, 60, cfl=0.5, chem=True)
    assert s == 0
    iOH = H2AIR["species"].index("OH")
    assert U1[4 + iOH].max() > 1e-6  # chemistry is active in the igniter
    M = H2AIR["M"]
    E = _elements_matrix(H2AIR)

    def totals(U):
        rhoY = np.concatenate([U[4:], (U[0] - U[4:].sum(axis=0))[None]], axis=0)
        moles = rhoY.reshape(H2AIR["ns"], -1).sum(axis=1) / M
        return np.concatenate([[U[0].sum(), U[3].sum()], E @ moles])

    a, b = totals(U), totals(U1)
    assert np.max(np.abs(b - a) / np.abs(a)) < 1e-12, (a, b)


def test_symmetry_and_transpose_bitwise():
    st = inputs.tube(H2AIR, 32, 12)
    # make the state symmetric about the mid-height with a y-dependent T
    y = np.arange(12)
    st["T"] = st["T"] * (1.0 + 0.02 * np.cos(2 * np.pi * (y[:, None] + 0.5) / 12))
    st["T"][6:] = st["T"][5::-1]  # exact mirror image, bit for bit
    U = _cons(H2AIR, st)
    # flux operator only: on this coarse grid the CFL step is far beyond the
    # point-implicit chemistry's stable range (negative species appear)
    U1, T1, s, _, _ = orc.step(H2AIR, st["grid"], U, st["T"].copy(), 25, cfl=0.5, chem=False)
    assert s == 0
    for k in range(U.shape[0]):
        mirrored = U1[k, ::-1, :]
        if k == 2:
            assert np.array_equal(U1[k], -mirrored)
        else:
            assert np.array_equal(U1[k], mirrored)
    # transposition (dx = dy): swap axes and the two momenta
    Ut = np.transpose(U, (0, 2, 1)).copy()
    Ut[[1, 2]] = Ut[[2, 1]]
    gt = dict(st["grid"], nx=st["grid"]["ny"], ny=st["grid"]["nx"])
    Ut1, Tt1, s, _, _ = orc.step(H2AIR, gt, Ut, st["T"].T.copy(), 25, cfl=0.5, chem=False)
    back = np.transpose(Ut1, (0, 2, 1))
    back[[1, 2]] = back[[2, 1]]
    assert np.array_equal(back, U1)
    assert np.array_equal(Tt1.T, T1)


# ----------------------------------------------------------------------------
# Anisotropic spacing (dx != dy): Eq. 4.10 divides the x-flux difference by dx
# and the y-flux difference by dy; the CFL step of Sec. 4.3 uses the smaller
# spacing. A swapped spacing, or a CFL on one axis only, fails one of these.
# ----------------------------------------------------------------------------
def test_transpose_with_swapped_spacing_bitwise():
    """Transposing the state and swapping (nx, dx) with (ny, dy) transposes
    the result bit for bit on a dx != dy tube (the two flux differences are
    summed with one rounding each, which commutes)."""
    st = inputs.tube(H2AIR, 32, 12, Lx=0.05 * 32 / 256, aspect=1.7, perturb_seed=2)
    rng = np.random.default_rng(11)
    st["u"] = rng.normal(0.0, 60.0, st["T"].shape)
    st["v"] = rng.normal(0.0, 60.0, st["T"].shape)
    assert st["grid"]["dy"] == 1.7 * st["grid"]["dx"]
    U = _cons(H2AIR, st)
    U1, T1, s, t1, _ = orc.step(H2AIR, st["grid"], U, st["T"].copy(), 20, cfl=0.5, chem=False)
    assert s == 0
    Ut = np.transpose(U, (0, 2, 1)).copy()
    Ut[[1, 2]] = Ut[[2, 1]]
    g = st["grid"]
    gt = dict(g, nx=g["ny"], ny=g["nx"], dx=g["dy"], dy=g["dx"])
    Ut1, Tt1, s, tt1, _ = orc.step(H2AIR, gt, Ut, st["T"].T.copy(), 20, cfl=0.5, chem=False)
    assert s == 0 and tt1 == t1
    back = np.transpose(Ut1, (0, 2, 1))
    back[[1, 2]] = back[[2, 1]]
    assert np.array_equal(back, U1)
    assert np.array_equal(Tt1.T, T1)


@pytest.mark.parametrize("axis", ["y", "x"])
def test_one_dimensional_state_ignores_the_other_spacing(axis):
    """A reacting state that varies along one axis only, at a fixed dt: its
    flux differences along the other axis are exactly zero, so the result
    must not depend on the other axis' spacing at all, bit for bit. An L that
    divided the varying axis' flux difference by the wrong spacing would
    change with it."""
    n, m = 32, 4
    h = 0.05 / 256
    z = (np.arange(n) + 0.5) / n
    T1 = np.where(z < 0.1, 2000.0, 300.0 * (1.0 + 0.05 * np.sin(6.0 * z)))
    p1 = np.where(z < 0.1, 20.0 * inputs.ATM, inputs.ATM)
    Y = inputs.premix_Y(H2AIR, inputs.TUBE_Y)
    if axis == "y":
        shape, T, p = (n, m), np.repeat(T1[:, None], m, 1), np.repeat(p1[:, None], m, 1)
        bc = [1, 1, 0, 0]
    else:
        shape, T, p = (m, n), np.repeat(T1[None, :], m, 0), np.repeat(p1[None, :], m, 0)
        bc = [0, 0, 1, 1]
    ny, nx = shape
    Yf = np.repeat(Y[:, None, None], ny, 1).repeat(nx, 2)
    z0 = np.zeros(shape)
    U = orc.prim_to_cons(H2AIR, T, p, z0, z0, Yf)
    out = []
    for other in (h, 3.7 * h, 0.31 * h):
        dx, dy = (other, h) if axis == "y" else (h, other)
        g = inputs.grid_dict(nx, ny, dx, dy, bc)
        Un, Tn, s, _, _ = orc.step(H2AIR, g, U, T.copy(), 12, dt=2e-9, chem=True)
        assert s == 0
        out.append((Un, Tn))
    for Un, Tn in out[1:]:
        assert np.array_equal(Un, out[0][0]) and np.array_equal(Tn, out[0][1])
    # and the varying axis moved: the blast has left the igniter
    U0 = out[0][0]
    moved = U0[0, :, 0] if axis == "y" else U0[0, 0, :]
    start = U[0, :, 0] if axis == "y" else U[0, 0, :]
    assert np.max(np.abs(moved - start)) > 1e-3 * np.max(start)


def test_cfl_dt_uses_the_smaller_spacing():
    """dt = CFL min(dx, dy) / max(alpha_x, alpha_y), by hand for a uniform
    calorically perfect gas (c = sqrt(1.4 R T), R = 287): the same dt with the
    spacings swapped, and the larger LF speed in either direction wins."""
    T0, p0 = 300.0, 1e5
    c = np.sqrt(1.4 * R_GAS * T0)
    for (u, v) in ((120.0, -40.0), (30.0, 210.0)):
        one = np.ones((5, 6))
        U = orc.prim_to_cons(GAS, T0 * one, p0 * one, u * one, v * one, one[None])
        expect = 0.5 * 5e-4 / (max(abs(u), abs(v)) + c)
        for dx, dy in ((2e-3, 5e-4), (5e-4, 2e-3)):
            g = inputs.grid_dict(6, 5, dx, dy, [2, 2, 2, 2])
            dt = orc.cfl_dt(GAS, g, U, T0 * one, 0.5)
            assert abs(dt - expect) <= 1e-13 * expect, (u, v, dx, dy, dt, expect)


def _oblique_advection(nx, ny, tend=0.002, u0=100.0, v0=-70.0):
    """Contact wave rho = 1 + 0.2 sin(2 pi x) sin(2 pi y), u, v, p constant,
    periodic unit square with nx != ny (dx != dy). The exact solution is the
    translation by (u0 t, v0 t)."""
    dx, dy = 1.0 / nx, 1.0 / ny
    X, Yc = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)
    rho = 1 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Yc)
    p = 1e5 * np.ones((ny, nx))
    T = p / (rho * R_GAS)
    g = inputs.grid_dict(nx, ny, dx, dy, [inputs.BC_PERIODIC] * 4)
    U = orc.prim_to_cons(GAS, T, p, u0 * np.ones((ny, nx)), v0 * np.ones((ny, nx)), np.ones((1, ny, nx)))
    h = min(dx, dy)
    n = int(np.ceil(tend / (0.5 * h ** (5 / 3) / 450.0)))
    U, _, st, _, _ = orc.step(GAS, g, U, T, n, dt=tend / n, chem=False)
    assert st == 0
    ex = 1 + 0.2 * np.sin(2 * np.pi * (X - u0 * tend)) * np.sin(2 * np.pi * (Yc - v0 * tend))
    return np.mean(np.abs(U[0] - ex))


def test_oblique_advection_on_anisotropic_grid_converges_at_order_five():
    """Both axes at once with dy = 2 dx: the wave must land where the exact
    translation puts it (a spacing applied to the wrong axis moves it at the
    wrong speed, an O(0.1) error that does not converge) and converge at the
    order of WENO5."""
    e1 = _oblique_advection(32, 16)
    e2 = _oblique_advection(64, 32)
    # measured 5.2e-4 and 1.7e-5 (order 4.9); the same data with the two
    # spacings exchanged in the difference ends 8.8e-2 from the translation
    assert e2 < 4e-5, (e1, e2)
    assert np.log2(e1 / e2) > 4.5, (e1, e2)


def test_tangent_model_matches_finite_differences():
    st = inputs.tube(H2AIR, 12, 6)
    rng = np.random.default_rng(7)
    # per-cell T spread so that the global max of Eq. 4.11 has a unique argmax
    st["T"] = st["T"] + rng.normal(0.0, 5.0, st["T"].shape)
    U = _cons(H2AIR, st)
    T = st["T"].copy()
    dt = 0.5 * orc.cfl_dt(H2AIR, st["grid"], U, T, 0.5)
    dT0 = rng.normal(0, 1.0, T.shape)
    # a temperature direction at fixed p and Y, by linearising prim_to_cons
    h = 1e-3
    Up = orc.prim_to_cons(H2AIR, st["T"] + h * dT0, st["p"], st["u"], st["v"], st["Y"])
    Um = orc.prim_to_cons(H2AIR, st["T"] - h * dT0, st["p"], st["u"], st["v"], st["Y"])
    dU0 = (Up - Um) / (2 * h)
    _, _, dU, _, s = orc.step_tangent(H2AIR, st["grid"], U, T, dU0, dT0, 4, dt)
    assert s == 0
    hs = 1e-4
    Ua, _, _, _, _ = orc.step(H2AIR, st["grid"], U + hs * dU0, T + hs * dT0, 4, dt=dt)
    Ub, _, _, _, _ = orc.step(H2AIR, st["grid"], U - hs * dU0, T - hs * dT0, 4, dt=dt)
    fd = (Ua - Ub) / (2 * hs)
    for k in range(U.shape[0]):
        scale = np.max(np.abs(dU[k])) + 1e-300
        assert np.max(np.abs(fd[k] - dU[k])) <= 1e-5 * scale + 1e-12 * np.max(np.abs(U[k])), k


def _smooth_reacting_state(nx, ny):
    """Premixed H2-air at 1150 K with a smooth 80 K bump, smooth p, u, v:
    no discontinuity anywhere, unique arg-max of the LF speeds."""
    X, Yg = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
    T = 1150 + 80 * np.exp(-((X - 0.3) ** 2 + (Yg - 0.4) ** 2) / 0.05)
    p = 2 * inputs.ATM * (1 + 0.05 * np.cos(2 * np.pi * X))
    u = 5 * np.sin(2 * np.pi * Yg)
    v = 3 * np.cos(2 * np.pi * X)
    Y = np.repeat(inputs.h2air_Y(H2AIR, 1.0)[:, None, None], ny, 1).repeat(nx, 2)
    g = inputs.grid_dict(nx, ny, 1e-4, 1e-4, [0, 0, 1, 1])
    return g, T, p, u, v, Y, X, Yg


def test_trajectory_tangent_loss_and_lanes():
    """The trajectory tangent (reference of the adjoint tests): its loss is
    the time-integrated end-wall pressure recomputed step by step with
    step() and primitives(); the 1-lane and 8-lane builds agree; the tangents
    of the loss and of U^N match Richardson-extrapolated central differences.

    The differences use steps of 1.25e-3 and 6.25e-4 K: WENO-JS with an
    absolute eps = 1e-6 on SI-unit fluxes makes the weights nonlinear where
    neighbouring fluxes differ by ~1e-3, so directions that vary across the
    nearly uniform rows only converge below about 1e-2 K."""
    g, T, p, u, v, Y, X, Yg = _smooth_reacting_state(12, 6)
    U = orc.prim_to_cons(H2AIR, T, p, u, v, Y)
    dt, n = 2e-8, 4
    Uc, Tc, L_def = U.copy(), T.copy(), 0.0
    for _ in range(n):
        Uc, Tc, s, _, _ = orc.step(H2AIR, g, Uc, Tc, 1, dt=dt)
        assert s == 0
        L_def += dt * np.mean(orc.primitives(H2AIR, Uc, Tc)[0][:, -1])
    dirs = [np.cos(np.pi * Yg), X, np.cos(np.pi * X) * np.cos(np.pi * Yg)]
    h = 1e-3
    V = np.stack([(orc.prim_to_cons(H2AIR, T + h * d, p, u, v, Y) - orc.prim_to_cons(H2AIR, T - h * d, p, u, v, Y))
                  / (2 * h) for d in dirs])
    dUN8, L8, dL8, s8 = orc.trajectory_tangent(H2AIR, g, U, T, V, n, dt)
    assert s8 == 0
    assert abs(L8 - L_def) <= 1e-13 * abs(L_def)
    for l in range(len(dirs)):
        dUN1, L1, dL1, s1 = orc.trajectory_tangent(H2AIR, g, U, T, V[l:l + 1], n, dt)
        assert s1 == 0 and L1 == L8
        assert abs(dL1[0] - dL8[l]) <= 1e-13 * abs(dL8[l])
        assert np.allclose(dUN1[0], dUN8[l], rtol=1e-12, atol=0)

    def loss_UN(eps, d):
        Te = T + eps * d
        Ue, L = orc.prim_to_cons(H2AIR, Te, p, u, v, Y), 0.0
        for _ in range(n):
            Ue, Te, _, _, _ = orc.step(H2AIR, g, Ue, Te, 1, dt=dt)
            L += dt * np.mean(orc.primitives(H2AIR, Ue, Te)[0][:, -1])
        return L, Ue

    for l, d in enumerate(dirs):
        fd = []
        for hh in (1.25e-3, 6.25e-4):
            (Lp, Up), (Lm, Um) = loss_UN(hh, d), loss_UN(-hh, d)
            fd.append(((Lp - Lm) / (2 * hh), (Up - Um) / (2 * hh)))
        fdL = (4 * fd[1][0] - fd[0][0]) / 3
        fdU = (4 * fd[1][1] - fd[0][1]) / 3
        assert abs(fdL - dL8[l]) <= 1e-5 * abs(dL8[l]), (l, fdL, dL8[l])
        for k in range(U.shape[0]):
            scale = np.max(np.abs(dUN8[l, k]))
            if scale == 0.0:
                continue
            assert np.max(np.abs(fdU[k] - dUN8[l, k])) <= 1e-5 * scale + 1e-13 * np.max(np.abs(U[k])), (l, k)


def _igniting_state(nx=10, ny=4, seed=5):
    st = inputs.tube(H2AIR, nx, ny)
    rng = np.random.default_rng(seed)
    st["T"] = 1400.0 + 200.0 * rng.random(st["T"].shape)
    st["p"] = np.full_like(st["T"], 5 * inputs.ATM)
    st["u"] = rng.normal(0.0, 20.0, st["T"].shape)
    return st, _cons(H2AIR, st)


def test_strang_step_is_half_chemistry_flux_half_chemistry():
    """CHEM_STRANG = chemistry(dt/2), flux RK3(dt), chemistry(dt/2) (the
    Strang order Sec. 4.3 names), assembled here from the oracle's separate
    entry points: point_implicit + newton, and a flux-only step."""
    st, U = _igniting_state()
    g, T = st["grid"], st["T"]
    dt = 2e-8

    def half_chem(U, T):
        Uc, s1 = orc.point_implicit(H2AIR, U, T, 0.5 * dt)
        Tc, s2 = orc.newton(H2AIR, g, Uc, T)
        assert s1 == 0 and s2 == 0
        return Uc, Tc

    Ua, Ta = half_chem(U, T)
    Ub, Tb, s, _, _ = orc.step(H2AIR, g, Ua, Ta, 1, dt=dt, chem=False)
    assert s == 0
    Uc, Tc = half_chem(Ub, Tb)
    Us, Ts, s, _, _ = orc.step(H2AIR, g, U, T, 1, dt=dt, chem=orc.CHEM_STRANG)
    assert s == 0
    assert np.array_equal(Us, Uc) and np.array_equal(Ts, Tc)
    # and the Lie step is flux then a full chemistry step
    Ul, Tl, s, _, _ = orc.step(H2AIR, g, U, T, 1, dt=dt, chem=orc.CHEM_LIE)
    Uf, Tf, _, _, _ = orc.step(H2AIR, g, U, T, 1, dt=dt, chem=False)
    Uf2, _ = orc.point_implicit(H2AIR, Uf, Tf, dt)
    assert np.array_equal(Ul, Uf2)


def test_strang_and_lie_differ_at_second_order_per_step():
    """Both orders split the same two operators, so one step of each differs
    by O(dt^2) (the commutator term): halving dt divides the difference by
    about 4. A missing or doubled half step would leave an O(dt) gap."""
    st, U = _igniting_state()
    g, T = st["grid"], st["T"]
    diffs = []
    for dt in (4e-8, 2e-8, 1e-8):
        Ul, _, s1, _, _ = orc.step(H2AIR, g, U, T, 1, dt=dt, chem=orc.CHEM_LIE)
        Us, _, s2, _, _ = orc.step(H2AIR, g, U, T, 1, dt=dt, chem=orc.CHEM_STRANG)
        assert s1 == 0 and s2 == 0
        diffs.append(np.max(np.abs(Ul[4:] - Us[4:])))
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, (diffs, r1, r2)


def test_explicit_source_is_third_order_rk3():
    """CHEM_EXPLICIT adds the production rates to L(U) in every TVD-RK3 stage
    (the source_terms path of Sec. 4.3). In a 0-D cell the flux terms vanish,
    so a step is RK3 applied to the constant-volume reactor ODE: against an
    independent stiff integration the error falls by about 2^3 per halving
    of dt (one-step global H2-O2 mechanism, gamma = 1.29)."""
    glob = inputs.load_mechanism("global_h2o2_g129")
    Y = inputs.premix_Y(glob, {"H2": 4.032, "O2": 31.998})
    T0, t_end = 2000.0, 2e-6
    st = inputs.ignition_cell(glob, T0=T0, p0=10 * inputs.ATM, Y=Y)
    U0 = orc.prim_to_cons(glob, st["T"], st["p"], st["u"], st["v"], st["Y"])
    R = ref_exact.ConstantVolumeReactor(glob)
    _, _, yr = R.ignition(U0[0, 0, 0], st["Y"][:, 0, 0], T0, t_end, np.array([0.0, t_end]))
    errs = []
    for n in (16, 32, 64):
        U, T, s, _, _ = orc.step(glob, st["grid"], U0, st["T"], n, dt=t_end / n, chem=orc.CHEM_EXPLICIT)
        assert s == 0
        errs.append(np.max(np.abs(U[4:6, 0, 0] / U[0, 0, 0] - yr[:2, -1])))
    assert 1e-9 < errs[-1] < 1e-6, errs
    for a_, b_ in zip(errs, errs[1:]):
        assert 6.0 < a_ / b_ < 9.0, errs
    # and the Lie-split point-implicit step is a different (first-order) scheme
    Ul, _, _, _, _ = orc.step(glob, st["grid"], U0, st["T"], 16, dt=t_end / 16, chem=orc.CHEM_LIE)
    assert np.max(np.abs(Ul[4:6, 0, 0] / Ul[0, 0, 0] - yr[:2, -1])) > 10 * errs[0]


def test_opcount_is_positive_and_fixed():
    g = inputs.grid_dict(8, 4, 1.0, 1.0, [0] * 4)
    ops = orc.opcount(H2AIR, g, 0)
    # a WENO5 reconstruction in its plain textbook form
    assert ops["add"] > 15 and ops["mul"] > 15 and ops["div"] >= 4 and ops["exp"] == 0
