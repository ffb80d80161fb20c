"""Independent references used to pin the oracle (test helpers, no solver code shared).

* ``riemann_exact``: exact solution of the 1D Riemann problem for a
  calorically perfect gas (pressure function root by Newton, then sampling of
  the self-similar solution; E. F. Toro, "Riemann Solvers and Numerical
  Methods for Fluid Dynamics", ch. 4), written from the mathematics.
* ``ConstantVolumeReactor``: a numpy restatement of Eq. 4.3-4.9 of arXiv
  2504.13750 integrated with scipy's Radau method at tight tolerances, for the
  ignition comparison of Sec. 5.1(2). It shares no code with the oracle.
* ``gibbs_equilibrium``: composition at fixed T and V that minimises the
  Helmholtz free energy under element conservation (scipy.optimize), the
  thermodynamic statement that detailed balance through Eq. 4.9 must reach.
"""
from __future__ import annotations

import numpy as np

RU = 8.314472
P0 = 101325.0


# ----------------------------------------------------------------------------
# Exact Riemann solver, ideal gas with constant gamma.
# ----------------------------------------------------------------------------
def _pressure_fn(p, rho, pk, ck, g):
    if p > pk:  # shock branch
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction branch
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4):
    """(p*, u*) of the Riemann problem with states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dfl = _pressure_fn(p, rl, pl, cl, g)
        fr, dfr = _pressure_fn(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(p - dp, 1e-12 * p)
        if abs(p_new - p) <= 1e-14 * p_new:
            p = p_new
            break
        p = p_new
    fl, _ = _pressure_fn(p, rl, pl, cl, g)
    fr, _ = _pressure_fn(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_exact(left, right, x, t, g=1.4, x0=0.0):
    """(rho, u, p) sampled at positions x at time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    gm = (g - 1.0) / (g + 1.0)
    out = np.zeros((3, len(x)))
    for n, xi in enumerate((np.asarray(x) - x0) / t):
        if xi <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - cl * np.sqrt((g + 1.0) / (2 * g) * ps / pl + (g - 1.0) / (2 * g))
                out[:, n] = (rl, ul, pl) if xi <= sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2 * g))
                if xi <= ul - cl:
                    out[:, n] = (rl, ul, pl)
                elif xi >= us - cs:
                    out[:, n] = (rs, us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2 * ul + xi)
                    c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2 * (ul - xi))
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    out[:, n] = (r, u, pl * (c / cl) ** (2 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + cr * np.sqrt((g + 1.0) / (2 * g) * ps / pr + (g - 1.0) / (2 * g))
                out[:, n] = (rs, us, ps) if xi <= sr else (rr, ur, pr)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2 * g))
                if xi >= ur + cr:
                    out[:, n] = (rr, ur, pr)
                elif xi <= us + cs:
                    out[:, n] = (rs, us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2 * ur + xi)
                    c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2 * (ur - xi))
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    out[:, n] = (r, u, pr * (c / cr) ** (2 * g / (g - 1.0)))
    return out


# ----------------------------------------------------------------------------
# Constant-volume reactor (numpy restatement of Eq. 4.3-4.9) for scipy.
# ----------------------------------------------------------------------------
class ConstantVolumeReactor:
    def __init__(self, mech):
        self.ns = mech["ns"]
        self.M = np.asarray(mech["M"])
        self.a = np.asarray(mech["nasa"])
        self.A, self.b, self.Ea = (np.asarray(mech[k]) for k in ("A", "b", "Ea"))
        self.nuf = np.asarray(mech["nuf"], dtype=float)
        self.nub = np.asarray(mech["nub"], dtype=float)
        self.tb = np.asarray(mech["tb"], dtype=bool)
        self.eff = np.asarray(mech["eff"])
        self.nu = self.nub - self.nuf

    # per-mole dimensionless thermo of all species at T
    def cp_R(self, T):
        a = self.a
        return a[:, 0] + T * (a[:, 1] + T * (a[:, 2] + T * (a[:, 3] + T * a[:, 4])))

    def h_RT(self, T):
        a = self.a
        poly = a[:, 0] + T * (a[:, 1] / 2 + T * (a[:, 2] / 3 + T * (a[:, 3] / 4 + T * a[:, 4] / 5)))
        return poly + a[:, 5] / T

    def s_R(self, T):
        a = self.a
        return a[:, 0] * np.log(T) + T * (a[:, 1] + T * (a[:, 2] / 2 + T * (a[:, 3] / 3 + T * a[:, 4] / 4))) + a[:, 6]

    def internal_energy(self, Y, T):
        """Mass-specific internal energy e = sum Y_k (h_k - Ru T / M_k)."""
        return float(np.sum(Y * RU * T / self.M * (self.h_RT(T) - 1.0)))

    def temperature(self, Y, e, T0):
        T = T0
        for _ in range(100):
            f = self.internal_energy(Y, T) - e
            cv = float(np.sum(Y * RU / self.M * (self.cp_R(T) - 1.0)))
            dT = -f / cv
            T += dT
            if abs(dT) < 1e-13 * T:
                break
        return T

    def rates(self, T, X):
        """Production rates (kg/m^3/s) of all species."""
        lnT = np.log(T)
        kf = self.A * np.exp(self.b * lnT - self.Ea / (RU * T))
        g = self.s_R(T) - self.h_RT(T)  # dimensionless, per species
        dnu = self.nu.sum(axis=1)
        Kc = np.exp(self.nu @ g) * (P0 / (RU * T)) ** dnu
        kb = kf / Kc
        fwd = kf * np.prod(np.where(self.nuf > 0, X[None, :] ** self.nuf, 1.0), axis=1)
        bwd = kb * np.prod(np.where(self.nub > 0, X[None, :] ** self.nub, 1.0), axis=1)
        third = np.where(self.tb, self.eff @ X, 1.0)
        q = third * (fwd - bwd)
        return self.M * (self.nu.T @ q)

    def ignition(self, rho, Y0, T0, t_end, t_eval):
        from scipy.integrate import solve_ivp

        e = self.internal_energy(Y0, T0)
        Tcache = [T0]

        def f(t, Y):
            T = self.temperature(Y, e, Tcache[0])
            Tcache[0] = T
            return self.rates(T, rho * Y / self.M) / rho

        sol = solve_ivp(f, (0.0, t_end), Y0, method="Radau", rtol=1e-10, atol=1e-14, t_eval=t_eval)
        T = np.array([self.temperature(sol.y[:, i], e, T0 if i == 0 else 2000.0) for i in range(sol.y.shape[1])])
        return sol.t, T, sol.y


def gibbs_equilibrium(mech, T, conc0, elements):
    """Equilibrium molar concentrations at fixed T and volume: minimise
    sum_k c_k (g_k/(Ru T) + ln(c_k Ru T / P0) - 1) subject to element totals.
    ``elements`` maps species -> {element: count}."""
    from scipy.optimize import minimize

    R = ConstantVolumeReactor(mech)
    g = R.h_RT(T) - R.s_R(T)
    sp = mech["species"]
    els = sorted({e for s in sp for e in elements[s]})
    E = np.array([[elements[s].get(e, 0) for s in sp] for e in els], dtype=float)
    b = E @ conc0
    lc = np.log(RU * T / P0)

    def obj(z):
        c = np.exp(z)
        return float(np.sum(c * (g + z + lc - 1.0)))

    def jac(z):
        c = np.exp(z)
        return c * (g + z + lc)

    cons = {"type": "eq", "fun": lambda z: (E @ np.exp(z) - b) / b, "jac": lambda z: (E * np.exp(z)[None, :]) / b[:, None]}
    z0 = np.log(np.maximum(conc0, 1e-8 * conc0.max()))
    res = minimize(obj, z0, jac=jac, constraints=[cons], method="SLSQP", options={"maxiter": 2000, "ftol": 1e-15})
    return np.exp(res.x), res
