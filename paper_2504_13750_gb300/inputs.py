"""Seeded synthetic inputs: mechanism tables and initial fields.

This module holds data and random draws only. It contains none of the
solver's arithmetic (no EOS, thermo, kinetics or flux code): it returns
primitive fields (T, p, u, v, mass fractions) and flat mechanism arrays, and
each consumer converts them with its own code. It is the one module that both
the CUDA path's callers and the oracle's tests read from.

Workloads (stand-ins for the paper's detonation tube of Sec. 5.2.1 and its
validation cases of Sec. 5.1; no external dataset is involved):
  * ``tube``: 2D H2-O2-N2 detonation tube, L_x = 0.05 m, dx = dy = L_x/n_x,
    premixed Y(H2:O2:N2) = 0.028:0.226:0.746 at 300 K / 1 atm, left 5 % at
    2000 K / 20 atm, slip walls, optional seeded 1 % sinusoidal density
    perturbation at fixed pressure in the unburnt gas.
  * ``sod``: Sod shock tube of Sec. 5.1(1), x in [-10, 10] m.
  * ``ignition_cell``: one cell at constant volume, Sec. 5.1(2).
  * ``serving_requests``: Poisson-arriving solves of mixed size and mixture.
  * ``adjoint_case``: tube with a seeded per-cell initial T perturbation.
"""
from __future__ import annotations

import json
import os

import numpy as np

ATM = 101325.0
_MECH_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mechanisms")

BC_WALL, BC_ZEROGRAD, BC_PERIODIC = 0, 1, 2

# Standard atomic masses, kg/mol.
ATOMIC_MASS = {"H": 1.00794e-3, "O": 15.9994e-3, "N": 14.0067e-3, "Ar": 39.948e-3}


def mechanism_path(name: str) -> str:
    if os.path.isfile(name):
        return name
    return os.path.join(_MECH_DIR, name if name.endswith(".json") else name + ".json")


def load_mechanism(name: str = "h2air_synth") -> dict:
    """Mechanism table as flat arrays.

    Keys: name, species (list), ns, nr, M[ns] (kg/mol), nasa[ns, 7],
    A[nr], b[nr], Ea[nr] (SI; Ea in J/mol), nuf[nr, ns], nub[nr, ns] (int32),
    tb[nr] (int32, 1 = third-body reaction), eff[nr, ns] (third-body
    coefficients), equations (list of str). The last species is the one not
    carried in the conserved vector.
    """
    with open(mechanism_path(name)) as f:
        d = json.load(f)
    sp = list(d["species"])
    ns = len(sp)
    rx = d.get("reactions", [])
    nr = len(rx)
    idx = {s: i for i, s in enumerate(sp)}
    nuf = np.zeros((nr, ns), dtype=np.int32)
    nub = np.zeros((nr, ns), dtype=np.int32)
    eff = np.ones((nr, ns))
    tb = np.zeros(nr, dtype=np.int32)
    A = np.zeros(nr)
    b = np.zeros(nr)
    Ea = np.zeros(nr)
    for i, r in enumerate(rx):
        for s, n in r["reactants"].items():
            nuf[i, idx[s]] += int(n)
        for s, n in r["products"].items():
            nub[i, idx[s]] += int(n)
        A[i], b[i], Ea[i] = float(r["A"]), float(r["b"]), float(r["Ea"])
        if r.get("third_body", False):
            tb[i] = 1
            for s, e in r.get("efficiencies", {}).items():
                eff[i, idx[s]] = float(e)
    return {
        "name": d.get("name", name), "species": sp, "ns": ns, "nr": nr,
        "M": np.asarray(d["M"], dtype=np.float64),
        "nasa": np.asarray(d["nasa7"], dtype=np.float64).reshape(ns, 7),
        "A": A, "b": b, "Ea": Ea, "nuf": nuf, "nub": nub, "tb": tb, "eff": eff,
        "equations": [r.get("equation", "") for r in rx],
        "elements": d.get("elements", {}),
    }


def grid_dict(nx, ny, dx, dy, bc, weno_eps=1e-6, newton_tol=1e-12, newton_maxit=50) -> dict:
    return {"nx": int(nx), "ny": int(ny), "dx": float(dx), "dy": float(dy), "bc": [int(x) for x in bc],
            "weno_eps": float(weno_eps), "newton_tol": float(newton_tol), "newton_maxit": int(newton_maxit)}


def premix_Y(mech: dict, mass: dict) -> np.ndarray:
    """Mass-fraction vector [ns] from a dict species -> mass share (normalised)."""
    Y = np.zeros(mech["ns"])
    for s, v in mass.items():
        Y[mech["species"].index(s)] = v
    return Y / Y.sum()


def h2air_Y(mech: dict, phi: float) -> np.ndarray:
    """H2-air mass fractions at equivalence ratio phi: moles H2 : O2 : N2 = 2 phi : 1 : 3.76."""
    moles = {"H2": 2.0 * phi, "O2": 1.0, "N2": 3.76}
    M = dict(zip(mech["species"], mech["M"]))
    return premix_Y(mech, {s: n * M[s] for s, n in moles.items()})


TUBE_Y = {"H2": 0.028, "O2": 0.226, "N2": 0.746}


def tube(mech: dict, nx: int, ny: int, Lx: float = 0.05, T0=300.0, p0=ATM, Ti=2000.0, pi=20 * ATM,
         ign_frac=0.05, Y=None, perturb_seed=None, perturb_amp=0.01, aspect=1.0):
    """Detonation-tube initial state (primitive fields, each [ny, nx]).

    Returns dict(T, p, u, v, Y[ns, ny, nx], grid). dx = Lx / nx and
    dy = aspect * dx (Ly = ny * dy). Cells whose centre lies at
    x < ign_frac * Lx form the igniter. With ``perturb_seed`` the unburnt gas
    gets rho -> rho (1 + amp sin(2 pi m y / Ly + phase)) at fixed p, i.e.
    T -> T / (1 + amp sin(...)), with m in {2..8} and phase in [0, 2 pi) drawn
    from the seed.
    """
    dx = Lx / nx
    dy = float(aspect) * dx
    Ly = ny * dy
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Yc = np.meshgrid(x, y)
    ign = X < ign_frac * Lx
    T = np.where(ign, Ti, T0).astype(np.float64)
    p = np.where(ign, pi, p0).astype(np.float64)
    if perturb_seed is not None:
        rng = np.random.default_rng(perturb_seed)
        m = int(rng.integers(2, 9))
        ph = float(rng.uniform(0.0, 2 * np.pi))
        fac = 1.0 + perturb_amp * np.sin(2 * np.pi * m * Yc / Ly + ph)
        T = np.where(ign, T, T / fac)
    Yv = premix_Y(mech, TUBE_Y) if Y is None else np.asarray(Y, dtype=np.float64)
    Yf = np.broadcast_to(Yv[:, None, None], (mech["ns"], ny, nx)).copy()
    z = np.zeros((ny, nx))
    return {"T": T, "p": p, "u": z.copy(), "v": z.copy(), "Y": Yf,
            "grid": grid_dict(nx, ny, dx, dy, [BC_WALL] * 4)}


def sod(mech: dict, nx: int = 400, R_gas: float = 287.0):
    """Sod shock tube (Sec. 5.1(1)): x in [-10, 10] m, one row of cells,
    zero-gradient boundaries, (rho, u, p) = (1, 0, 1e5) left of x = 0 and
    (0.125, 0, 1e4) right of it. T = p / (rho R_gas) for the given gas constant."""
    dx = 20.0 / nx
    x = -10.0 + (np.arange(nx) + 0.5) * dx
    rho = np.where(x < 0.0, 1.0, 0.125)
    p = np.where(x < 0.0, 1e5, 1e4)
    T = p / (rho * R_gas)
    z = np.zeros(nx)
    return {"T": T[None, :], "p": p[None, :].astype(np.float64), "u": z[None, :].copy(), "v": z[None, :].copy(),
            "Y": np.ones((mech["ns"], 1, nx)), "x": x,
            "grid": grid_dict(nx, 1, dx, dx, [BC_ZEROGRAD] * 4)}


def ignition_cell(mech: dict, T0=1500.0, p0=20 * ATM, Y=None):
    """One cell at constant volume (Sec. 5.1(2)): zero-gradient on all sides."""
    Yv = premix_Y(mech, TUBE_Y) if Y is None else np.asarray(Y, dtype=np.float64)
    one = np.ones((1, 1))
    return {"T": T0 * one, "p": p0 * one, "u": 0 * one, "v": 0 * one, "Y": Yv[:, None, None] * one,
            "grid": grid_dict(1, 1, 1e-3, 1e-3, [BC_ZEROGRAD] * 4)}


SERVING_GRIDS = ((128, 16), (256, 32), (512, 64), (1024, 128), (2048, 256))


def serving_requests(mech: dict, n: int = 256, seed: int = 1, rate_hz: float = 50.0,
                     steps_range=(100, 1000), grids=SERVING_GRIDS):
    """Seeded request stream: list of dicts with arrival time (s), grid size,
    equivalence ratio phi ~ U[0.5, 1.5], p0 ~ U[0.5, 2] atm, step count
    ~ U{steps_range}. The state of each request is ``tube`` with that mixture,
    300 K / p0 premix, igniter 2000 K / 20 p0."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    out = []
    for r in range(n):
        nx, ny = grids[int(rng.integers(0, len(grids)))]
        phi = float(rng.uniform(0.5, 1.5))
        p0 = float(rng.uniform(0.5, 2.0)) * ATM
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append({"id": r, "arrival": float(t[r]), "nx": nx, "ny": ny, "phi": phi, "p0": p0, "steps": steps})
    return out


def request_state(mech: dict, req: dict):
    return tube(mech, req["nx"], req["ny"], p0=req["p0"], pi=20.0 * req["p0"], Y=h2air_Y(mech, req["phi"]))


def adjoint_case(mech: dict, nx: int = 512, ny: int = 64, seed: int = 2, sigma_T: float = 5.0):
    """Tube layout with a per-cell initial temperature perturbation dT ~ N(0, sigma_T)
    applied at fixed p and Y. Returns (state dict, dT0 [ny, nx])."""
    st = tube(mech, nx, ny)
    rng = np.random.default_rng(seed)
    dT = rng.normal(0.0, sigma_T, size=(ny, nx))
    return st, dT
