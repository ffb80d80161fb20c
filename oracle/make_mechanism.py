"""Writes the seeded synthetic H2-air mechanism table and the Sod ideal-gas table.

The paper's 9-species / 19-reaction mechanism and its gri30 NASA-7 data
(Sec. 5.1(2)) are not available here, so the tables are synthetic:

* Reaction list: the 19 element-balanced elementary steps of the H2-O2
  system among H2, O2, H, O, OH, HO2, H2O2, H2O with N2 inert except as a
  third body (N2 is the Ns-th species, not carried in U).
* Arrhenius parameters: drawn from a fixed seed inside per-class bounded
  ranges (chain branching, propagation, recombination, dissociation); five
  recombinations and the H2O2 dissociation carry a third body with seeded
  efficiencies for H2 and H2O.
* NASA-7 (single range): a smooth saturating cp/R curve per species class,
  perturbed by the seed and fitted by a quartic in T; a_5 and a_6 are then
  fixed with the oracle's own Eq. 4.4 / Eq. 4.5 so that h(298.15 K) and
  s(298.15 K) equal textbook standard formation enthalpies and entropies.
* Acceptance: the seed is kept when a stoichiometric cell at 1500 K / 20 atm
  ignites (T rises by 400 K) within 5 us .. 200 us under the oracle's own
  point-implicit step (dt = 1e-8 s); otherwise the next seed is tried.

Also writes the one-step global mechanism global_h2o2_g129 (write_global_g129).

Run from the repository root:  python oracle/make_mechanism.py
(python oracle/make_mechanism.py global writes only the global mechanism)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, HERE)
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2504_13750_gb300 import inputs  # noqa: E402

RU = 8.314472
SPECIES = ["H2", "O2", "H", "O", "OH", "HO2", "H2O2", "H2O", "N2"]
ATOMS = {"H2": {"H": 2}, "O2": {"O": 2}, "H": {"H": 1}, "O": {"O": 1}, "OH": {"O": 1, "H": 1},
         "HO2": {"H": 1, "O": 2}, "H2O2": {"H": 2, "O": 2}, "H2O": {"H": 2, "O": 1}, "N2": {"N": 2}}
# Standard-state (298.15 K, 1 atm) formation enthalpy, kJ/mol, and entropy, J/(mol K).
HF298 = {"H2": 0.0, "O2": 0.0, "H": 218.0, "O": 249.2, "OH": 39.0, "HO2": 12.0, "H2O2": -136.1,
         "H2O": -241.8, "N2": 0.0}
S298 = {"H2": 130.7, "O2": 205.2, "H": 114.7, "O": 161.1, "OH": 183.7, "HO2": 229.0, "H2O2": 232.7,
        "H2O": 188.8, "N2": 191.6}
# cp/R near 300 K and its high-temperature plateau, by molecular class.
CP_SHAPE = {"H2": (3.50, 4.40), "O2": (3.55, 4.70), "H": (2.50, 2.50), "O": (2.60, 2.55),
            "OH": (3.55, 4.50), "HO2": (4.20, 6.60), "H2O2": (5.20, 8.40), "H2O": (4.00, 6.60),
            "N2": (3.50, 4.50)}

REACTIONS = [
    ("H + O2 <=> OH + O", {"H": 1, "O2": 1}, {"OH": 1, "O": 1}, False, "branch"),
    ("O + H2 <=> OH + H", {"O": 1, "H2": 1}, {"OH": 1, "H": 1}, False, "branch2"),
    ("H2 + OH <=> H2O + H", {"H2": 1, "OH": 1}, {"H2O": 1, "H": 1}, False, "prop"),
    ("OH + OH <=> H2O + O", {"OH": 2}, {"H2O": 1, "O": 1}, False, "fast"),
    ("H + H + M <=> H2 + M", {"H": 2}, {"H2": 1}, True, "recomb"),
    ("H + OH + M <=> H2O + M", {"H": 1, "OH": 1}, {"H2O": 1}, True, "recomb"),
    ("H + O + M <=> OH + M", {"H": 1, "O": 1}, {"OH": 1}, True, "recomb"),
    ("O + O + M <=> O2 + M", {"O": 2}, {"O2": 1}, True, "recomb"),
    ("H + O2 + M <=> HO2 + M", {"H": 1, "O2": 1}, {"HO2": 1}, True, "recomb"),
    ("HO2 + H <=> H2 + O2", {"HO2": 1, "H": 1}, {"H2": 1, "O2": 1}, False, "fast"),
    ("HO2 + H <=> OH + OH", {"HO2": 1, "H": 1}, {"OH": 2}, False, "fast"),
    ("HO2 + O <=> O2 + OH", {"HO2": 1, "O": 1}, {"O2": 1, "OH": 1}, False, "fast"),
    ("HO2 + OH <=> H2O + O2", {"HO2": 1, "OH": 1}, {"H2O": 1, "O2": 1}, False, "fast"),
    ("HO2 + HO2 <=> H2O2 + O2", {"HO2": 2}, {"H2O2": 1, "O2": 1}, False, "slow"),
    ("H2O2 + M <=> OH + OH + M", {"H2O2": 1}, {"OH": 2}, True, "dissoc"),
    ("H2O2 + H <=> H2O + OH", {"H2O2": 1, "H": 1}, {"H2O": 1, "OH": 1}, False, "mid"),
    ("H2O2 + H <=> HO2 + H2", {"H2O2": 1, "H": 1}, {"HO2": 1, "H2": 1}, False, "mid"),
    ("H2O2 + O <=> HO2 + OH", {"H2O2": 1, "O": 1}, {"HO2": 1, "OH": 1}, False, "mid"),
    ("H2O2 + OH <=> HO2 + H2O", {"H2O2": 1, "OH": 1}, {"HO2": 1, "H2O": 1}, False, "fast"),
]
# Bounded ranges per class: log10 A (SI: m^3/mol/s bimolecular, m^6/mol^2/s
# with a third body on a two-reactant step), temperature exponent b, Ea (kJ/mol).
CLASS_RANGES = {
    "branch": ((7.0, 7.6), (-0.4, 0.0), (66.0, 74.0)),
    "branch2": ((6.4, 7.0), (0.0, 1.0), (28.0, 40.0)),
    "prop": ((6.5, 7.5), (0.0, 1.0), (10.0, 25.0)),
    "fast": ((6.8, 7.8), (-0.3, 0.3), (0.0, 8.0)),
    "slow": ((5.8, 6.8), (0.0, 0.0), (0.0, 6.0)),
    "mid": ((6.2, 7.2), (0.0, 0.0), (10.0, 35.0)),
    "recomb": ((3.8, 5.0), (-1.0, -0.3), (0.0, 0.0)),
    "dissoc": ((10.5, 11.5), (0.0, 0.0), (180.0, 200.0)),
}


def molar_mass(sp):
    return sum(n * inputs.ATOMIC_MASS[a] for a, n in ATOMS[sp].items())


def check_balance():
    for eq, re, pr, _, _ in REACTIONS:
        for el in ("H", "O", "N"):
            lhs = sum(n * ATOMS[s].get(el, 0) for s, n in re.items())
            rhs = sum(n * ATOMS[s].get(el, 0) for s, n in pr.items())
            assert lhs == rhs, eq


def cp_curve(lo, hi, T, theta=1100.0):
    return lo + (hi - lo) * (1.0 - np.exp(-np.maximum(T - 300.0, 0.0) / theta))


def fit_nasa(lo, hi):
    """Quartic cp/R(T) fit of the saturating curve over 200..6000 K."""
    T = np.linspace(200.0, 6000.0, 400)
    t = T / 1000.0
    c = np.polyfit(t, cp_curve(lo, hi, T), 4)[::-1]  # ascending powers of t
    return [c[0], c[1] / 1e3, c[2] / 1e6, c[3] / 1e9, c[4] / 1e12]


def build_table(seed: int) -> dict:
    rng = np.random.default_rng(seed)
    nasa = []
    for sp in SPECIES:
        lo, hi = CP_SHAPE[sp]
        f = 1.0 + rng.uniform(-0.03, 0.03)
        nasa.append(fit_nasa(lo * f, hi * f) + [0.0, 0.0])
    mech = {"species": SPECIES, "M": [molar_mass(s) for s in SPECIES], "nasa7": nasa, "reactions": []}
    # a_5, a_6 from the standard-state anchors, with the oracle's Eq. 4.4 / 4.5.
    flat = _flat(mech)
    for k, sp in enumerate(SPECIES):
        cp, h, s = orc.thermo(flat, k, 298.15)
        nasa[k][5] = HF298[sp] * 1e3 / RU - h
        nasa[k][6] = S298[sp] / RU - s
    for eq, re, pr, tb, cls in REACTIONS:
        (la, lb), (ba, bb), (ea, eb) = CLASS_RANGES[cls]
        r = {"equation": eq, "reactants": re, "products": pr,
             "A": float(10.0 ** rng.uniform(la, lb)), "b": float(rng.uniform(ba, bb)),
             "Ea": float(rng.uniform(ea, eb) * 1e3), "third_body": tb}
        if tb:
            r["efficiencies"] = {"H2": float(rng.uniform(2.0, 3.0)), "H2O": float(rng.uniform(5.0, 12.0))}
        mech["reactions"].append(r)
    return mech


def _flat(mech):
    tmp = os.path.join(HERE, "_build", "_mech_tmp.json")
    os.makedirs(os.path.dirname(tmp), exist_ok=True)
    with open(tmp, "w") as f:
        json.dump(mech, f)
    return inputs.load_mechanism(tmp)


def ignition_delay(flat, T0=1500.0, p0=20 * inputs.ATM, dt=1e-8, t_max=5e-4, chunk=20):
    st = inputs.ignition_cell(flat, T0=T0, p0=p0)
    U = orc.prim_to_cons(flat, st["T"], st["p"], st["u"], st["v"], st["Y"])
    T = st["T"].copy()
    t = 0.0
    while t < t_max:
        U, T, status, tt, _ = orc.step(flat, st["grid"], U, T, chunk, dt=dt, chem=True)
        t += tt
        if status != 0:
            return None
        if T[0, 0] > T0 + 400.0:
            return t
    return None


def write_global_g129(out_dir):
    """One-step global H2-O2 mechanism on a calorically perfect gas with
    gamma = 1.29 (the fixed-gamma, single-step setting of Sec. 6.2; its
    parameters are not printed in the paper, so these are synthetic):
    cp/R = gamma / (gamma - 1) for every species; formation enthalpy of H2O
    scaled to -60 kJ/mol (an adiabatic rise of about 2000 K for the
    stoichiometric mixture) and its standard entropy set to 240 J/(mol K) so
    that the equilibrium lies on the product side up to about 4000 K;
    2 H2 + O2 => 2 H2O, mass action of order 3, A = 1e5 (m^3/mol)^2/s,
    b = 0, Ea = 120 kJ/mol (slow enough for an explicit RK3 source at
    CFL 0.5 on 0.1 mm cells)."""
    gamma = 1.29
    a0 = gamma / (gamma - 1.0)
    hf = {"H2": 0.0, "O2": 0.0, "H2O": -60.0e3}
    s298 = {"H2": 130.7, "O2": 205.2, "H2O": 240.0}
    species = ["H2", "O2", "H2O"]
    nasa = []
    for sp in species:
        a5 = hf[sp] / RU - a0 * 298.15
        a6 = s298[sp] / RU - a0 * np.log(298.15)
        nasa.append([a0, 0.0, 0.0, 0.0, 0.0, a5, a6])
    mech = {"name": "global_h2o2_g129", "species": species, "M": [molar_mass(sp) for sp in species],
            "nasa7": nasa,
            "reactions": [{"equation": "2 H2 + O2 <=> 2 H2O", "reactants": {"H2": 2, "O2": 1},
                           "products": {"H2O": 2}, "A": 1.0e5, "b": 0.0, "Ea": 1.2e5, "third_body": False,
                           "efficiencies": {}}],
            "units": "SI: M kg/mol; A in (m^3/mol)^2/s; Ea J/mol; NASA-7 single range, dimensionless",
            "provenance": "synthetic, written by oracle/make_mechanism.py (write_global_g129)",
            "elements": {sp: ATOMS[sp] for sp in species}}
    with open(os.path.join(out_dir, "global_h2o2_g129.json"), "w") as f:
        json.dump(mech, f, indent=1)


def main():
    if sys.argv[1:] == ["global"]:
        write_global_g129(os.path.join(ROOT, "paper_2504_13750_gb300", "mechanisms"))
        return
    check_balance()
    out_dir = os.path.join(ROOT, "paper_2504_13750_gb300", "mechanisms")
    os.makedirs(out_dir, exist_ok=True)
    for seed in range(0, 100):
        mech = build_table(seed)
        flat = _flat(mech)
        tau = ignition_delay(flat)
        print(f"seed {seed}: ignition delay at 1500 K / 20 atm = {tau}")
        if tau is not None and 5e-6 <= tau <= 2e-4:
            mech.update({
                "name": "h2air_synth",
                "seed": seed,
                "ignition_delay_1500K_20atm_s": tau,
                "units": "SI: M kg/mol; A in (m^3/mol)^(order-1)/s with a third body counted in the order; "
                         "Ea J/mol; NASA-7 single range, dimensionless",
                "provenance": "synthetic, written by oracle/make_mechanism.py; no published mechanism values",
                "elements": {s: ATOMS[s] for s in SPECIES},
            })
            with open(os.path.join(out_dir, "h2air_synth.json"), "w") as f:
                json.dump(mech, f, indent=1)
            break
    ideal = {"name": "ideal_gamma14", "species": ["GAS"], "M": [RU / 287.0],
             "nasa7": [[3.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]], "reactions": [],
             "units": "calorically perfect gas, cp/R = 3.5 (gamma = 1.4), R = 287 J/(kg K)",
             "provenance": "Sod shock tube gas of Sec. 5.1(1)"}
    with open(os.path.join(out_dir, "ideal_gamma14.json"), "w") as f:
        json.dump(ideal, f, indent=1)
    write_global_g129(out_dir)


if __name__ == "__main__":
    main()
