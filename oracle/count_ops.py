"""Writes tests/golden/oracle_opcounts.json: algorithmic FP64 operation counts
of the plain algorithm, taken with the oracle's operation-counting scalar.

  weno5           one WENO5-JS reconstruction (Jiang & Shu form)
  rhs_per_cell    one right-hand side L(U) (Eq. 4.10-4.11 + WENO5) per cell,
                  on a 64 x 16 tube state (includes ghost-cell work)
  newton_per_cell one warm-started Newton T recovery per cell (stage-like
                  change of state, so the iteration count is representative)
  chem_per_cell   one point-implicit chemistry update per cell (Eq. 4.12-4.13)
  step_per_cell   one full step per cell (CFL dt, RK3, chemistry)
Division, square root, exp and log are counted separately; the 'flops'
entry counts add + mul + div + sqrt (exp and log are listed, not weighted).

Run from the repository root: python oracle/count_ops.py
"""
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


def flops(c):
    return c["add"] + c["mul"] + c["div"] + c["sqrt"]


def main():
    mech = inputs.load_mechanism("h2air_synth")
    st = inputs.tube(mech, 64, 16, perturb_seed=0)
    g = st["grid"]
    U = orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])
    T = st["T"]
    n = g["nx"] * g["ny"]
    dt = orc.cfl_dt(mech, g, U, T, 0.5)
    # a state one step in, so Newton starts from a changed state
    U1, T1, s, _, _ = orc.step(mech, g, U, T, 1, dt=dt)
    out = {"mechanism": mech["name"], "grid": [g["nx"], g["ny"]]}
    out["weno5"] = orc.opcount(mech, g, 0)
    for name, part in (("rhs_per_cell", 1), ("chem_per_cell", 3), ("step_per_cell", 4)):
        c = orc.opcount(mech, g, part, U1, T1, dt)
        out[name] = {k: v / n for k, v in c.items()}
    # Newton: recover T of U1 warm-started from T (one step earlier)
    W = orc.opcount(mech, g, 2, U1, T)
    out["newton_per_cell"] = {k: v / n for k, v in W.items()}
    for k in ("weno5", "rhs_per_cell", "chem_per_cell", "step_per_cell", "newton_per_cell"):
        out[k]["flops"] = flops(out[k])
    path = os.path.join(ROOT, "tests", "golden", "oracle_opcounts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
