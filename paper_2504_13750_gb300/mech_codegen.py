"""Writes csrc/janc_mech_fixed.cuh: the reaction structure of the shipped
H2-air mechanism (mechanisms/h2air_synth.json) as compile-time constants.

The structure is what the chemistry kernels index by: each reaction's
reactant and product species with their stoichiometric coefficients (Eq. 4.6),
whether it carries the third-body factor of Eq. 4.7, and which species have a
third-body coefficient other than one. With it compiled in, every index of
the per-cell rates, Jacobian and production arrays is a constant, so those
arrays live in registers. The numbers (A, b, Ea, the coefficients' values, the
thermodynamic fits) stay run-time data. A grid whose mechanism has this
structure takes the compiled kernels; any other mechanism takes the generic
ones, which run the same operations in the same order.

Run by build.build() before compiling (it rewrites the header only when its
text changes); `python -m paper_2504_13750_gb300.mech_codegen` prints it.
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "mechanisms", "h2air_synth.json")
HEADER = os.path.join(HERE, "csrc", "janc_mech_fixed.cuh")
MAX_SIDE = 3


def structure(path: str = SOURCE):
    """(species, reactions) with reactions as dicts: reactants / products as
    [(species index, coefficient)] in species order, tb, eff_ne1 (species
    indices whose third-body coefficient is not one, in species order)."""
    with open(path) as f:
        d = json.load(f)
    sp = list(d["species"])
    idx = {s: k for k, s in enumerate(sp)}
    out = []
    for r in d["reactions"]:
        nuf = [0] * len(sp)
        nub = [0] * len(sp)
        for s, n in r["reactants"].items():
            nuf[idx[s]] += int(n)
        for s, n in r["products"].items():
            nub[idx[s]] += int(n)
        tb = 1 if r.get("third_body", False) else 0
        eff = [1.0] * len(sp)
        for s, e in r.get("efficiencies", {}).items():
            eff[idx[s]] = float(e)
        out.append({
            "reactants": [(k, nuf[k]) for k in range(len(sp)) if nuf[k]],
            "products": [(k, nub[k]) for k in range(len(sp)) if nub[k]],
            "tb": tb,
            "eff_ne1": [k for k in range(len(sp)) if tb and eff[k] != 1.0],
            "nuf": nuf, "nub": nub,
        })
    return sp, out


def _sel(values, default):
    """A constexpr selector expression over r: values[r] for r < len, else default."""
    expr = str(default)
    for k in range(len(values) - 1, -1, -1):
        expr = f"r == {k} ? {values[k]} : ({expr})"
    return expr


def render(path: str = SOURCE) -> str:
    sp, rx = structure(path)
    ns, nr = len(sp), len(rx)
    for r in rx:
        if len(r["reactants"]) > MAX_SIDE or len(r["products"]) > MAX_SIDE:
            raise ValueError("more than 3 species on one side of a reaction")
    L = []
    L.append("// Generated by paper_2504_13750_gb300/mech_codegen.py from mechanisms/h2air_synth.json;")
    L.append("// regenerate instead of editing. The reaction structure (Eq. 4.6-4.7) of the shipped")
    L.append("// H2-air mechanism as compile-time constants: species " + ", ".join(f"{k} {s}" for k, s in enumerate(sp)) + ".")
    L.append("#pragma once")
    L.append("")
    L.append("namespace janc {")
    L.append("namespace fixed_h2air {")
    L.append("")
    L.append(f"constexpr int NS = {ns};")
    L.append(f"constexpr int NR = {nr};")
    L.append("")
    L.append("// Reaction I: reactant / product species and coefficients in species order,")
    L.append("// the sum of product minus reactant coefficients, the third-body flag and the")
    L.append("// species whose third-body coefficient differs from one (in species order).")
    L.append("template <int I>")
    L.append("struct Rx;")
    for i, r in enumerate(rx):
        re, pr = r["reactants"], r["products"]
        dnu = sum(n for _, n in pr) - sum(n for _, n in re)
        L.append("template <>")
        L.append(f"struct Rx<{i}> {{")
        L.append(f"  static constexpr int i = {i}, nre = {len(re)}, npr = {len(pr)}, dnu = {dnu}, tb = {r['tb']}, "
                 f"neff = {len(r['eff_ne1'])};")
        L.append(f"  __host__ __device__ static constexpr int rsp(int r) {{ return {_sel([k for k, _ in re], -1)}; }}")
        L.append(f"  __host__ __device__ static constexpr int rnu(int r) {{ return {_sel([n for _, n in re], 0)}; }}")
        L.append(f"  __host__ __device__ static constexpr int psp(int r) {{ return {_sel([k for k, _ in pr], -1)}; }}")
        L.append(f"  __host__ __device__ static constexpr int pnu(int r) {{ return {_sel([n for _, n in pr], 0)}; }}")
        L.append(f"  __host__ __device__ static constexpr int effsp(int r) {{ return {_sel(r['eff_ne1'], -1)}; }}")
        L.append("};")
    L.append("")
    L.append("// The same structure as plain tables, for the host-side match of a run-time")
    L.append("// mechanism: nuf / nub [NR][NS], tb [NR], eff_ne1 [NR][NS] (1 where the")
    L.append("// third-body coefficient of a third-body reaction is not one).")
    for name, key in (("kNuf", "nuf"), ("kNub", "nub")):
        L.append(f"constexpr int {name}[NR * NS] = {{")
        for r in rx:
            L.append("    " + ", ".join(str(v) for v in r[key]) + ",")
        L.append("};")
    L.append("constexpr int kTb[NR] = {" + ", ".join(str(r["tb"]) for r in rx) + "};")
    L.append("constexpr int kEffNe1[NR * NS] = {")
    for r in rx:
        L.append("    " + ", ".join("1" if k in r["eff_ne1"] else "0" for k in range(ns)) + ",")
    L.append("};")
    L.append("")
    L.append("}  // namespace fixed_h2air")
    L.append("}  // namespace janc")
    return "\n".join(L) + "\n"


def generate(path: str = SOURCE, header: str = HEADER) -> bool:
    """Writes the header if its text changed; returns whether it wrote."""
    text = render(path)
    if os.path.exists(header):
        with open(header) as f:
            if f.read() == text:
                return False
    tmp = header + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write(text)
    os.replace(tmp, header)
    return True


if __name__ == "__main__":
    print(render(), end="")
