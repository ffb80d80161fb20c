"""Mechanism variants for tests: the same physics under another reaction
structure, so that grids take the run-time-table chemistry kernels instead of
the ones with the shipped H2-air structure compiled in."""
import numpy as np


def reordered(mech):
    """The mechanism with its reactions in reverse order."""
    m = dict(mech)
    perm = np.arange(mech["nr"])[::-1]
    for k in ("A", "b", "Ea", "nuf", "nub", "tb", "eff"):
        m[k] = np.ascontiguousarray(np.asarray(mech[k])[perm])
    m["equations"] = [mech["equations"][i] for i in perm]
    return m
