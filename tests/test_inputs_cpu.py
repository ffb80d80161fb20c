"""The seeded input recipes (paper_2504_13750_gb300/inputs.py) against the
workloads they stand in for: the detonation tube of Sec. 5.2.1 (premix
H2:O2:N2 = 0.028:0.226:0.746 by mass at 300 K / 1 atm, the left 5 % at
2000 K / 20 atm, slip walls, dx = Lx / nx), its 1 % density perturbation at
fixed p, the Sod problem of Sec. 5.1(1), the adjoint case's N(0, 5 K)
temperature perturbation and the serving stream's distributions. Every
recipe is a pure function of its seed."""
import numpy as np
import pytest

from paper_2504_13750_gb300 import inputs

H2AIR = inputs.load_mechanism("h2air_synth")
GAS = inputs.load_mechanism("ideal_gamma14")


def test_tube_layout():
    nx, ny = 400, 50
    st = inputs.tube(H2AIR, nx, ny)
    g = st["grid"]
    assert g["nx"] == nx and g["ny"] == ny and g["bc"] == [0, 0, 0, 0]
    assert g["dx"] == g["dy"] == pytest.approx(0.05 / nx, rel=1e-15)
    x = (np.arange(nx) + 0.5) * g["dx"]
    ign = x < 0.05 * 0.05
    assert ign.sum() == 20                      # the left 5 % of 400 cells
    assert np.all(st["T"][:, ign] == 2000.0) and np.all(st["p"][:, ign] == 20 * inputs.ATM)
    assert np.all(st["T"][:, ~ign] == 300.0) and np.all(st["p"][:, ~ign] == inputs.ATM)
    assert np.all(st["u"] == 0.0) and np.all(st["v"] == 0.0)
    sp = H2AIR["species"]
    Y = st["Y"][:, 0, 0]
    assert abs(Y.sum() - 1.0) < 1e-15
    for s, w in (("H2", 0.028), ("O2", 0.226), ("N2", 0.746)):
        assert Y[sp.index(s)] == pytest.approx(w, rel=1e-12)
    assert np.all(st["Y"] == Y[:, None, None])


def test_tube_perturbation_is_one_percent_at_fixed_pressure():
    nx, ny = 256, 64
    a = inputs.tube(H2AIR, nx, ny, perturb_seed=0)
    b = inputs.tube(H2AIR, nx, ny, perturb_seed=0)
    c = inputs.tube(H2AIR, nx, ny, perturb_seed=1)
    assert np.array_equal(a["T"], b["T"]) and not np.array_equal(a["T"], c["T"])
    base = inputs.tube(H2AIR, nx, ny)
    np.testing.assert_array_equal(a["p"], base["p"])             # fixed p
    cold = base["T"] == 300.0
    rho_ratio = base["T"][cold] / a["T"][cold]                   # rho ~ 1 / T at fixed p and Y
    assert np.max(np.abs(rho_ratio - 1.0)) == pytest.approx(0.01, rel=2e-2)
    assert np.array_equal(a["T"][~cold], base["T"][~cold])       # the igniter is untouched
    # the perturbation is a sine in y with an integer number m in {2..8} of waves over Ly
    dev = rho_ratio.reshape(ny, -1) - 1.0
    col = dev[:, 0]
    assert np.allclose(dev, col[:, None], rtol=0.0, atol=1e-15)   # uniform along x
    spec = np.abs(np.fft.rfft(col))
    assert 2 <= int(np.argmax(spec)) <= 8


def test_sod_states():
    st = inputs.sod(GAS, 400)
    rho = st["p"][0] / (287.0 * st["T"][0])
    left = st["x"] < 0.0
    assert left.sum() == 200
    np.testing.assert_allclose(rho[left], 1.0, rtol=1e-15)
    np.testing.assert_allclose(rho[~left], 0.125, rtol=1e-15)
    assert np.all(st["p"][0, left] == 1e5) and np.all(st["p"][0, ~left] == 1e4)
    assert st["grid"]["bc"] == [1, 1, 1, 1] and st["grid"]["dx"] == pytest.approx(0.05)


def test_adjoint_case_perturbation():
    st, dT = inputs.adjoint_case(H2AIR)
    assert dT.shape == (64, 512) and st["T"].shape == (64, 512)
    assert abs(dT.mean()) < 0.1 and dT.std() == pytest.approx(5.0, rel=0.02)
    _, dT2 = inputs.adjoint_case(H2AIR)
    assert np.array_equal(dT, dT2)


def test_serving_stream_distributions():
    reqs = inputs.serving_requests(H2AIR, n=2000, seed=1, rate_hz=50.0)
    assert reqs == inputs.serving_requests(H2AIR, n=2000, seed=1, rate_hz=50.0)
    t = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 50.0, rel=0.06)   # Poisson arrivals at 50 Hz
    phi = np.array([r["phi"] for r in reqs])
    p0 = np.array([r["p0"] for r in reqs]) / inputs.ATM
    steps = np.array([r["steps"] for r in reqs])
    assert phi.min() >= 0.5 and phi.max() <= 1.5 and p0.min() >= 0.5 and p0.max() <= 2.0
    assert steps.min() >= 100 and steps.max() <= 1000
    sizes = {(r["nx"], r["ny"]) for r in reqs}
    assert sizes == set(inputs.SERVING_GRIDS)
    # a request's state: H2-air at its phi (O2 : N2 = 1 : 3.76 by moles), p0, igniter at 20 p0
    r = reqs[0]
    st = inputs.request_state(H2AIR, r)
    M = dict(zip(H2AIR["species"], H2AIR["M"]))
    Y = st["Y"][:, 0, 0]
    n = {s: Y[H2AIR["species"].index(s)] / M[s] for s in ("H2", "O2", "N2")}
    assert n["H2"] / n["O2"] == pytest.approx(2 * r["phi"], rel=1e-12)
    assert n["N2"] / n["O2"] == pytest.approx(3.76, rel=1e-12)
    assert st["p"].min() == pytest.approx(r["p0"]) and st["p"].max() == pytest.approx(20 * r["p0"])
