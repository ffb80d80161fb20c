"""Ignition-delay sweep (the 0-D constant-volume case of Sec. 5.1(2)) on the
GPU through janc_source_step: every cell of one grid is an independent
reactor at its own initial temperature, 1200-2000 K at 20 atm, dt = 5 ns.
Against the oracle (a 1 x 1 zero-gradient grid per temperature, whose flux
terms vanish) sample by sample, and against an independent stiff
integration (scipy Radau) of the same mechanism."""
import numpy as np
import pytest

import oracle as orc
import ref_exact
from paper_2504_13750_gb300 import inputs

pytestmark = pytest.mark.gpu

H2AIR = inputs.load_mechanism("h2air_synth")
TEMPS = np.array([1200.0, 1300.0, 1400.0, 1600.0, 1800.0, 2000.0])
P0 = 20 * inputs.ATM
DT = 5e-9
EVERY = 20            # samples every 100 ns
T_END = 1.0e-3        # beyond the slowest delay (about 0.84 ms at 1200 K)


@pytest.fixture(scope="module")
def J():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_13750_gb300 import build, janc

    build.build()
    return janc


def _crossing(t, T, level):
    i = int(np.argmax(T >= level))
    assert i > 0
    return t[i - 1] + (level - T[i - 1]) * (t[i] - t[i - 1]) / (T[i] - T[i - 1])


@pytest.fixture(scope="module")
def gpu_sweep(J):
    n = len(TEMPS)
    st = inputs.ignition_cell(H2AIR, T0=1500.0, p0=P0)
    g = J.Grid(H2AIR, n, 1, 1e-3, 1e-3, [1, 1, 1, 1], chemistry=True)
    Y = np.ascontiguousarray(np.repeat(st["Y"], n, axis=2))
    g.set_primitive(TEMPS[None, :].copy(), np.full((1, n), P0), np.zeros((1, n)), np.zeros((1, n)), Y)
    nsamp = int(round(T_END / DT)) // EVERY
    Ts = np.zeros((nsamp + 1, n))
    Ts[0] = TEMPS
    U_first = None
    for k in range(1, nsamp + 1):
        J.janc_source_step(g.handle, EVERY, DT)
        U, T = g.get_state()
        Ts[k] = T[0]
        if k == 10:
            U_first = U.copy()
    assert g.status()["status"] == 0
    g.close()
    return np.arange(nsamp + 1) * EVERY * DT, Ts, U_first


def test_sweep_matches_the_oracle(J, gpu_sweep):
    t, Ts, U_first = gpu_sweep
    threads = orc.set_threads(0)   # the current count (0 only queries)
    orc.set_threads(1)
    try:
        _sweep_vs_oracle(t, Ts, U_first)
    finally:
        orc.set_threads(threads)


def _sweep_vs_oracle(t, Ts, U_first):
    for c, T0 in enumerate(TEMPS):
        st = inputs.ignition_cell(H2AIR, T0=T0, p0=P0)
        U = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
        T = st["T"].copy()
        To = [T0]
        tau_gpu = _crossing(t, Ts[:, c], T0 + 400.0)
        nsamp = min(len(t) - 1, int(np.ceil(1.3 * tau_gpu / (EVERY * DT))))
        for k in range(1, nsamp + 1):
            U, T, s, _, _ = orc.step(H2AIR, st["grid"], U, T, EVERY, dt=DT, chem=True)
            assert s == 0
            To.append(T[0, 0])
            if k == 10:
                ref = U[:, 0, 0]
                got = U_first[:, 0, c]
                assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300 + np.abs(ref).max() * 1e-12)) < 1e-9
        To = np.array(To)
        rel = np.max(np.abs(Ts[: nsamp + 1, c] - To) / To)
        assert rel < 1e-6, (T0, rel)
        tau_orc = _crossing(t[: nsamp + 1], To, T0 + 400.0)
        assert abs(tau_gpu - tau_orc) <= 1e-6 * tau_orc, (T0, tau_gpu, tau_orc)
    # Arrhenius behaviour: the delay falls monotonically with T0
    taus = [_crossing(t, Ts[:, c], T0 + 400.0) for c, T0 in enumerate(TEMPS)]
    assert all(a > b for a, b in zip(taus, taus[1:]))


@pytest.mark.parametrize("T0", [1600.0, 2000.0])
def test_sweep_matches_stiff_integration(J, gpu_sweep, T0):
    t, Ts, _ = gpu_sweep
    c = int(np.where(TEMPS == T0)[0][0])
    tau_gpu = _crossing(t, Ts[:, c], T0 + 400.0)
    st = inputs.ignition_cell(H2AIR, T0=T0, p0=P0)
    U0 = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    t_end = 1.5 * tau_gpu
    tr, Tr, _ = ref_exact.ConstantVolumeReactor(H2AIR).ignition(U0[0, 0, 0], st["Y"][:, 0, 0], T0, t_end,
                                                                np.linspace(0, t_end, 20001))
    tau_ref = _crossing(tr, Tr, T0 + 400.0)
    # first-order splitting error at dt = 5 ns, as for the oracle's own pin
    assert abs(tau_gpu - tau_ref) / tau_ref < 0.01, (T0, tau_gpu, tau_ref)
