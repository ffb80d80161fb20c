"""Continuous-batching server (janc_server_*): every request's result is the
same alone (janc_step on its own grid) and in a batched mix, bit for bit, under
any admission pattern; admission respects the pool and the slot count; a
served request matches the oracle."""
import numpy as np
import pytest

import mech_variants
import oracle as orc
from paper_2504_13750_gb300 import inputs

pytestmark = pytest.mark.gpu

H2AIR = inputs.load_mechanism("h2air_synth")
# (nx, ny, steps, dy / dx): two requests have dy != dx
SIZES = [(64, 16, 12, 1.0), (96, 24, 7, 1.0), (128, 16, 20, 1.7), (40, 40, 9, 1.0), (256, 32, 15, 1.0),
         (33, 17, 11, 0.6), (70, 9, 5, 1.0)]


@pytest.fixture(scope="module")
def J():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_13750_gb300 import build, janc

    build.build()
    return janc


def _requests():
    rng = np.random.default_rng(11)
    out = []
    for k, (nx, ny, steps, aspect) in enumerate(SIZES):
        req = {"nx": nx, "ny": ny, "phi": float(rng.uniform(0.5, 1.5)), "p0": float(rng.uniform(0.5, 2.0)) * inputs.ATM,
               "steps": steps}
        st = inputs.request_state(H2AIR, req)
        if k % 2 or aspect != 1.0:
            st = inputs.tube(H2AIR, nx, ny, p0=req["p0"], pi=20 * req["p0"], Y=inputs.h2air_Y(H2AIR, req["phi"]),
                             perturb_seed=k, aspect=aspect)
        out.append((req, st))
    return out


def _alone(J, st, steps):
    g = J.Grid.from_grid_dict(H2AIR, st["grid"], chemistry=True)
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    g.step(steps, cfl=0.5)
    U, T = g.get_state()
    g.close()
    return U, T


def _serve(J, reqs, pool_bytes=2 << 30, max_active=64, stagger=0, watch=None, budget=None, mech_dict=None):
    mech = J.Mechanism(H2AIR if mech_dict is None else mech_dict)
    s = J.janc_server_create(mech, chemistry=True, pool_bytes=pool_bytes, max_active=max_active)
    if budget is not None:
        J.janc_server_set_cell_budget(s, *budget)
    ids = []
    pending = list(reqs)
    try:
        while pending or True:
            # submit `stagger` requests per macro-step (all at once when 0)
            take = len(pending) if stagger == 0 else min(stagger, len(pending))
            for req, st in pending[:take]:
                g = st["grid"]
                d = J.make_desc(g["nx"], g["ny"], g["dx"], g["dy"], g["bc"], chemistry=True)
                ids.append(J.janc_server_submit(s, d, st["T"], st["p"], st["u"], st["v"], st["Y"], req["steps"],
                                                cfl=0.5))
            pending = pending[take:]
            info = J.janc_server_run(s, 1)
            if watch is not None:
                watch(info, s, ids)
            if not pending and info["n_active"] == 0 and info["n_queued"] == 0 and info["n_copying"] == 0:
                break
        out = []
        for rid, (req, st) in zip(ids, reqs):
            r = J.janc_server_poll(s, rid)
            assert r["state"] == J.REQ_DONE and r["steps_done"] == req["steps"], r
            U = np.zeros((12, req["ny"], req["nx"]))
            T = np.zeros((req["ny"], req["nx"]))
            J.janc_server_fetch(s, rid, U, T)
            out.append((U, T))
        return out
    finally:
        J.janc_server_destroy(s)


def test_alone_equals_mix_bitwise(J):
    reqs = _requests()
    alone = [_alone(J, st, req["steps"]) for req, st in reqs]
    mixed = _serve(J, reqs)
    for (Ua, Ta), (Um, Tm) in zip(alone, mixed):
        assert np.array_equal(Ua, Um)
        assert np.array_equal(Ta, Tm)


def test_one_slot_and_staggered_arrivals_match(J):
    reqs = _requests()
    one = _serve(J, reqs, max_active=1)
    stag = _serve(J, reqs, stagger=2)
    for (U1, T1), (U2, T2) in zip(one, stag):
        assert np.array_equal(U1, U2) and np.array_equal(T1, T2)


def test_admission_respects_pool(J):
    reqs = _requests()
    mech = J.Mechanism(H2AIR)
    s = J.janc_server_create(mech, chemistry=True, pool_bytes=64 << 20, max_active=8)
    try:
        # footprint of the largest request; a pool of ~2.5 of them
        g = reqs[4][1]["grid"]
        big = J.janc_server_footprint(s, J.make_desc(g["nx"], g["ny"], g["dx"], g["dy"], g["bc"]))
    finally:
        J.janc_server_destroy(s)
    pool = int(2.5 * big) + (1 << 20)
    peak = {"used": 0, "active": 0}

    def watch(info, *_):
        assert info["pool_used"] <= info["pool_bytes"]
        peak["used"] = max(peak["used"], info["pool_used"])
        peak["active"] = max(peak["active"], info["n_active"])

    served = _serve(J, reqs, pool_bytes=pool, watch=watch)
    alone = [_alone(J, st, req["steps"]) for req, st in reqs]
    for (Ua, Ta), (Um, Tm) in zip(alone, served):
        assert np.array_equal(Ua, Um) and np.array_equal(Ta, Tm)
    assert peak["used"] > 0


@pytest.mark.parametrize("max_skip_s", [0.0, 10.0])
def test_cell_budget_bounds_the_active_set(J, max_skip_s):
    """With a cell budget the active set never holds more cells than the cap
    unless one request runs alone, and every result is still the alone one,
    bit for bit."""
    reqs = _requests()
    cap = 9000

    def watch(info, s, ids):
        # ids[k] is the id of reqs[k] (submission order)
        active = [k for k, rid in enumerate(ids) if J.janc_server_poll(s, rid)["state"] == J.REQ_ACTIVE]
        tot = sum(reqs[k][0]["nx"] * reqs[k][0]["ny"] for k in active)
        assert len(active) <= 1 or tot <= cap, (active, tot)

    served = _serve(J, reqs, watch=watch, budget=(cap, max_skip_s))
    alone = [_alone(J, st, req["steps"]) for req, st in reqs]
    for (Ua, Ta), (Um, Tm) in zip(alone, served):
        assert np.array_equal(Ua, Um) and np.array_equal(Ta, Tm)


@pytest.mark.parametrize("k", [0, 2])
def test_served_request_matches_oracle(J, k):
    """Requests 0 (dy = dx) and 2 (dy = 1.7 dx) served alone against the oracle."""
    req, st = _requests()[k]
    assert st["grid"]["dy"] == SIZES[k][3] * st["grid"]["dx"]
    (U, T), = _serve(J, [(req, st)])
    U0 = orc.prim_to_cons(H2AIR, st["T"], st["p"], st["u"], st["v"], st["Y"])
    Uo, To, s, _, _ = orc.step(H2AIR, st["grid"], U0, st["T"], req["steps"], cfl=0.5)
    assert s == 0
    for k in range(U.shape[0]):
        assert np.max(np.abs(U[k] - Uo[k])) <= 1e-10 * np.max(np.abs(Uo[k])) + 1e-300


def test_submit_validation(J):
    mech = J.Mechanism(H2AIR)
    s = J.janc_server_create(mech, chemistry=True, pool_bytes=8 << 20, max_active=2)
    try:
        st = inputs.tube(H2AIR, 512, 64)
        g = st["grid"]
        d = J.make_desc(g["nx"], g["ny"], g["dx"], g["dy"], g["bc"])
        with pytest.raises(J.JancError) as e:  # larger than the whole pool
            J.janc_server_submit(s, d, st["T"], st["p"], st["u"], st["v"], st["Y"], 5, cfl=0.5)
        assert e.value.rc == -4
        small = inputs.tube(H2AIR, 16, 8)
        g = small["grid"]
        d = J.make_desc(g["nx"], g["ny"], g["dx"], g["dy"], g["bc"])
        with pytest.raises(J.JancError):  # both dt and cfl
            J.janc_server_submit(s, d, small["T"], small["p"], small["u"], small["v"], small["Y"], 5, dt=1e-9,
                                 cfl=0.5)
    finally:
        J.janc_server_destroy(s)


def test_run_until_returns_each_request_once(J):
    """janc_server_run_until serves the stream without polling: every request
    is returned exactly once (at most `cap` per call, the rest on later
    calls), and its result is the one it gets alone, bit for bit."""
    reqs = _requests()
    alone = [_alone(J, st, req["steps"]) for req, st in reqs]
    mech = J.Mechanism(H2AIR)
    s = J.janc_server_create(mech, chemistry=True, pool_bytes=2 << 30, max_active=64)
    try:
        ids = []
        for req, st in reqs:
            g = st["grid"]
            d = J.make_desc(g["nx"], g["ny"], g["dx"], g["dy"], g["bc"], chemistry=True)
            ids.append(J.janc_server_submit(s, d, st["T"], st["p"], st["u"], st["v"], st["Y"], req["steps"], cfl=0.5))
        done, info = J.janc_server_run_until(s, max_macro_steps=1, cap=2)
        assert info["macro_steps"] == 1 and done == []  # one macro-step: nothing can have finished
        seen = []
        for _ in range(1000):
            done, info = J.janc_server_run_until(s, cap=2)
            assert len(done) <= 2
            seen += done
            if len(seen) == len(ids):
                break
        assert sorted(seen) == sorted(ids) and len(set(seen)) == len(seen)
        assert J.janc_server_run_until(s, cap=2)[0] == []
        for rid, (req, st), (Ua, Ta) in zip(ids, reqs, alone):
            U = np.zeros((12, req["ny"], req["nx"]))
            T = np.zeros((req["ny"], req["nx"]))
            J.janc_server_fetch(s, rid, U, T)
            assert np.array_equal(U, Ua) and np.array_equal(T, Ta)
    finally:
        J.janc_server_destroy(s)


def test_served_request_with_run_time_table_chemistry(J):
    """A server whose 9-species table has another reaction structure than the
    compiled one (the shipped reactions in reverse order) runs the batched
    run-time-table chemistry kernel: two requests served together, each
    against the oracle on the same table."""
    rev = mech_variants.reordered(H2AIR)
    reqs = [_requests()[k] for k in (0, 2)]
    served = _serve(J, reqs, mech_dict=rev)
    for (req, st), (U, T) in zip(reqs, served):
        U0 = orc.prim_to_cons(rev, st["T"], st["p"], st["u"], st["v"], st["Y"])
        Uo, To, s, _, _ = orc.step(rev, st["grid"], U0, st["T"], req["steps"], cfl=0.5)
        assert s == 0
        for k in range(U.shape[0]):
            assert np.max(np.abs(U[k] - Uo[k])) <= 1e-10 * np.max(np.abs(Uo[k])) + 1e-300
