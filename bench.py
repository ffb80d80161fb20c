"""Benchmark: FP64 cell-steps/s of the reacting-flow step on a 4096 x 512
H2-air detonation tube (2.1 M cells, 9 species / 19 reactions, slip walls,
CFL 0.5, seeded 1 % density perturbation), one JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one advance_one_step (CFL dt, 3 LF-split WENO5 RK stages with
Newton T recovery, point-implicit chemistry) over the whole grid. By default
each rank runs its own replica of the tube (the solve is independent per GPU:
weak scaling, no data-path collective); `value` is the sum over ranks of
cells x steps / the max over ranks of the device-timed region. With --split
the ranks share one tube as x-slabs (Sec. 4.4: halo exchange and LF-speed
max through NCCL after every state-producing phase; strong scaling); `value`
is the tube's cells x steps / the max over ranks of the timed region.

`--impl reference` times the CPU FP64 oracle (the plain restatement of the
method used by the tests) on the host cores on a slab of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 512
CFL = 0.5


def workload_name():
    return f"h2air_detonation_tube_{NX}x{NY}_9sp19r_cfl0.5"


METRIC = "FP64 cell-steps/s per GB300"
UNIT = "cell-steps/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def tube_state():
    from paper_2504_13750_gb300 import inputs

    mech = inputs.load_mechanism("h2air_synth")
    st = inputs.tube(mech, NX, NY, perturb_seed=0)
    return mech, st


# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def weno_flops():
    """Algorithmic flops of one textbook WENO5 reconstruction, as counted by
    the oracle's operation-counting scalar (stored by oracle/count_ops.py)."""
    with open(os.path.join(ROOT, "tests", "golden", "oracle_opcounts.json")) as f:
        return json.load(f)["weno5"]["flops"]


def chem_flops_per_cell(mech):
    """Algorithmic FP64 flops of one point-implicit chemistry update of one
    cell (Eq. 4.6-4.13) followed by the Newton T recovery (Eq. 4.2-4.4), in
    the plain analytic form of the method, counted from the mechanism's
    structure: a fused multiply-add is 2 flops, and exp, log, reciprocal and
    square root 1 each (so the count is a lower bound of the work). It is
    the method's count, not the kernel's instruction count nor the oracle's
    (whose Jacobian comes from dual numbers).

    Terms: concentrations and their sum; per species the Gibbs polynomial of
    Eq. 4.9 and exp(G), 1/exp(G); per reaction k_f (Eq. 4.8), k_b through
    K_eq (products of exp(G) and P_ref/RT), the mass-action products, the
    third-body sum (Eq. 4.7), the rate of progress, the production rates and
    the analytic Jacobian entries (participants x carried rows, the closure
    column of the last species, the third-body rows); A = I - dt J and dt w;
    the 8 x 8 LU with partial pivoting and the two triangular solves; the
    update; Newton with the mixture-sum form of the thermodynamics (two
    iterations, as the tube's cells take) and p, c."""
    ns = int(mech["ns"])
    nsp = ns - 1
    f = 0
    f += 2 * nsp + 1 + (ns - 1)             # X_k, X_ns, C_tot
    f += 2                                  # ln T, 1/T
    f += ns * (2 * 6 + 2)                   # G_k (6 FMA), exp, reciprocal
    f += 2                                  # P_ref/(Ru T), its inverse
    for i in range(int(mech["nr"])):
        nuf, nub = mech["nuf"][i], mech["nub"][i]
        re = [(k, int(nuf[k])) for k in range(ns) if nuf[k]]
        pr = [(k, int(nub[k])) for k in range(ns) if nub[k]]
        dnu = sum(n for _, n in pr) - sum(n for _, n in re)
        f += 2 * 2 + 1                      # ln k_f = lnA + b ln T - Ea/(Ru T); exp
        f += sum(n for _, n in re) + sum(n for _, n in pr) + abs(dnu)   # k_b
        f += sum(n for _, n in re) + sum(n for _, n in pr)              # mass action
        tb = int(mech["tb"][i])
        neff = sum(1 for k in range(ns) if tb and mech["eff"][i][k] != 1.0)
        f += 2 * neff                       # third-body sum
        f += 2                              # net, q
        rows = [k for k, _ in re + pr if k < nsp]
        f += 2 * len(rows)                  # production rates
        for side in (re, pr):               # d q / d X_j of every participant
            for _, n in side:
                f += (1 if n > 1 else 0) + sum(m for _, m in side) - 1 + 1
        for k in rows:                      # Jacobian rows
            for j, _ in re + pr:
                f += 2 if j < nsp else 1 + 2 * nsp
            if tb:
                f += 1 + 2 * nsp
    f += 2 * nsp * nsp + nsp                # A = I - dt J, b = dt w
    for c in range(nsp):                    # LU with partial pivoting
        f += 1 + (nsp - 1 - c) * (1 + 2 * (nsp - 1 - c) + 2)
    f += sum(2 * (nsp - 1 - r) + 1 for r in range(nsp))   # back substitution
    f += 2 * nsp                            # rho Y_k += M_k x_k
    f += 1 + 2 * nsp + 6 * (1 + 2 * nsp)    # Newton: 1/rho, W and the enthalpy sums
    f += 8                                  # kinetic energy, rho e / Ru, constants
    f += 2 * (2 * 5 + 2 * 4 + 1 + 1 + 1)    # two iterations: F, F', dT = -F/F', T += dT
    f += 2 * 4 + 1 + 1 + 4 + 1              # C_v, C_p, p, c (with the square root)
    return f


# ----------------------------------------------------------------------------
def cpu_baseline_oracle(mech, st, steps=5):
    """The oracle as it stands on the host cores: `steps` full steps of the
    4096 x 512 tube (about 10 s on 16 cores), plus one step of a 4096 x 32
    slab on one thread. Returns (cell-steps/s, cores, sample text, single-
    thread cell-steps/s)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as orc

    orc.build()
    cores = orc.set_threads(0)
    U = orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])
    t0 = time.perf_counter()
    orc.step(mech, st["grid"], U, st["T"], steps, cfl=CFL)
    dt = time.perf_counter() - t0
    rows = 32
    g1 = dict(st["grid"], ny=rows)
    orc.set_threads(1)
    t1 = time.perf_counter()
    orc.step(mech, g1, np.ascontiguousarray(U[:, :rows]), np.ascontiguousarray(st["T"][:rows]), 1, cfl=CFL)
    d1 = time.perf_counter() - t1
    orc.set_threads(cores)
    return (NX * NY * steps / dt, cores, f"{steps} full steps of the {NX}x{NY} tube ({dt:.1f} s)",
            NX * rows / d1)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as orc
    from paper_2504_13750_gb300 import inputs

    orc.build()
    mech = inputs.load_mechanism("h2air_synth")
    # each step: one oracle step on an nx x 32 slab of the same tube (the
    # bottom rows, slip walls), so the whole run stays within minutes
    rows = 32
    st = inputs.tube(mech, NX, rows, perturb_seed=0)
    cores = orc.set_threads(0)
    U = orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])
    T = st["T"].copy()
    for _ in range(args.warmup):
        U, T, _, _, _ = orc.step(mech, st["grid"], U, T, 1, cfl=CFL)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, T, _, _, _ = orc.step(mech, st["grid"], U, T, 1, cfl=CFL)
    el = time.perf_counter() - t0
    value = NX * rows * args.steps / el
    sample = f"one oracle step of a {NX}x{rows} slab of the tube per step ({args.steps} timed, {args.warmup} warm-up)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "nx": NX, "ny": NY, "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
def serve_stream(janc, mech_c, reqs, states, arrivals, max_active, pool_bytes, stream, cell_budget=0, max_skip_s=0.0):
    """Replays the request stream in real time through one server: a request
    is submitted once its arrival time has passed. Between arrivals the
    server runs on its own (janc_server_run_until: macro-steps until a
    request finishes or the next arrival is due) and returns the ids of the
    requests that finished; nothing polls the others. Returns per-request
    latencies (completion - arrival, s) and the makespan."""
    s = janc.janc_server_create(mech_c, chemistry=True, pool_bytes=pool_bytes, max_active=max_active,
                                stream=stream.cuda_stream)
    if cell_budget:
        janc.janc_server_set_cell_budget(s, cell_budget, max_skip_s)
    try:
        n = len(reqs)
        index = {}
        done_t = [None] * n
        nxt = 0
        t0 = time.perf_counter()
        finished = 0
        idle = True
        while finished < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                st, rq = states[nxt], reqs[nxt]
                g = st["grid"]
                d = janc.make_desc(g["nx"], g["ny"], g["dx"], g["dy"], g["bc"], chemistry=True)
                index[janc.janc_server_submit(s, d, st["T"], st["p"], st["u"], st["v"], st["Y"], rq["steps"],
                                              cfl=CFL)] = nxt
                nxt += 1
                idle = False
            if idle and nxt < n:  # nothing submitted and unfinished: wait for the next arrival
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
                continue
            budget = arrivals[nxt] - (time.perf_counter() - t0) if nxt < n else 1e9
            ids, info = janc.janc_server_run_until(s, max_wall_s=max(budget, 0.0), cap=n)
            now = time.perf_counter() - t0
            for rid in ids:
                k = index[rid]
                r = janc.janc_server_poll(s, rid)
                if r["state"] == janc.REQ_FAILED or r["status"] != 0:
                    raise RuntimeError(f"request {k} failed with status {r['status']}")
                done_t[k] = now
                finished += 1
                janc.janc_server_fetch(s, rid)
            idle = info["n_active"] == 0 and info["n_queued"] == 0 and info["n_copying"] == 0
        lat = [done_t[k] - arrivals[k] for k in range(n)]
        return lat, max(done_t) - arrivals[0]
    finally:
        janc.janc_server_destroy(s)


SERVE_BUDGET_CELLS = 600_000   # just above the largest request (2048 x 256)
SERVE_MAX_SKIP_S = 1.0


def run_serving(janc, stream, n_req, steps_range, seed=1, grids="all"):
    """Serving leg: solves of mixed size and mixture arriving as a Poisson
    stream at 1.5x the one-at-a-time capacity, served by the batched server
    (active set capped at 600k cells, later requests may pass a blocked one
    for 1 s) and by a one-slot server running the same kernels. The closed-
    system capacity of the uncapped batched server is reported beside."""
    from paper_2504_13750_gb300 import inputs

    mech = inputs.load_mechanism("h2air_synth")
    mech_c = janc.Mechanism(mech)
    sizes = inputs.SERVING_GRIDS if grids == "all" else inputs.SERVING_GRIDS[:2]
    reqs = inputs.serving_requests(mech, n=n_req, seed=seed, steps_range=steps_range, grids=sizes)
    states = [inputs.request_state(mech, r) for r in reqs]
    cell_steps = [r["nx"] * r["ny"] * r["steps"] for r in reqs]
    pool = 16 << 30
    zero = [0.0] * n_req
    budget = dict(cell_budget=SERVE_BUDGET_CELLS, max_skip_s=SERVE_MAX_SKIP_S)
    # closed system (everything queued at t = 0): the capacity of each mode
    _, span_seq = serve_stream(janc, mech_c, reqs, states, zero, 1, pool, stream)
    _, span_bat = serve_stream(janc, mech_c, reqs, states, zero, 256, pool, stream, **budget)
    _, span_ps = serve_stream(janc, mech_c, reqs, states, zero, 256, pool, stream)
    cap_seq = n_req / span_seq
    # open system: Poisson arrivals at 1.5x the one-at-a-time capacity
    rate = 1.5 * cap_seq
    rng = np.random.default_rng(seed + 100)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    arrivals = list(arrivals - arrivals[0])
    out = {"requests": n_req, "steps_range": list(steps_range), "grids": [list(g) for g in sizes],
           "cell_steps": int(sum(cell_steps)),
           "capacity_solves_per_s": {"batched": n_req / span_bat, "one_at_a_time": cap_seq,
                                     "batched_uncapped": n_req / span_ps},
           "capacity_cell_steps_per_s": {"batched": sum(cell_steps) / span_bat,
                                         "one_at_a_time": sum(cell_steps) / span_seq},
           "offered_rate_per_s": rate, "offered_load_vs_one_at_a_time": 1.5,
           "batched_policy": {"max_active": 256, "cell_budget": SERVE_BUDGET_CELLS, "max_skip_s": SERVE_MAX_SKIP_S}}
    for name, slots, kw in (("batched", 256, budget), ("one_at_a_time", 1, {})):
        lat, span = serve_stream(janc, mech_c, reqs, states, arrivals, slots, pool, stream, **kw)
        out[name] = {"solves_per_s": n_req / span, "cell_steps_per_s": sum(cell_steps) / span,
                     "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                     "mean_latency_s": float(np.mean(lat)), "makespan_s": span, "max_active": slots}
    out["batched_vs_one_at_a_time_solves"] = out["batched"]["solves_per_s"] / out["one_at_a_time"]["solves_per_s"]
    out["batched_vs_one_at_a_time_capacity"] = span_seq / span_bat
    return out


def run_adjoint(janc, stream, nsteps=500, ckpt=50):
    """Adjoint leg: 512 x 64 tube with a seeded per-cell initial T
    perturbation, gradient of the time-integrated end-wall pressure through
    janc_step_adjoint (forward with checkpoints, segment recompute, reverse
    sweep) against the plain forward (janc_step) over the same fixed-dt
    trajectory. Timed at the stated checkpoint interval and with the whole
    trajectory kept in HBM (interval = n steps: nothing recomputed)."""
    import torch
    from paper_2504_13750_gb300 import inputs

    mech = inputs.load_mechanism("h2air_synth")
    st, dT0 = inputs.adjoint_case(mech)
    g = janc.Grid.from_grid_dict(mech, st["grid"], chemistry=True, stream=stream)
    Y = np.ascontiguousarray(st["Y"])
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], Y)
    _, dt = g.step(1, cfl=0.5, want_time=True)
    T0 = np.ascontiguousarray(st["T"] + dT0)
    gU0 = torch.empty((g.nv, g.ny, g.nx), dtype=torch.float64, device="cuda")

    def timed(fn):
        g.set_primitive(T0, st["p"], st["u"], st["v"], Y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    g.set_primitive(T0, st["p"], st["u"], st["v"], Y)
    g.step(5, dt=dt)  # warm-up
    _, t_fwd = timed(lambda: g.step(nsteps, dt=dt))
    res = {}
    for mode in (janc.ADJ_RECOMPUTE, janc.ADJ_STORE_FACES):
        janc.janc_set_adjoint_mode(g.handle, mode)
        for ck in (ckpt, nsteps):
            nbytes = janc.janc_adjoint_workspace_bytes(g.handle, nsteps, ck)
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            wp = (ws.data_ptr() + 255) & ~255
            g.set_primitive(T0, st["p"], st["u"], st["v"], Y)
            janc.janc_step_adjoint(g.handle, 5, dt, ck, janc.LOSS_ENDWALL_P, None, gU0, wp, nbytes)  # warm-up
            loss_f, _ = timed(lambda: janc.janc_step_adjoint(g.handle, nsteps, dt, ck, janc.LOSS_ENDWALL_P, None,
                                                              None, wp, nbytes))
            loss_a, t_adj = timed(lambda: janc.janc_step_adjoint(g.handle, nsteps, dt, ck, janc.LOSS_ENDWALL_P, None,
                                                                  gU0, wp, nbytes))
            res[mode, ck] = {"ckpt_every": ck, "adjoint_s": t_adj, "adjoint_over_forward": t_adj / t_fwd,
                             "workspace_bytes": nbytes, "loss": loss_a, "loss_forward_only": loss_f}
            del ws
            torch.cuda.empty_cache()
    g.close()
    # the headline: the faster mode at the stated checkpoint interval
    best = min((janc.ADJ_RECOMPUTE, janc.ADJ_STORE_FACES), key=lambda m: res[m, ckpt]["adjoint_s"])
    names = {janc.ADJ_RECOMPUTE: "recompute", janc.ADJ_STORE_FACES: "store_faces"}
    head = res[best, ckpt]
    return {"workload": f"h2air_tube_{st['grid']['nx']}x{st['grid']['ny']}_{nsteps}steps_ckpt{ckpt}",
            "mode": names[best], "loss": head["loss"], "loss_forward_only": head["loss_forward_only"],
            "forward_s": t_fwd, "adjoint_s": head["adjoint_s"], "adjoint_over_forward": head["adjoint_over_forward"],
            "workspace_bytes": head["workspace_bytes"], "dt": dt,
            "store_all": res[best, nsteps],
            "modes": {names[m]: {"ckpt": res[m, ckpt], "store_all": res[m, nsteps]} for m in names},
            "note": "forward_s is janc_step over the trajectory; adjoint_s covers the forward with checkpoints, the "
                    "recompute of every segment but the last two and the reverse sweep; store_all keeps the whole "
                    "trajectory in HBM (one segment, nothing recomputed). Modes: recompute rebuilds the WENO5 "
                    "derivatives in the reverse face pass; store_faces keeps them from the forward / recompute "
                    "(JANC_ADJ_STORE_FACES); the headline is the faster mode at the stated interval",
            "accuracy_target": "partial: <= 1e-6 against the oracle's tangent and central differences where the "
                               "derivative is well conditioned (the 100-step lane ahead of the igniter, a smooth "
                               "reacting case); the 500-step gradient is not comparable at 1e-6 by any "
                               "implementation: the exact derivative moves 34 % under a 1e-10 K shift of T0 at "
                               "200 steps while the loss moves 3e-13 (tests/test_oracle_conditioning.py)"}


def _amr_timed(janc, stream, mech, st, levels, every, sync, warm, steps):
    import torch

    thr = 50.0 / st["grid"]["dx"]
    a = janc.Amr(mech, st["grid"], chemistry=True, levels=levels, threshold=thr, n_buffer=4, regrid_every=every,
                 stream=stream, synchronous=sync)
    a.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    a.step(warm, cfl=0.5)
    torch.cuda.synchronize()
    updates, t_sim = 0, 0.0
    t0 = time.perf_counter()
    # chunks of one regrid period: the layers (and so the updates per step)
    # only change at a regrid, which opens each chunk; one host read per chunk
    done = 0
    while done < steps:  # the warm-up is a multiple of `every`, so every chunk opens with a regrid
        k = min(every, steps - done)
        t_sim += a.step(k, cfl=0.5)
        updates += a.cell_updates() * k
        done += k
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    status = a.status()
    blocks = [janc.janc_amr_layer_blocks(a.handle, i) for i in range(1, levels + 1)]
    a.close()
    if status != 0:
        raise RuntimeError(f"AMR status word {status:#x}")
    return wall, t_sim, updates, blocks


def run_amr(janc, stream, levels=3, warm=20, steps=40, every=10):
    """AMR leg: 2048 x 256 H2-air tube base, `levels` layers of 16 x 16
    blocks refined where |grad T| > 50 K per base cell (buffer 4), CFL 0.5 on
    the base. Crossover advance (Fig. 2a): `warm` base steps, then `steps`
    timed (a multiple of `every`), regrid every `every` base steps.
    Synchronous advance (Fig. 2b) over the same simulated span: 2^levels
    times as many steps, each of the deepest layer's dt. Both are timed by
    wall clock, regrids included, and compared per simulated time.
    Cell updates count base cells plus the cells of layer i, 2^i times
    (crossover) or once (synchronous)."""
    from paper_2504_13750_gb300 import inputs

    mech = inputs.load_mechanism("h2air_synth")
    st = inputs.tube(mech, 2048, 256, perturb_seed=0)
    r = 2 ** levels
    wall, t_sim, updates, blocks = _amr_timed(janc, stream, mech, st, levels, every, False, warm, steps)
    ws, ts, us, bs = _amr_timed(janc, stream, mech, st, levels, every * r, True, warm * r, steps * r)
    nx0, ny0 = st["grid"]["nx"], st["grid"]["ny"]
    uniform = nx0 * ny0 * 8 ** levels  # finest-resolution cells x 2^levels substeps per base step
    return {"workload": f"h2air_tube_base{nx0}x{ny0}_{levels}layers_16x16blocks_grad50K_regrid{every}",
            "base_steps_timed": steps, "warmup_base_steps": warm, "ms_per_base_step": 1e3 * wall / steps,
            "cell_updates_per_s": updates / wall, "cell_updates_per_base_step": updates / steps,
            "blocks_per_layer_at_end": blocks, "uniform_finest_updates_per_base_step": uniform,
            "fraction_of_uniform_finest": updates / steps / uniform,
            "synchronous": {"steps_timed": steps * r, "ms_per_step": 1e3 * ws / (steps * r),
                            "cell_updates_per_s": us / ws, "blocks_per_layer_at_end": bs,
                            "wall_s_per_simulated_us": ws / (ts * 1e6)},
            "crossover_wall_s_per_simulated_us": wall / (t_sim * 1e6),
            "crossover_vs_synchronous_wall_per_sim_time": (wall / t_sim) / (ws / ts),
            "note": "wall clock, regrids included (device-built block lists; one 4-byte count per layer and regrid "
                    "and one clock read per regrid period reach the host); paper (A100): crossover 0.10 s vs "
                    "synchronous 0.18 s per base dt (-44 %)"}


def run_inverse(janc, iters=15):
    """Inverse-problem leg (the synthetic form of Sec. 6.2): 1000 x 400
    periodic channel, one-step global reaction as an explicit source, loss of
    Eq. 6.6 after 100 fixed-dt steps; Adam iterations per second, each one a
    forward of 100 steps with the whole trajectory and its face derivatives
    kept on the device, the reverse sweep over them and the two state set-ups
    of dU_0/dtheta."""
    from paper_2504_13750_gb300 import inverse

    import torch

    t0 = time.perf_counter()
    P = inverse.ChannelInverse(nx=1000, ny=400, n_steps=100, dev_steps=400, store_faces=True)
    setup = time.perf_counter() - t0
    P.loss_and_grad(0.8)  # warm-up
    hist, wall = P.optimize(0.8, iters=iters, lr=0.01)
    nbytes = P.nbytes
    P.close()
    del P
    torch.cuda.empty_cache()
    return {"workload": "channel_1000x400_global_h2o2_g129_explicit_100steps_adam_lr0.01",
            "iterations": iters, "iterations_per_s": iters / wall, "setup_s": setup,
            "theta_start": hist[0][0], "theta_end": hist[-1][0], "loss_start": hist[0][1], "loss_end": hist[-1][1],
            "adjoint_mode": "store_faces", "workspace_bytes": nbytes,
            "note": "paper (A100, JAX): 1.20 iterations/s on its 1000 x 400 RDC case with 100 steps per iteration"}


def reduce_max(pg, x, device="cuda"):
    """Max over ranks of a per-rank scalar (the slowest rank's time); x
    itself when there is no process group."""
    if pg is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, seconds):
    """Units processed by all ranks (weak scaling: every rank runs its own
    replica) per second of the slowest rank."""
    return world * units_per_rank / seconds


def run_split_leg(janc, stream, n_slabs=4, steps=10, warm=3):
    """The tube cut into n_slabs x-slabs on one GPU (janc_split_*, Sec. 4.4):
    the rate over `steps` CFL steps, for comparison with the undivided grid's
    (the exchange's cost: one pack launch per slab and state-producing phase,
    and the smaller launches of each slab)."""
    import torch

    mech, st = tube_state()
    s = janc.Split(mech, NX, NY, st["grid"]["dx"], st["grid"]["dy"], st["grid"]["bc"], n_slabs, chemistry=True,
                   stream=stream)
    s.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    s.step(warm, cfl=CFL)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps, cfl=CFL)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st_ = s.status()
    cols = s.columns()
    s.close()
    if st_["status"] != 0:
        raise RuntimeError(f"split: device status {st_['status']:#x}")
    return {"workload": workload_name(), "slabs": n_slabs, "columns": cols, "steps": steps,
            "value": NX * NY * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps}


def tube_totals(mech, U):
    """Host totals of a tube state for the conservation record: mass, energy
    and the moles of each element (from the species' element counts)."""
    ns = int(mech["ns"])
    rhoY = np.concatenate([U[4:4 + ns - 1], (U[0] - U[4:4 + ns - 1].sum(axis=0))[None]], axis=0)
    moles = rhoY.reshape(ns, -1).sum(axis=1) / np.asarray(mech["M"])
    el = mech["elements"]
    names = sorted({e for sp in mech["species"] for e in el[sp]})
    E = np.array([[el[sp].get(e, 0) for sp in mech["species"]] for e in names], dtype=float)
    out = {"mass": float(U[0].sum()), "energy": float(U[3].sum())}
    out.update({f"element_{e}": float(v) for e, v in zip(names, E @ moles)})
    return out


def run_config2_full(janc, stream, steps=2000):
    """The 4096 x 512 tube for its full horizon (cellular detonation): one
    janc_step call of `steps` CFL steps, timed with CUDA events; the status
    word afterwards, the minimum rho, p, T of the final state, and the drift
    of mass, energy and element totals (slip walls conserve them to roundoff)."""
    import torch

    mech, st = tube_state()
    g = janc.Grid(mech, NX, NY, st["grid"]["dx"], st["grid"]["dy"], st["grid"]["bc"], chemistry=True, stream=stream)
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    U0, _ = g.get_state()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps, cfl=CFL)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stt = g.status()
    U1, T1 = g.get_state(check=False)
    g.close()
    a, b = tube_totals(mech, U0), tube_totals(mech, U1)
    nv = U1.shape[0]
    rho = U1[0]
    # p = Ru T sum_k rho Y_k / M_k (Eq. 4.2), for the record of the final state
    M = np.asarray(mech["M"])
    rhoY = np.concatenate([U1[4:nv], (rho - U1[4:nv].sum(axis=0))[None]], axis=0)
    p = float(np.min(8.314472 * (rhoY / M[:, None, None]).sum(axis=0) * T1))
    return {"workload": workload_name(), "steps": steps, "value": NX * NY * steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / steps, "t_sim_s": stt["t"], "status": stt["status"],
            "min_rho": float(rho.min()), "min_T": float(T1.min()), "max_T": float(T1.max()), "min_p": p,
            "relative_drift": {k: (b[k] - a[k]) / abs(a[k]) for k in a}}


def run_config1(janc, stream, with_cpu=True):
    """The 256 x 32 tube of config 1, all 200 steps at CFL 0.5: on the GPU
    (one janc_step call, CUDA events) and, on rank 0, through the oracle on
    the host cores (the whole run)."""
    import torch
    from paper_2504_13750_gb300 import inputs

    mech = inputs.load_mechanism("h2air_synth")
    st = inputs.tube(mech, 256, 32)
    g = janc.Grid(mech, 256, 32, st["grid"]["dx"], st["grid"]["dy"], st["grid"]["bc"], chemistry=True, stream=stream)
    Y = np.ascontiguousarray(st["Y"])
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], Y)
    g.step(5, cfl=CFL)
    g.set_primitive(st["T"], st["p"], st["u"], st["v"], Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(200, cfl=CFL)
    e1.record(stream)
    torch.cuda.synchronize()
    gpu_s = e0.elapsed_time(e1) * 1e-3
    g.close()
    out = {"workload": "h2air_detonation_tube_256x32_200steps_cfl0.5", "gpu_cell_steps_per_s": 256 * 32 * 200 / gpu_s}
    if with_cpu:
        sys.path.insert(0, os.path.join(ROOT, "oracle"))
        import oracle as orc

        cores = orc.set_threads(0)
        U = orc.prim_to_cons(mech, st["T"], st["p"], st["u"], st["v"], st["Y"])
        t0 = time.perf_counter()
        orc.step(mech, st["grid"], U, st["T"], 200, cfl=CFL)
        cpu_s = time.perf_counter() - t0
        out.update({"cpu_cell_steps_per_s": 256 * 32 * 200 / cpu_s, "cpu_cores": cores, "cpu_s": cpu_s})
    return out


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2504_13750_gb300 import build, janc

    build.build()
    mech, st = tube_state()
    # CPU baseline first (rank 0, N = 1 only), before the GPU is busy
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, v1 = cpu_baseline_oracle(mech, st)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": v1, "unit": UNIT, "sample": f"1 step of a {NX}x32 slab on 1 thread"}}

    stream = torch.cuda.Stream()
    if args.split:
        # this rank's x-slab of the one tube; halos and alpha through NCCL
        from paper_2504_13750_gb300 import slab

        comm = slab.TorchExchange(rank, world, periodic=False)
        g = slab.Slab(mech, st["grid"], rank, world, comm, chemistry=True, stream=stream)
        x0, nxl = g.columns()
        cut = lambda a: np.ascontiguousarray(a[..., x0:x0 + nxl])  # noqa: E731
        g.set_primitive(cut(st["T"]), cut(st["p"]), cut(st["u"]), cut(st["v"]), cut(st["Y"]))
    else:
        nxl = NX
        g = janc.Grid(mech, NX, NY, st["grid"]["dx"], st["grid"]["dy"], st["grid"]["bc"], chemistry=True,
                      stream=stream)
        g.set_primitive(st["T"], st["p"], st["u"], st["v"], np.ascontiguousarray(st["Y"]))
    g.step(args.warmup, cfl=CFL)
    torch.cuda.synchronize()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if world == 1 else str(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as clk:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        janc.janc_profile(g.handle, True)
        ev0.record(stream)
        g.step(args.steps, cfl=CFL)
        ev1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    janc.janc_profile(g.handle, False)
    ms = ev0.elapsed_time(ev1)
    prof = janc.janc_profile_read(g.handle)
    stt = g.status()
    if stt["status"] != 0:
        raise RuntimeError(f"device status {stt['status']:#x} after the timed region")
    ms = reduce_max(pg, ms)
    cells = nxl * NY  # this rank's cells
    # replicas: every rank's tube counts; split: the ranks share one tube
    value = (NX * NY * args.steps / (ms * 1e-3) if args.split
             else whole_job_rate(world, cells * args.steps, ms * 1e-3))

    # ---- end to end through the C ABI with pinned host buffers ----
    nv = g.nv
    e2e = None
    if not args.no_e2e:
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()  # noqa: E731
        Uh, Th = pin((nv, NY, nxl)), pin((NY, nxl))
        janc.janc_get_state(g.handle, Uh, Th)
        e2e_steps = max(5, args.steps // 2)
        nb = int(Uh.nbytes + Th.nbytes)
        if args.split:
            # one slab per rank, its jobs in sequence: load, one step, read back
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                g.set_state(Uh, Th)
                g.step(1, cfl=CFL)
                janc.janc_get_state(g.handle, Uh, Th)
            e2e_s = reduce_max(pg, time.perf_counter() - t0)
            e2e = {"value": NX * NY * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nb,
                   "d2h_bytes_per_step": nb, "steps": e2e_steps, "pipeline": "none"}
        else:
            # Independent jobs through the C ABI: each loads the host state
            # (pinned), runs one CFL step and reads its result back. Two grids
            # on two streams take alternate jobs, so one job's copies run
            # beside the other's step (set_state / get_state return once their
            # own stream's copies are done). Each step waits for the previous
            # job's step, so the steps themselves run one at a time, as in the
            # device-timed figure.
            e2e_steps = max(20, args.steps)
            g2 = janc.Grid(mech, NX, NY, st["grid"]["dx"], st["grid"]["dy"], st["grid"]["bc"], chemistry=True,
                           stream=torch.cuda.Stream())
            gs = (g, g2)
            evs = (torch.cuda.Event(), torch.cuda.Event())
            Uo, To = (pin((nv, NY, nxl)), pin((nv, NY, nxl))), (pin((NY, nxl)), pin((NY, nxl)))
            for q in range(2):  # warm-up job on each grid, into each output buffer
                gs[q].set_state(Uh, Th)
                gs[q].step(1, cfl=CFL)
                janc.janc_get_state(gs[q].handle, Uo[q], To[q])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gs[0].set_state(Uh, Th)
            gs[0].step(1, cfl=CFL)
            evs[0].record(gs[0].stream)
            for k in range(e2e_steps):
                c, x = k % 2, (k + 1) % 2
                if k + 1 < e2e_steps:
                    gs[x].set_state(Uh, Th)
                    gs[x].stream.wait_event(evs[c])
                    gs[x].step(1, cfl=CFL)
                    evs[x].record(gs[x].stream)
                janc.janc_get_state(gs[c].handle, Uo[c], To[c])
            e2e_s = reduce_max(pg, time.perf_counter() - t0)
            for q in gs:
                stq = q.status()
                if stq["status"] != 0:
                    raise RuntimeError(f"device status {stq['status']:#x} in the end-to-end jobs")
            if not np.array_equal(Uo[0], Uo[1]):
                raise RuntimeError("end-to-end jobs on the two grids disagree")
            g2.close()
            e2e = {"value": whole_job_rate(world, cells * e2e_steps, e2e_s), "unit": UNIT,
                   "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "steps": e2e_steps,
                   "ms_per_step": e2e_s / e2e_steps * 1e3,
                   "pipeline": "two grids on two streams: one job's host copies beside the other's step; "
                               "the steps one at a time"}

    # ---- roofline of the dominant kernel (face fluxes: FP64-pipe bound) ----
    ff_ms, ff_n = prof["face_flux"]
    faces = (nxl + 1) * NY + nxl * (NY + 1)
    flops_launch = nv * faces * (2 * weno_flops() + 1)
    achieved = flops_launch / (ff_ms / ff_n * 1e-3) / 1e12
    peaks = measured_peaks()
    fp64_nominal = 1.25  # TFLOP/s, GB300 FP64 (recipe's nominal figure)
    dfma = janc.janc_fp64_peak(stream.cuda_stream, 4000)
    fp64_measured = 2.0 * dfma / 1e12
    total_prof = sum(v[0] for v in prof.values())
    # DRAM bytes per face from one ncu capture of this kernel (2048 x 512 tube,
    # 12 variables: 248.1 MB read + 172.7 MB written over 2,099,712 faces),
    # scaled to this launch by its face count.
    traffic = 420.771e6 / 2099712 * faces if nv == 12 else None
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_nominal, "unit": "TFLOP/s",
            "frac": achieved / fp64_nominal, "traffic": traffic, "kernel": "k_face_flux",
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz)",
            "peak_measured_dfma_tflops": fp64_measured, "frac_of_measured_dfma": achieved / fp64_measured,
            "flops_per_launch": flops_launch, "avg_launch_ms": ff_ms / ff_n}
    # HBM view of the same kernel, beside the FP64 view
    bytes_launch = 8 * (nv + 2) * cells + 8 * nv * faces  # state + u/v/p planes read, face fluxes written
    hbm = peaks.get("hbm_gbs", 6800.0)
    roof_hbm = {"achieved_gbs": bytes_launch / (ff_ms / ff_n * 1e-3) / 1e9, "peak_gbs": hbm,
                "frac": bytes_launch / (ff_ms / ff_n * 1e-3) / 1e9 / hbm, "bytes_per_launch": bytes_launch}
    kernels = {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / total_prof if total_prof else None}
               for k, v in prof.items()}
    # chemistry: FP64 ALU bound; algorithmic flops of the method per cell
    ch_ms, ch_n = prof["chemistry"]
    chem_fpc = chem_flops_per_cell(mech)
    chem_ach = chem_fpc * cells / (ch_ms / ch_n * 1e-3) / 1e12
    roof_chem = {"bound": "alu", "achieved": chem_ach, "peak": fp64_nominal, "unit": "TFLOP/s",
                 "frac": chem_ach / fp64_nominal, "kernel": "k_chem", "flops_per_cell": chem_fpc,
                 "flops_count": "plain analytic form of Eq. 4.6-4.13 and Newton T from the mechanism's structure; "
                                "FMA = 2 flops, exp/log/reciprocal/sqrt = 1",
                 "avg_launch_ms": ch_ms / ch_n, "frac_of_measured_dfma": chem_ach / fp64_measured,
                 "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if args.split else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "nx": NX, "ny": NY, "cells": cells, "species": 9, "reactions": 19,
                   "cfl": CFL, "parallelism": f"x-slab x{world}" if args.split else f"replicas x{world}",
                   "l2": f"inputs larger than L2 (129 MB): each state buffer is 16 planes x {cells} cells = {16 * 8 * cells / 1e6:.0f} MB"},
        "e2e": e2e,
        "roofline": roof,
        "roofline_hbm": roof_hbm,
        "roofline_chem": roof_chem,
        "kernels": kernels,
        "gpu_launches": int(sum(v[1] for v in prof.values())),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "t_sim_s": stt["t"],
    }
    g.close()
    if not args.no_adjoint:
        line["adjoint"] = run_adjoint(janc, stream)
    if rank == 0:
        line["config1"] = run_config1(janc, stream, with_cpu=world == 1 and not args.no_cpu_baseline)
    if rank == 0 and world == 1 and not args.no_split:
        sp = run_split_leg(janc, stream)
        sp["vs_undivided"] = sp["value"] / value
        line["split"] = sp
    if rank == 0 and not args.no_amr:
        line["amr"] = run_amr(janc, stream)
    if rank == 0 and not args.no_inverse:
        line["inverse"] = run_inverse(janc)
    if not args.no_serving:
        line["serving"] = run_serving(janc, stream, args.serving_requests, tuple(args.serving_steps))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_only(args):
    import torch
    from paper_2504_13750_gb300 import build, janc

    build.build()
    stream = torch.cuda.Stream()
    if args.only == "adjoint":
        n = args.leg_steps or 500
        out = run_adjoint(janc, stream, nsteps=n, ckpt=max(1, n // 10))
    elif args.only == "inverse":
        out = run_inverse(janc, iters=args.leg_steps or 15)
    elif args.only == "serving":
        out = run_serving(janc, stream, args.serving_requests, tuple(args.serving_steps), grids=args.serving_grids)
    elif args.only == "split":
        out = run_split_leg(janc, stream, steps=args.leg_steps or 10)
    elif args.only == "config2":
        out = run_config2_full(janc, stream, steps=args.leg_steps or 2000)
    else:
        out = run_amr(janc, stream, steps=args.leg_steps or 40)
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-amr", action="store_true")
    ap.add_argument("--no-inverse", action="store_true")
    ap.add_argument("--no-split", action="store_true", help="skip the 4-slab split leg (N = 1)")
    ap.add_argument("--split", action="store_true",
                    help="ranks share one tube as x-slabs (strong scaling) instead of running replicas")
    ap.add_argument("--serving-requests", type=int, default=64,
                    help="requests in the serving leg (the full stream is 256 with --serving-steps 100 1000)")
    ap.add_argument("--serving-steps", type=int, nargs=2, default=(50, 150))
    ap.add_argument("--nx", type=int, default=NX, help="tube cells along x (default: the 4096 x 512 workload)")
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--serving-grids", choices=("all", "small"), default="all",
                    help="request grids: all five sizes, or only 128x16 and 256x32")
    ap.add_argument("--only", choices=("adjoint", "amr", "inverse", "serving", "split", "config2"), default=None,
                    help="run one side leg alone and print its JSON object (for profiling)")
    ap.add_argument("--leg-steps", type=int, default=None,
                    help="with --only: adjoint trajectory steps (checkpoint every steps/10) or timed AMR base steps")
    args = ap.parse_args()
    globals()["NX"], globals()["NY"] = args.nx, args.ny
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
