"""Thin Python binding of the C ABI in include/janc.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all work runs in libjanc.so. Arrays may be numpy
arrays (host) or CUDA torch tensors (device); the ``where`` argument of the C
call is chosen from the array type. Errors raise ``JancError`` with the
library's message. The library must have been built (``build.build()``); a
missing library is an error, never a silent fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

JANC_HOST, JANC_DEVICE = 0, 1
BC_WALL, BC_ZEROGRAD, BC_PERIODIC = 0, 1, 2
ST_NONFINITE, ST_NONPOSITIVE, ST_NEWTON_FAIL, ST_SINGULAR = 1, 2, 4, 8

_lock = threading.Lock()
_lib = None


class JancError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"janc error {rc}: {msg}")
        self.rc = rc


class janc_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("chemistry", ctypes.c_int), ("weno_eps", ctypes.c_double),
                ("newton_tol", ctypes.c_double), ("newton_maxit", ctypes.c_int)]


class janc_mechanism(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("nr", ctypes.c_int)] + [
        (k, ctypes.c_void_p) for k in ("M", "nasa", "A", "b", "Ea", "nuf", "nub", "tb", "eff")]


class janc_server_info(ctypes.Structure):
    _fields_ = [("n_queued", ctypes.c_int), ("n_active", ctypes.c_int), ("n_copying", ctypes.c_int),
                ("n_done", ctypes.c_int), ("pool_used", ctypes.c_size_t), ("pool_bytes", ctypes.c_size_t),
                ("macro_steps", ctypes.c_longlong)]


class janc_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("steps_done", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("status", ctypes.c_int), ("t", ctypes.c_double), ("dt_last", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double)]


REQ_QUEUED, REQ_ACTIVE, REQ_COPYING, REQ_DONE, REQ_FAILED, REQ_FETCHED = range(6)


class janc_status_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_int), ("t", ctypes.c_double),
                ("dt_last", ctypes.c_double), ("alpha", ctypes.c_double * 2)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libjanc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run paper_2504_13750_gb300.build.build() first")
            L = ctypes.CDLL(path)
            p, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.janc_last_error.restype = ctypes.c_char_p
            L.janc_workspace_bytes.argtypes = [p, p, ctypes.POINTER(ctypes.c_size_t)]
            L.janc_create_grid.argtypes = [p, p, p, ctypes.c_size_t, p, ctypes.POINTER(p)]
            L.janc_set_state.argtypes = [p, p, p, i]
            L.janc_set_state_primitive.argtypes = [p, p, p, p, p, p, i]
            L.janc_step.argtypes = [p, i, d, d, p, p]
            L.janc_get_state.argtypes = [p, p, p, i]
            L.janc_rhs.argtypes = [p, p, p, p, p, i]
            L.janc_status.argtypes = [p, p]
            L.janc_destroy_grid.argtypes = [p]
            L.janc_destroy_grid.restype = None
            L.janc_fp64_peak.argtypes = [p, i, ctypes.POINTER(d)]
            L.janc_selfcheck_rcp.argtypes = [p, i, ctypes.POINTER(ctypes.c_longlong)]
            L.janc_rhs_static.argtypes = [p, p, p, p, p, p, p]
            L.janc_selfcheck_exp.argtypes = [p, i, ctypes.POINTER(ctypes.c_longlong)]
            L.janc_server_create.argtypes = [p, i, ctypes.c_size_t, p, i, p, ctypes.POINTER(p)]
            L.janc_server_footprint.argtypes = [p, p, ctypes.POINTER(ctypes.c_size_t)]
            L.janc_server_submit.argtypes = [p, p, p, p, p, p, p, i, d, d, ctypes.POINTER(i)]
            L.janc_server_run.argtypes = [p, i, p]
            L.janc_server_run_until.argtypes = [p, i, d, p, i, ctypes.POINTER(i), p]
            L.janc_server_poll.argtypes = [p, i, p]
            L.janc_server_fetch.argtypes = [p, i, p, p]
            L.janc_server_set_cell_budget.argtypes = [p, ctypes.c_longlong, d]
            L.janc_server_destroy.argtypes = [p]
            L.janc_server_destroy.restype = None
            L.janc_adjoint_workspace_bytes.argtypes = [p, i, i, ctypes.POINTER(ctypes.c_size_t)]
            L.janc_set_adjoint_mode.argtypes = [p, i]
            L.janc_step_adjoint.argtypes = [p, i, d, i, i, p, p, p, p, ctypes.c_size_t, i]
            L.janc_adjoint_forward.argtypes = [p, i, d, i, i, p, p, ctypes.c_size_t]
            L.janc_adjoint_reverse.argtypes = [p, p, p, i]
            L.janc_rhs_vjp.argtypes = [p, p, p, p, ctypes.c_size_t, i]
            L.janc_primitive_T_vjp.argtypes = [p, p, p, p, p, p, p, p]
            L.janc_profile.argtypes = [p, i]
            L.janc_profile_read.argtypes = [p, p, p]
            L.janc_source_step.argtypes = [p, i, d]
            L.janc_amr_create.argtypes = [p, p, p, p, ctypes.POINTER(p)]
            L.janc_amr_set_state_primitive.argtypes = [p, p, p, p, p, p, i]
            L.janc_amr_step.argtypes = [p, i, d, d, ctypes.POINTER(d)]
            L.janc_amr_layer_blocks.argtypes = [p, i, ctypes.POINTER(i)]
            L.janc_amr_get_layer.argtypes = [p, i, p, p, p]
            L.janc_amr_get_base.argtypes = [p, p, p, i]
            L.janc_amr_status.argtypes = [p, ctypes.POINTER(i)]
            L.janc_amr_cell_updates.argtypes = [p, ctypes.POINTER(ctypes.c_longlong)]
            L.janc_amr_block_lists.argtypes = [p, i, i, p, p, p, p, ctypes.POINTER(i)]
            L.janc_amr_destroy.argtypes = [p]
            L.janc_amr_destroy.restype = None
            sz = ctypes.c_size_t
            L.janc_slab_partition.argtypes = [i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
            L.janc_slab_halo_doubles.argtypes = [p, p, ctypes.POINTER(sz)]
            L.janc_slab_create.argtypes = [p, p, i, i, p, p, sz, p, ctypes.POINTER(p)]
            L.janc_split_create.argtypes = [p, p, i, p, ctypes.POINTER(p)]
            L.janc_split_set_state.argtypes = [p, p, p, i]
            L.janc_split_set_state_primitive.argtypes = [p, p, p, p, p, p, i]
            L.janc_split_step.argtypes = [p, i, d, d, p, p]
            L.janc_split_get_state.argtypes = [p, p, p, i]
            L.janc_split_status.argtypes = [p, p]
            L.janc_split_slab.argtypes = [p, i, ctypes.POINTER(p)]
            L.janc_split_destroy.argtypes = [p]
            L.janc_split_destroy.restype = None
            _lib = L
        return _lib


def _check(rc):
    if rc != 0:
        raise JancError(rc, lib().janc_last_error().decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, writable=False):
    """(pointer, where, keepalive) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, JANC_HOST, None
    if _is_torch(a):
        import torch

        if not a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float64 CUDA tensors")
        return ctypes.c_void_p(a.data_ptr()), JANC_DEVICE, a
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise ValueError("host arrays must be C-contiguous float64 numpy arrays")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return a.ctypes.data_as(ctypes.c_void_p), JANC_HOST, a


def _where(*args):
    ws = {w for (_, w, k) in args if k is not None}
    if len(ws) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ws.pop() if ws else JANC_HOST


CHEM_OFF, CHEM_LIE, CHEM_STRANG, CHEM_EXPLICIT = 0, 1, 2, 3


def chem_mode(chemistry) -> int:
    """False/True -> JANC_CHEM_OFF/JANC_CHEM_LIE, or one of the JANC_CHEM_* values."""
    if isinstance(chemistry, bool):
        return CHEM_LIE if chemistry else CHEM_OFF
    return int(chemistry)


def make_desc(nx, ny, dx, dy, bc, chemistry=True, weno_eps=1e-6, newton_tol=1e-12, newton_maxit=50):
    d = janc_grid_desc()
    d.nx, d.ny, d.dx, d.dy = int(nx), int(ny), float(dx), float(dy)
    for k in range(4):
        d.bc[k] = int(bc[k])
    d.chemistry = chem_mode(chemistry)
    d.weno_eps, d.newton_tol, d.newton_maxit = float(weno_eps), float(newton_tol), int(newton_maxit)
    return d


class Mechanism:
    """ctypes view of a mechanism dict (flat arrays, see inputs.load_mechanism)."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech["ns"]), int(mech["nr"])
        self._a = {
            "M": np.ascontiguousarray(mech["M"], np.float64), "nasa": np.ascontiguousarray(mech["nasa"], np.float64),
            "A": np.ascontiguousarray(mech["A"], np.float64), "b": np.ascontiguousarray(mech["b"], np.float64),
            "Ea": np.ascontiguousarray(mech["Ea"], np.float64),
            "nuf": np.ascontiguousarray(mech["nuf"], np.int32), "nub": np.ascontiguousarray(mech["nub"], np.int32),
            "tb": np.ascontiguousarray(mech["tb"], np.int32), "eff": np.ascontiguousarray(mech["eff"], np.float64),
        }
        self.c = janc_mechanism(self.ns, self.nr, *[self._a[k].ctypes.data_as(ctypes.c_void_p) for k in
                                                    ("M", "nasa", "A", "b", "Ea", "nuf", "nub", "tb", "eff")])


def janc_workspace_bytes(desc, mech: Mechanism) -> int:
    out = ctypes.c_size_t()
    _check(lib().janc_workspace_bytes(ctypes.byref(desc), ctypes.byref(mech.c), ctypes.byref(out)))
    return out.value


def janc_create_grid(desc, mech: Mechanism, workspace_ptr=None, workspace_bytes=0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().janc_create_grid(ctypes.byref(desc), ctypes.byref(mech.c),
                                  ctypes.c_void_p(workspace_ptr) if workspace_ptr else None,
                                  int(workspace_bytes), ctypes.c_void_p(stream) if stream else None,
                                  ctypes.byref(h)))
    return h


def janc_set_state(g, U, T0=None):
    a, b = _arg(U), _arg(T0)
    _check(lib().janc_set_state(g, a[0], b[0], _where(a, b)))


def janc_set_state_primitive(g, T, p, u, v, Y):
    args = [_arg(x) for x in (T, p, u, v, Y)]
    _check(lib().janc_set_state_primitive(g, *[x[0] for x in args], _where(*args)))


def janc_step(g, n_steps, dt=0.0, cfl=0.0, want_time=False):
    """Returns (t, dt_last) when want_time (synchronises), else None."""
    if want_time:
        t, dl = ctypes.c_double(), ctypes.c_double()
        _check(lib().janc_step(g, int(n_steps), float(dt), float(cfl), ctypes.byref(t), ctypes.byref(dl)))
        return t.value, dl.value
    _check(lib().janc_step(g, int(n_steps), float(dt), float(cfl), None, None))
    return None


def janc_source_step(g, n_steps, dt):
    _check(lib().janc_source_step(g, int(n_steps), float(dt)))


def janc_get_state(g, U=None, T=None, check=True):
    a, b = _arg(U, True), _arg(T, True)
    rc = lib().janc_get_state(g, a[0], b[0], _where(a, b))
    if check:
        _check(rc)
    return rc


def janc_rhs(g, Fx=None, Gy=None, L=None, alpha=None):
    args = [_arg(x, True) for x in (Fx, Gy, L, alpha)]
    _check(lib().janc_rhs(g, *[x[0] for x in args], _where(*args)))


def janc_status(g):
    s = janc_status_info()
    _check(lib().janc_status(g, ctypes.byref(s)))
    return {"status": s.status, "steps_done": s.steps_done, "t": s.t, "dt_last": s.dt_last,
            "alpha": (s.alpha[0], s.alpha[1])}


def _rhs_static_shapes(desc, ns, U, T, L, alpha, device):
    """Refuses, before the C call, buffers that do not match the grid (the
    kernels would read or write past their ends) or that sit on another
    device than `device` (the current one, whose scratch the call uses)."""
    cells = int(desc.nx) * int(desc.ny)
    want = {"U": (U, (ns + 3) * cells), "T": (T, cells), "L": (L, (ns + 3) * cells)}
    for name, (t, n) in want.items():
        if t is None or t.numel() != n:
            raise ValueError(f"janc_rhs_static: {name} must hold {n} elements for a {desc.nx} x {desc.ny} grid")
    if alpha is not None and alpha.numel() < 2:
        raise ValueError("janc_rhs_static: alpha must hold 2 elements")
    if any(t is not None and t.device.index != device for t in (U, T, L, alpha)):
        raise ValueError(f"janc_rhs_static: every tensor must be on the current device (cuda:{device})")


def janc_rhs_static(desc, mech: Mechanism, U, T, L, alpha=None, stream=None):
    """Right-hand side with no device allocation (see include/janc.h): for
    callers that cannot allocate, e.g. inside another framework's memory pool.
    U, T, L (and alpha) must be CUDA tensors the caller owns, on the current
    device (the one whose copy of the static scratch array the call uses):
    U and L of (ns + 3) nx ny elements, T of nx ny, alpha of at least 2."""
    args = [_arg(x, True) for x in (U, T, L, alpha)]
    if any(a[2] is not None and a[1] != JANC_DEVICE for a in args):
        raise ValueError("janc_rhs_static takes device tensors only")
    import torch

    _rhs_static_shapes(desc, mech.ns, U, T, L, alpha, torch.cuda.current_device())
    _check(lib().janc_rhs_static(ctypes.byref(desc), ctypes.byref(mech.c), args[0][0], args[1][0], args[2][0],
                                 args[3][0], ctypes.c_void_p(stream) if stream else None))


LOSS_ENDWALL_P, LOSS_SEEDED = 0, 1
ADJ_RECOMPUTE, ADJ_STORE_FACES = 0, 1


def janc_set_adjoint_mode(g, mode):
    """ADJ_RECOMPUTE (default) or ADJ_STORE_FACES (face derivatives kept in
    the segment stores); read by the next workspace query and forward."""
    _check(lib().janc_set_adjoint_mode(g, int(mode)))


def janc_adjoint_workspace_bytes(g, n_steps, ckpt_every) -> int:
    out = ctypes.c_size_t()
    _check(lib().janc_adjoint_workspace_bytes(g, int(n_steps), int(ckpt_every), ctypes.byref(out)))
    return out.value


def janc_adjoint_forward(g, n_steps, dt, ckpt_every, loss_kind=LOSS_SEEDED, workspace_ptr=None, workspace_bytes=0):
    """Checkpointed forward of n_steps; U^N stays in the grid. Returns the
    end-wall loss for LOSS_ENDWALL_P, else 0."""
    loss = ctypes.c_double()
    _check(lib().janc_adjoint_forward(g, int(n_steps), float(dt), int(ckpt_every), int(loss_kind), ctypes.byref(loss),
                                      ctypes.c_void_p(workspace_ptr) if workspace_ptr else None, int(workspace_bytes)))
    return loss.value


def janc_adjoint_reverse(g, seed, dL_dU0):
    """dL/dU^0 into dL_dU0 for the cotangent seed = dL/dU^N (None: zero)."""
    a, b = _arg(seed), _arg(dL_dU0, True)
    _check(lib().janc_adjoint_reverse(g, a[0], b[0], _where(a, b)))


def janc_step_adjoint(g, n_steps, dt, ckpt_every, loss_kind=LOSS_ENDWALL_P, seed=None, dL_dU0=None,
                      workspace_ptr=None, workspace_bytes=0):
    """Returns the loss; fills dL_dU0 (numpy or CUDA tensor) when given."""
    a, b = _arg(seed), _arg(dL_dU0, True)
    loss = ctypes.c_double()
    _check(lib().janc_step_adjoint(g, int(n_steps), float(dt), int(ckpt_every), int(loss_kind), a[0], b[0],
                                   ctypes.byref(loss), ctypes.c_void_p(workspace_ptr) if workspace_ptr else None,
                                   int(workspace_bytes), _where(a, b)))
    return loss.value


def janc_rhs_vjp(g, mu, nu, workspace_ptr=None, workspace_bytes=0):
    a, b = _arg(mu), _arg(nu, True)
    _check(lib().janc_rhs_vjp(g, a[0], b[0], ctypes.c_void_p(workspace_ptr) if workspace_ptr else None,
                              int(workspace_bytes), _where(a, b)))


def janc_primitive_T_vjp(g, T, p, u, v, Y, dL_dU, dL_dT):
    args = [_arg(x, True) for x in (T, p, u, v, Y, dL_dU, dL_dT)]
    if any(x[2] is not None and x[1] != JANC_DEVICE for x in args):
        raise ValueError("janc_primitive_T_vjp takes device tensors")
    _check(lib().janc_primitive_T_vjp(g, *[x[0] for x in args]))


def janc_profile(g, enable=True):
    _check(lib().janc_profile(g, int(bool(enable))))


KERNEL_CLASSES = ("face_flux", "rk_update", "chemistry")


def janc_profile_read(g):
    """{class: (ms, launches)} since the last read (synchronises)."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_longlong * 3)()
    _check(lib().janc_profile_read(g, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p)))
    return {KERNEL_CLASSES[c]: (ms[c], n[c]) for c in range(3)}


def janc_last_error() -> str:
    return lib().janc_last_error().decode()


def janc_destroy_grid(g):
    lib().janc_destroy_grid(g)


def janc_fp64_peak(stream=None, n_iter=4000) -> float:
    out = ctypes.c_double()
    _check(lib().janc_fp64_peak(ctypes.c_void_p(stream) if stream else None, int(n_iter), ctypes.byref(out)))
    return out.value


def janc_selfcheck_rcp(x) -> int:
    x = np.ascontiguousarray(x, np.float64)
    out = ctypes.c_longlong()
    _check(lib().janc_selfcheck_rcp(x.ctypes.data_as(ctypes.c_void_p), int(x.size), ctypes.byref(out)))
    return out.value


def janc_server_set_cell_budget(s, cells, max_skip_s=0.0):
    _check(lib().janc_server_set_cell_budget(s, int(cells), float(max_skip_s)))


def janc_server_create(mech: Mechanism, chemistry=True, pool_bytes=1 << 30, pool_ptr=None, max_active=64,
                       stream=None):
    h = ctypes.c_void_p()
    _check(lib().janc_server_create(ctypes.byref(mech.c), chem_mode(chemistry), int(pool_bytes),
                                    ctypes.c_void_p(pool_ptr) if pool_ptr else None, int(max_active),
                                    ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
    return h


def janc_server_footprint(s, desc) -> int:
    out = ctypes.c_size_t()
    _check(lib().janc_server_footprint(s, ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def janc_server_submit(s, desc, T, p, u, v, Y, n_steps, dt=0.0, cfl=0.0) -> int:
    arrs = [_arg(np.ascontiguousarray(x, np.float64)) for x in (T, p, u, v, Y)]
    if any(a[1] != JANC_HOST for a in arrs):
        raise ValueError("janc_server_submit takes host arrays")
    rid = ctypes.c_int()
    _check(lib().janc_server_submit(s, ctypes.byref(desc), *[a[0] for a in arrs], int(n_steps), float(dt),
                                    float(cfl), ctypes.byref(rid)))
    return rid.value


def janc_server_run(s, macro_steps=1) -> dict:
    info = janc_server_info()
    _check(lib().janc_server_run(s, int(macro_steps), ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in janc_server_info._fields_}


def janc_server_run_until(s, max_macro_steps=1 << 30, max_wall_s=1e9, cap=256):
    """(ids of newly finished requests, info dict): see include/janc.h."""
    ids = np.zeros(max(int(cap), 1), dtype=np.int32)
    n = ctypes.c_int()
    info = janc_server_info()
    _check(lib().janc_server_run_until(s, int(max_macro_steps), float(max_wall_s),
                                       ids.ctypes.data_as(ctypes.c_void_p), int(cap), ctypes.byref(n),
                                       ctypes.byref(info)))
    return [int(x) for x in ids[:n.value]], {k: getattr(info, k) for k, _ in janc_server_info._fields_}


def janc_server_poll(s, rid) -> dict:
    ri = janc_request_info()
    _check(lib().janc_server_poll(s, int(rid), ctypes.byref(ri)))
    return {k: getattr(ri, k) for k, _ in janc_request_info._fields_}


def janc_server_fetch(s, rid, U=None, T=None, check=True) -> int:
    a, b = _arg(U, True), _arg(T, True)
    rc = lib().janc_server_fetch(s, int(rid), a[0], b[0])
    if check:
        _check(rc)
    return rc


def janc_server_destroy(s):
    lib().janc_server_destroy(s)


def janc_selfcheck_exp(x) -> int:
    x = np.ascontiguousarray(x, np.float64)
    out = ctypes.c_longlong()
    _check(lib().janc_selfcheck_exp(x.ctypes.data_as(ctypes.c_void_p), int(x.size), ctypes.byref(out)))
    return out.value


class Grid:
    """Convenience owner of one grid: a torch workspace on the current CUDA
    device and stream, and the C handle. Arrays go in and out as numpy (host)
    or CUDA torch tensors (device)."""

    def __init__(self, mech: dict, nx, ny, dx, dy, bc, chemistry=True, stream=None, **kw):
        import torch

        self.mech = Mechanism(mech)
        self.ns = self.mech.ns
        self.nv = self.ns + 3
        self.nx, self.ny = int(nx), int(ny)
        self.desc = make_desc(nx, ny, dx, dy, bc, chemistry=chemistry, **kw)
        nbytes = janc_workspace_bytes(self.desc, self.mech)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.handle = janc_create_grid(self.desc, self.mech, aligned, nbytes, self.stream.cuda_stream)

    @classmethod
    def from_grid_dict(cls, mech, g, chemistry=True, **kw):
        return cls(mech, g["nx"], g["ny"], g["dx"], g["dy"], g["bc"], chemistry=chemistry,
                   weno_eps=g.get("weno_eps", 1e-6), newton_tol=g.get("newton_tol", 1e-12),
                   newton_maxit=g.get("newton_maxit", 50), **kw)

    def set_state(self, U, T0=None):
        janc_set_state(self.handle, U, T0)

    def set_primitive(self, T, p, u, v, Y):
        janc_set_state_primitive(self.handle, T, p, u, v, Y)

    def step(self, n, dt=0.0, cfl=0.0, want_time=False):
        return janc_step(self.handle, n, dt=dt, cfl=cfl, want_time=want_time)

    def get_state(self, check=True):
        U = np.zeros((self.nv, self.ny, self.nx))
        T = np.zeros((self.ny, self.nx))
        janc_get_state(self.handle, U, T, check=check)
        return U, T

    def rhs(self):
        Fx = np.zeros((self.nv, self.ny, self.nx + 1))
        Gy = np.zeros((self.nv, self.ny + 1, self.nx))
        L = np.zeros((self.nv, self.ny, self.nx))
        al = np.zeros(2)
        janc_rhs(self.handle, Fx, Gy, L, al)
        return L, Fx, Gy, al

    def status(self):
        return janc_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            janc_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- x-slab decomposition ------------------------------------------------------------------

# int (*)(void* user, void* cuda_stream): the exchange callback of a stand-alone slab.
JANC_EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class janc_slab_exchange(ctypes.Structure):
    _fields_ = [("send_lo", ctypes.c_void_p), ("send_hi", ctypes.c_void_p), ("recv_lo", ctypes.c_void_p),
                ("recv_hi", ctypes.c_void_p), ("alpha2", ctypes.c_void_p), ("fn", JANC_EXCHANGE_FN),
                ("user", ctypes.c_void_p)]


def janc_slab_partition(nx, n_slabs, k):
    """(x0, nx_local) of slab k of n_slabs over nx columns."""
    x0, w = ctypes.c_int(), ctypes.c_int()
    _check(lib().janc_slab_partition(int(nx), int(n_slabs), int(k), ctypes.byref(x0), ctypes.byref(w)))
    return x0.value, w.value


def janc_slab_halo_doubles(desc, mech: Mechanism) -> int:
    out = ctypes.c_size_t()
    _check(lib().janc_slab_halo_doubles(ctypes.byref(desc), ctypes.byref(mech.c), ctypes.byref(out)))
    return out.value


def janc_slab_create(desc, mech: Mechanism, x0, nx_local, xch: janc_slab_exchange, workspace_ptr=None,
                     workspace_bytes=0, stream=None):
    """A slab grid handle (use it with janc_set_state, janc_step, ...). `xch`
    and the callback it holds must stay alive until janc_destroy_grid."""
    h = ctypes.c_void_p()
    _check(lib().janc_slab_create(ctypes.byref(desc), ctypes.byref(mech.c), int(x0), int(nx_local), ctypes.byref(xch),
                                  ctypes.c_void_p(workspace_ptr) if workspace_ptr else None, int(workspace_bytes),
                                  ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
    return h


def janc_split_create(desc, mech: Mechanism, n_slabs, stream=None):
    h = ctypes.c_void_p()
    _check(lib().janc_split_create(ctypes.byref(desc), ctypes.byref(mech.c), int(n_slabs),
                                   ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
    return h


def janc_split_set_state(s, U, T0=None):
    a, b = _arg(U), _arg(T0)
    _check(lib().janc_split_set_state(s, a[0], b[0], _where(a, b)))


def janc_split_set_state_primitive(s, T, p, u, v, Y):
    args = [_arg(x) for x in (T, p, u, v, Y)]
    _check(lib().janc_split_set_state_primitive(s, *[x[0] for x in args], _where(*args)))


def janc_split_step(s, n_steps, dt=0.0, cfl=0.0, want_time=False):
    """Returns (t, dt_last) when want_time (synchronises), else None."""
    if want_time:
        t, dl = ctypes.c_double(), ctypes.c_double()
        _check(lib().janc_split_step(s, int(n_steps), float(dt), float(cfl), ctypes.byref(t), ctypes.byref(dl)))
        return t.value, dl.value
    _check(lib().janc_split_step(s, int(n_steps), float(dt), float(cfl), None, None))
    return None


def janc_split_get_state(s, U=None, T=None, check=True):
    a, b = _arg(U, True), _arg(T, True)
    rc = lib().janc_split_get_state(s, a[0], b[0], _where(a, b))
    if check:
        _check(rc)
    return rc


def janc_split_status(s):
    st = janc_status_info()
    _check(lib().janc_split_status(s, ctypes.byref(st)))
    return {"status": st.status, "steps_done": st.steps_done, "t": st.t, "dt_last": st.dt_last,
            "alpha": (st.alpha[0], st.alpha[1])}


def janc_split_slab(s, k):
    h = ctypes.c_void_p()
    _check(lib().janc_split_slab(s, int(k), ctypes.byref(h)))
    return h


def janc_split_destroy(s):
    lib().janc_split_destroy(s)


class Split:
    """Owner of a single-process x-slab split of one domain (janc_split_*) on
    the current CUDA device and stream; whole-domain arrays in and out."""

    def __init__(self, mech: dict, nx, ny, dx, dy, bc, n_slabs, chemistry=True, stream=None, **kw):
        import torch

        self.mech = Mechanism(mech)
        self.ns = self.mech.ns
        self.nv = self.ns + 3
        self.nx, self.ny, self.n_slabs = int(nx), int(ny), int(n_slabs)
        self.desc = make_desc(nx, ny, dx, dy, bc, chemistry=chemistry, **kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = janc_split_create(self.desc, self.mech, n_slabs, self.stream.cuda_stream)

    @classmethod
    def from_grid_dict(cls, mech, g, n_slabs, chemistry=True, **kw):
        return cls(mech, g["nx"], g["ny"], g["dx"], g["dy"], g["bc"], n_slabs, chemistry=chemistry,
                   weno_eps=g.get("weno_eps", 1e-6), newton_tol=g.get("newton_tol", 1e-12),
                   newton_maxit=g.get("newton_maxit", 50), **kw)

    def columns(self):
        return [janc_slab_partition(self.nx, self.n_slabs, k) for k in range(self.n_slabs)]

    def set_state(self, U, T0=None):
        janc_split_set_state(self.handle, U, T0)

    def set_primitive(self, T, p, u, v, Y):
        janc_split_set_state_primitive(self.handle, T, p, u, v, Y)

    def step(self, n, dt=0.0, cfl=0.0, want_time=False):
        return janc_split_step(self.handle, n, dt=dt, cfl=cfl, want_time=want_time)

    def get_state(self, check=True):
        U = np.zeros((self.nv, self.ny, self.nx))
        T = np.zeros((self.ny, self.nx))
        janc_split_get_state(self.handle, U, T, check=check)
        return U, T

    def status(self):
        return janc_split_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            janc_split_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- block-structured AMR ------------------------------------------------------------------


class AmrDesc(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("block", ctypes.c_int), ("threshold", ctypes.c_double),
                ("n_buffer", ctypes.c_int), ("regrid_every", ctypes.c_int), ("synchronous", ctypes.c_int)]


def janc_amr_create(desc, mech: Mechanism, amr: AmrDesc, stream=None):
    h = ctypes.c_void_p()
    _check(lib().janc_amr_create(ctypes.byref(desc), ctypes.byref(mech.c), ctypes.byref(amr),
                                 ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
    return h


def janc_amr_set_state_primitive(a, T, p, u, v, Y):
    args = [_arg(x) for x in (T, p, u, v, Y)]
    _check(lib().janc_amr_set_state_primitive(a, *[x[0] for x in args], _where(*args)))


def janc_amr_step(a, n_steps, dt=0.0, cfl=0.0):
    """Advances n base steps; returns the simulated time advanced."""
    t = ctypes.c_double()
    _check(lib().janc_amr_step(a, int(n_steps), float(dt), float(cfl), ctypes.byref(t)))
    return t.value


def janc_amr_block_lists(flags, bc):
    """(pos [nblk, 2], map [nby, nbx], nbr [nblk, 4]) of the device block-list
    builder for the refinement flags [nby, nbx] (see include/janc.h)."""
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    nby, nbx = f.shape
    b = np.ascontiguousarray(bc, dtype=np.int32)
    pos = np.zeros(2 * nbx * nby, dtype=np.int32)
    mp = np.zeros(nbx * nby, dtype=np.int32)
    nbr = np.zeros(4 * nbx * nby, dtype=np.int32)
    n = ctypes.c_int()
    _check(lib().janc_amr_block_lists(f.ctypes.data_as(ctypes.c_void_p), nbx, nby, b.ctypes.data_as(ctypes.c_void_p),
                                      pos.ctypes.data_as(ctypes.c_void_p), mp.ctypes.data_as(ctypes.c_void_p),
                                      nbr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    k = n.value
    return pos[:2 * k].reshape(k, 2), mp.reshape(nby, nbx), nbr[:4 * k].reshape(k, 4)


def janc_amr_layer_blocks(a, level):
    n = ctypes.c_int()
    _check(lib().janc_amr_layer_blocks(a, int(level), ctypes.byref(n)))
    return n.value


def janc_amr_get_layer(a, level, nv):
    """(pos [nblk, 2] as (bx, by), U [nblk, nv, 16, 16], T [nblk, 16, 16]) on the host."""
    nb = janc_amr_layer_blocks(a, level)
    pos = np.zeros((nb, 2), dtype=np.int32)
    U = np.zeros((nb, nv, 16, 16))
    T = np.zeros((nb, 16, 16))
    _check(lib().janc_amr_get_layer(a, int(level), pos.ctypes.data_as(ctypes.c_void_p),
                                    U.ctypes.data_as(ctypes.c_void_p), T.ctypes.data_as(ctypes.c_void_p)))
    return pos, U, T


def janc_amr_get_base(a, U, T):
    ua, ta = _arg(U, True), _arg(T, True)
    _check(lib().janc_amr_get_base(a, ua[0], ta[0], _where(ua, ta)))


def janc_amr_status(a):
    s = ctypes.c_int()
    _check(lib().janc_amr_status(a, ctypes.byref(s)))
    return s.value


def janc_amr_cell_updates(a):
    n = ctypes.c_longlong()
    _check(lib().janc_amr_cell_updates(a, ctypes.byref(n)))
    return n.value


def janc_amr_destroy(a):
    lib().janc_amr_destroy(a)


class Amr:
    """Owner of one AMR hierarchy (janc_amr_*) on the current CUDA stream."""

    def __init__(self, mech: dict, grid: dict, chemistry=True, levels=2, threshold=1e6, n_buffer=2,
                 regrid_every=10, stream=None, synchronous=False):
        import torch

        self.mech = Mechanism(mech)
        self.nv = self.mech.ns + 3
        self.nx, self.ny = int(grid["nx"]), int(grid["ny"])
        self.levels = int(levels)
        self.desc = make_desc(grid["nx"], grid["ny"], grid["dx"], grid["dy"], grid["bc"], chemistry=chemistry,
                              weno_eps=grid.get("weno_eps", 1e-6), newton_tol=grid.get("newton_tol", 1e-12),
                              newton_maxit=grid.get("newton_maxit", 50))
        self.amr = AmrDesc(int(levels), 16, float(threshold), int(n_buffer), int(regrid_every), int(bool(synchronous)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = janc_amr_create(self.desc, self.mech, self.amr, self.stream.cuda_stream)

    def set_primitive(self, T, p, u, v, Y):
        janc_amr_set_state_primitive(self.handle, T, p, u, v, Y)

    def step(self, n=1, dt=0.0, cfl=0.0):
        return janc_amr_step(self.handle, n, dt=dt, cfl=cfl)

    def base(self):
        U = np.zeros((self.nv, self.ny, self.nx))
        T = np.zeros((self.ny, self.nx))
        janc_amr_get_base(self.handle, U, T)
        return U, T

    def layer(self, level):
        return janc_amr_get_layer(self.handle, level, self.nv)

    def status(self):
        return janc_amr_status(self.handle)

    def cell_updates(self):
        return janc_amr_cell_updates(self.handle)

    def close(self):
        if self.handle:
            janc_amr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
