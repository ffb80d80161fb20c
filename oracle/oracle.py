"""ctypes front end of the CPU FP64 oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. It compiles ``janc_oracle.cpp`` with the
host C++ compiler into ``oracle/_build/liboracle.so`` and exposes plain numpy
wrappers around the C entry points. The arithmetic lives in
``janc_oracle.hpp`` (a step-by-step restatement of arXiv 2504.13750 Sec. 4).

Every function takes a mechanism as the dict produced by
``paper_2504_13750_gb300.inputs.load_mechanism`` (flat numpy arrays only) and a
grid as a dict with keys nx, ny, dx, dy, bc (4 ints: left, right, bottom, top;
0 slip wall, 1 zero-gradient, 2 periodic), weno_eps, newton_tol, newton_maxit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "janc_oracle.cpp"), os.path.join(_HERE, "janc_oracle.hpp")]
_lock = threading.Lock()
_lib = None

BC_WALL, BC_ZEROGRAD, BC_PERIODIC = 0, 1, 2
ST_NONFINITE, ST_NONPOSITIVE, ST_NEWTON_FAIL, ST_SINGULAR = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its sources."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC[0]]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Mech(ctypes.Structure):
    _fields_ = [
        ("ns", ctypes.c_int), ("nr", ctypes.c_int),
        ("M", ctypes.c_void_p), ("nasa", ctypes.c_void_p),
        ("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("Ea", ctypes.c_void_p),
        ("nuf", ctypes.c_void_p), ("nub", ctypes.c_void_p), ("tb", ctypes.c_void_p),
        ("eff", ctypes.c_void_p),
    ]


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("weno_eps", ctypes.c_double), ("newton_tol", ctypes.c_double),
        ("newton_maxit", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            _lib.orc_weno5.restype = d
            _lib.orc_weno5.argtypes = [d, d, d, d, d, d]
            _lib.orc_cfl_dt.restype = d
            _lib.orc_cfl_dt.argtypes = [p, p, p, p, d]
            _lib.orc_set_threads.argtypes = [i]
            _lib.orc_step.argtypes = [p, p, p, p, i, d, d, i, p, p]
            _lib.orc_step_tangent.argtypes = [p, p, p, p, p, p, i, d, i]
            _lib.orc_rhs.argtypes = [p, p, p, p, p, p, p, p]
            _lib.orc_newton.argtypes = [p, p, i, p, p, p]
            _lib.orc_primitives.argtypes = [p, i, p, p, p, p]
            _lib.orc_prim_to_cons.argtypes = [p, i, p, p, p, p, p, p]
            _lib.orc_production_rates.argtypes = [p, d, p, p]
            _lib.orc_source_jacobian.argtypes = [p, p, d, p, p]
            _lib.orc_point_implicit.argtypes = [p, i, p, p, d]
            _lib.orc_lu_solve.argtypes = [i, p, p]
            _lib.orc_thermo.argtypes = [p, i, d, p, p, p]
            _lib.orc_opcount.argtypes = [p, p, i, p, p, d, p]
            _lib.orc_rhs_tangent.argtypes = [p, p, p, p, p, p]
            _lib.orc_trajectory_tangent8.argtypes = [p, p, p, p, p, i, i, d, i, p, p]
            _lib.orc_rhs_ghosted.argtypes = [p, p, p, p, d, d, p]
            _lib.orc_lf_alpha.argtypes = [p, i, p, p, p]
        return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _MechHandle:
    """Keeps the flat arrays alive while the C struct points into them."""

    def __init__(self, mech):
        self.ns = int(mech["ns"])
        self.nr = int(mech["nr"])
        self.arrs = {
            "M": _f64(mech["M"]), "nasa": _f64(mech["nasa"]),
            "A": _f64(mech["A"]), "b": _f64(mech["b"]), "Ea": _f64(mech["Ea"]),
            "nuf": np.ascontiguousarray(mech["nuf"], dtype=np.int32),
            "nub": np.ascontiguousarray(mech["nub"], dtype=np.int32),
            "tb": np.ascontiguousarray(mech["tb"], dtype=np.int32),
            "eff": _f64(mech["eff"]),
        }
        self.s = _Mech(self.ns, self.nr, *[_ptr(self.arrs[k]) for k in
                                          ("M", "nasa", "A", "b", "Ea", "nuf", "nub", "tb", "eff")])

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _grid(g):
    s = _Grid()
    s.nx, s.ny = int(g["nx"]), int(g["ny"])
    s.dx, s.dy = float(g["dx"]), float(g["dy"])
    for k in range(4):
        s.bc[k] = int(g["bc"][k])
    s.weno_eps = float(g.get("weno_eps", 1e-6))
    s.newton_tol = float(g.get("newton_tol", 1e-12))
    s.newton_maxit = int(g.get("newton_maxit", 50))
    return s


def nvar(mech) -> int:
    return 3 + int(mech["ns"])


def set_threads(n: int = 0) -> int:
    return lib().orc_set_threads(int(n))


def thermo(mech, k: int, T: float):
    """(cp/R, h/R, s/R) of species k at T (Eq. 4.3-4.5, per-mole dimensionless)."""
    mh = _MechHandle(mech)
    out = np.zeros(3)
    o = [ctypes.c_double() for _ in range(3)]
    lib().orc_thermo(mh.ref, int(k), float(T), *[ctypes.byref(x) for x in o])
    out[:] = [x.value for x in o]
    return out


def weno5(f, eps=1e-6) -> float:
    return lib().orc_weno5(*[float(x) for x in f], float(eps))


def prim_to_cons(mech, T, p, u, v, Y):
    """Conserved U[nv, ...] from T, p, u, v [...] and Y[ns, ...] (Eq. 4.2)."""
    mh = _MechHandle(mech)
    shape = np.shape(T)
    n = int(np.prod(shape))
    T, p, u, v = (_f64(np.broadcast_to(a, shape)).ravel() for a in (T, p, u, v))
    Y = _f64(np.asarray(Y).reshape(mh.ns, n))
    U = np.zeros((nvar(mech), n))
    lib().orc_prim_to_cons(mh.ref, n, _ptr(T), _ptr(p), _ptr(u), _ptr(v), _ptr(Y), _ptr(U))
    return U.reshape((nvar(mech),) + tuple(shape))


def newton(mech, grid, U, T0):
    mh = _MechHandle(mech)
    U = _f64(U)
    n = U[0].size
    T0 = _f64(T0).ravel()
    T = np.zeros(n)
    st = lib().orc_newton(mh.ref, ctypes.byref(_grid(grid)), n, _ptr(U.reshape(nvar(mech), n)), _ptr(T0), _ptr(T))
    return T.reshape(U.shape[1:]), st


def primitives(mech, U, T):
    """(p, c) per cell."""
    mh = _MechHandle(mech)
    U = _f64(U)
    n = U[0].size
    T = _f64(T).ravel()
    p, c = np.zeros(n), np.zeros(n)
    lib().orc_primitives(mh.ref, n, _ptr(U.reshape(nvar(mech), n)), _ptr(T), _ptr(p), _ptr(c))
    return p.reshape(U.shape[1:]), c.reshape(U.shape[1:])


def production_rates(mech, T, X):
    mh = _MechHandle(mech)
    X = _f64(X)
    w = np.zeros(mh.ns)
    lib().orc_production_rates(mh.ref, float(T), _ptr(X), _ptr(w))
    return w


def source_jacobian(mech, u, T):
    mh = _MechHandle(mech)
    u = _f64(u)
    nsp = mh.ns - 1
    S, J = np.zeros(nsp), np.zeros((nsp, nsp))
    rc = lib().orc_source_jacobian(mh.ref, _ptr(u), float(T), _ptr(S), _ptr(J))
    assert rc == 0
    return S, J


def point_implicit(mech, U, T, dt):
    mh = _MechHandle(mech)
    U = _f64(U).copy()
    n = U[0].size
    T = _f64(T).ravel()
    Uf = U.reshape(nvar(mech), n)
    st = lib().orc_point_implicit(mh.ref, n, _ptr(Uf), _ptr(T), float(dt))
    return Uf.reshape(U.shape), st


def lu_solve(A, b):
    A = _f64(A).copy()
    b = _f64(b).copy()
    st = lib().orc_lu_solve(int(b.size), _ptr(A), _ptr(b))
    return b, st


def rhs(mech, grid, U, T):
    """L(U), x-face fluxes Fx[nv, ny, nx+1], y-face fluxes Gy[nv, ny+1, nx], (alpha_x, alpha_y)."""
    mh = _MechHandle(mech)
    nx, ny, nv = int(grid["nx"]), int(grid["ny"]), nvar(mech)
    U = _f64(U)
    T = _f64(T)
    L = np.zeros((nv, ny, nx))
    Fx = np.zeros((nv, ny, nx + 1))
    Gy = np.zeros((nv, ny + 1, nx))
    al = np.zeros(2)
    lib().orc_rhs(mh.ref, ctypes.byref(_grid(grid)), _ptr(U), _ptr(T), _ptr(L), _ptr(Fx), _ptr(Gy), _ptr(al))
    return L, Fx, Gy, al


def rhs_ghosted(mech, nx, ny, dx, dy, Up, Tp, alpha, weno_eps=1e-6):
    """L(U) of an nx x ny field given with its 3 ghost layers Up[nv, ny+6,
    nx+6], Tp[ny+6, nx+6] (corners ignored) and given LF speeds alpha =
    (alpha_x, alpha_y) of Eq. 4.11."""
    mh = _MechHandle(mech)
    nv = nvar(mech)
    Up, Tp = _f64(Up), _f64(Tp)
    assert Up.shape == (nv, ny + 6, nx + 6) and Tp.shape == (ny + 6, nx + 6)
    g = {"nx": nx, "ny": ny, "dx": dx, "dy": dy, "bc": [0, 0, 0, 0], "weno_eps": weno_eps}
    L = np.zeros((nv, ny, nx))
    lib().orc_rhs_ghosted(mh.ref, ctypes.byref(_grid(g)), _ptr(Up), _ptr(Tp), float(alpha[0]), float(alpha[1]),
                          _ptr(L))
    return L


def lf_alpha(mech, U, T):
    """(alpha_x, alpha_y) of Eq. 4.11: max over the given cells of |u|+c and |v|+c."""
    mh = _MechHandle(mech)
    U = _f64(U)
    n = U[0].size
    a = np.zeros(2)
    lib().orc_lf_alpha(mh.ref, n, _ptr(U.reshape(nvar(mech), n)), _ptr(_f64(T).ravel()), _ptr(a))
    return a


def cfl_dt(mech, grid, U, T, cfl):
    mh = _MechHandle(mech)
    return lib().orc_cfl_dt(mh.ref, ctypes.byref(_grid(grid)), _ptr(_f64(U)), _ptr(_f64(T)), float(cfl))


CHEM_OFF, CHEM_LIE, CHEM_STRANG, CHEM_EXPLICIT = 0, 1, 2, 3


def _chem_mode(chem) -> int:
    """False/True -> off/Lie; or one of CHEM_OFF, CHEM_LIE, CHEM_STRANG, CHEM_EXPLICIT."""
    if isinstance(chem, bool):
        return CHEM_LIE if chem else CHEM_OFF
    mode = int(chem)
    if mode not in (CHEM_OFF, CHEM_LIE, CHEM_STRANG, CHEM_EXPLICIT):
        raise ValueError(f"chemistry mode {chem!r}")
    return mode


def step(mech, grid, U, T, nsteps, dt=0.0, cfl=0.0, chem=True):
    """Advance n steps (chem: False/True or a CHEM_* splitting mode).
    Returns (U, T, status, t, dt_log)."""
    mh = _MechHandle(mech)
    U = _f64(U).copy()
    T = _f64(T).copy()
    t = ctypes.c_double()
    dts = np.zeros(max(int(nsteps), 1))
    st = lib().orc_step(mh.ref, ctypes.byref(_grid(grid)), _ptr(U), _ptr(T), int(nsteps), float(dt), float(cfl),
                        _chem_mode(chem), ctypes.byref(t), _ptr(dts))
    return U, T, st, t.value, dts[:nsteps]


def step_tangent(mech, grid, U, T, dU, dT, nsteps, dt, chem=True):
    """Tangent-linear model: returns (U, T, dU, dT, status) after n fixed-dt steps."""
    mh = _MechHandle(mech)
    U, T, dU, dT = (_f64(a).copy() for a in (U, T, dU, dT))
    st = lib().orc_step_tangent(mh.ref, ctypes.byref(_grid(grid)), _ptr(U), _ptr(T), _ptr(dU), _ptr(dT),
                                int(nsteps), float(dt), _chem_mode(chem))
    return U, T, dU, dT, st


def rhs_tangent(mech, grid, U, T, dU):
    """(dL/dU) dU at (U, T), with the T tangent from a dual Newton solve."""
    mh = _MechHandle(mech)
    U, T, dU = _f64(U), _f64(T), _f64(dU)
    dL = np.zeros_like(U)
    st = lib().orc_rhs_tangent(mh.ref, ctypes.byref(_grid(grid)), _ptr(U), _ptr(T), _ptr(dU), _ptr(dL))
    return dL, st


def trajectory_tangent(mech, grid, U, T, dU0, nsteps, dt, chem=True):
    """Tangents of U^N and of the end-wall pressure loss along up to 8
    directions dU0[l]. Returns (dUN [nl, ...], loss value, dloss [nl], status)."""
    mh = _MechHandle(mech)
    U, T = _f64(U), _f64(T)
    dU0 = _f64(dU0)
    nl = dU0.shape[0]
    dUN = np.zeros_like(dU0)
    loss = np.zeros(1 + nl)
    st = lib().orc_trajectory_tangent8(mh.ref, ctypes.byref(_grid(grid)), _ptr(U), _ptr(T), _ptr(dU0), int(nl),
                                       int(nsteps), float(dt), _chem_mode(chem), _ptr(dUN), _ptr(loss))
    return dUN, loss[0], loss[1:], st


OPS_NAMES = ("add", "mul", "div", "sqrt", "exp", "log")


def opcount(mech, grid, part, U=None, T=None, dt=0.0):
    """Operation counts of the plain algorithm: part 0 = one WENO5 reconstruction,
    1 = rhs over the grid, 2 = Newton over the grid, 3 = chemistry over the grid,
    4 = one full step."""
    mh = _MechHandle(mech)
    if U is None:
        U = np.zeros((nvar(mech), int(grid["ny"]), int(grid["nx"])))
        T = np.zeros((int(grid["ny"]), int(grid["nx"])))
    out = np.zeros(6, dtype=np.int64)
    lib().orc_opcount(mh.ref, ctypes.byref(_grid(grid)), int(part), _ptr(_f64(U)), _ptr(_f64(T)), float(dt),
                      _ptr(out))
    return dict(zip(OPS_NAMES, (int(x) for x in out)))
