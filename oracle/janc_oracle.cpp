// C entry points of the CPU oracle (TEST INFRASTRUCTURE ONLY: loaded by the
// tests, the smoke check and the benchmark's CPU-baseline leg through ctypes).
// Every function forwards to the step-by-step restatement in janc_oracle.hpp.
#include "janc_oracle.hpp"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {
thread_local OpCount g_ops;
}

using namespace orc;

extern "C" {

struct orc_mech_c {
  int ns, nr;
  const double* M;
  const double* nasa;
  const double* A;
  const double* b;
  const double* Ea;
  const int* nuf;
  const int* nub;
  const int* tb;
  const double* eff;
};

struct orc_grid_c {
  int nx, ny;
  double dx, dy;
  int bc[4];
  double weno_eps;
  double newton_tol;
  int newton_maxit;
};

}  // extern "C"

static Mech to_mech(const orc_mech_c* c) {
  Mech m;
  m.ns = c->ns;
  m.nr = c->nr;
  m.M.assign(c->M, c->M + c->ns);
  m.nasa.assign(c->nasa, c->nasa + 7 * c->ns);
  if (c->nr > 0) {
    m.A.assign(c->A, c->A + c->nr);
    m.b.assign(c->b, c->b + c->nr);
    m.Ea.assign(c->Ea, c->Ea + c->nr);
    m.nuf.assign(c->nuf, c->nuf + c->nr * c->ns);
    m.nub.assign(c->nub, c->nub + c->nr * c->ns);
    m.tb.assign(c->tb, c->tb + c->nr);
    m.eff.assign(c->eff, c->eff + c->nr * c->ns);
  }
  return m;
}

static Grid to_grid(const orc_grid_c* c) {
  Grid g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.dx = c->dx;
  g.dy = c->dy;
  for (int s = 0; s < 4; ++s) g.bc[s] = c->bc[s];
  g.weno_eps = c->weno_eps;
  g.newton_tol = c->newton_tol;
  g.newton_maxit = c->newton_maxit;
  return g;
}

template <class S> static void load_field(Field<S>& F, const Mech& m, const Grid& g, const double* U,
                                          const double* T) {
  F.resize(nvar_of(m), g.nx, g.ny);
  for (size_t q = 0; q < F.U.size(); ++q) F.U[q] = S(U[q]);
  for (size_t q = 0; q < F.T.size(); ++q) F.T[q] = S(T[q]);
}

static void store_field(const Field<double>& F, double* U, double* T) {
  std::memcpy(U, F.U.data(), F.U.size() * sizeof(double));
  std::memcpy(T, F.T.data(), F.T.size() * sizeof(double));
}

// Tangent of an n-step fixed-dt trajectory along up to LANES directions at
// once. dU0: [nl][nv][ny][nx]; the temperature tangents are made consistent
// by a Newton solve. Outputs: dUN [nl][nv][ny][nx] and loss[0..nl] = the value
// and the tangents of L = sum_n dt mean_j p(nx-1, j) of U^{n+1}.
template <int LANES>
static int trajectory_tangent(const orc_mech_c* mc, const orc_grid_c* gc, const double* U, const double* T,
                              const double* dU0, int nl, int nsteps, double dt, int chem, double* dUN, double* loss) {
  using D = Dual<double, LANES>;
  if (nl < 1 || nl > LANES) return -1;
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<D> F;
  F.resize(nvar_of(m), g.nx, g.ny);
  const size_t N = F.U.size();
  for (size_t q = 0; q < N; ++q) {
    F.U[q] = D(U[q]);
    for (int l = 0; l < nl; ++l) F.U[q].d[l] = dU0[(size_t)l * N + q];
  }
  int st = 0;
  for (int j = 0; j < g.ny; ++j)
    for (int i = 0; i < g.nx; ++i) {
      D u[16];
      for (int k = 0; k < F.nv; ++k) u[k] = F.u(k, i, j);
      F.t(i, j) = newton_T(m, g, u, D(T[(size_t)j * g.nx + i]), &st);
    }
  D L(0.0);
  for (int n = 0; n < nsteps; ++n) {
    st |= advance_one_step(m, g, F, dt, chem);
    D s(0.0);
    for (int j = 0; j < g.ny; ++j) {
      D u[16];
      for (int k = 0; k < F.nv; ++k) u[k] = F.u(k, g.nx - 1, j);
      s = s + primitives(m, u, F.t(g.nx - 1, j)).p;
    }
    L = L + (dt / g.ny) * s;
  }
  for (size_t q = 0; q < N; ++q)
    for (int l = 0; l < nl; ++l) dUN[(size_t)l * N + q] = F.U[q].d[l];
  loss[0] = L.v;
  for (int l = 0; l < nl; ++l) loss[1 + l] = L.d[l];
  return st;
}

extern "C" {

// Sets the OpenMP thread count (n <= 0 keeps the default); returns the count in use.
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_thermo(const orc_mech_c* mc, int k, double T, double* cp, double* h, double* s) {
  Mech m = to_mech(mc);
  *cp = cp_R(m, k, T);
  *h = h_R(m, k, T);
  *s = s_R(m, k, T);
  return 0;
}

double orc_weno5(double f0, double f1, double f2, double f3, double f4, double eps) {
  return weno5(f0, f1, f2, f3, f4, eps);
}

// U[nv][n] from T, p, u, v [n] and Y[ns][n].
int orc_prim_to_cons(const orc_mech_c* mc, int n, const double* T, const double* p, const double* vx,
                     const double* vy, const double* Y, double* U) {
  Mech m = to_mech(mc);
  const int nv = nvar_of(m);
  for (int c = 0; c < n; ++c) {
    double Yc[16], u[16];
    for (int k = 0; k < m.ns; ++k) Yc[k] = Y[(size_t)k * n + c];
    prim_to_cons(m, T[c], p[c], vx[c], vy[c], Yc, u);
    for (int k = 0; k < nv; ++k) U[(size_t)k * n + c] = u[k];
  }
  return 0;
}

// Per-cell Newton T from warm starts T0; returns the OR of the status bits.
int orc_newton(const orc_mech_c* mc, const orc_grid_c* gc, int n, const double* U, const double* T0, double* T) {
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  const int nv = nvar_of(m);
  int st = 0;
  for (int c = 0; c < n; ++c) {
    double u[16];
    for (int k = 0; k < nv; ++k) u[k] = U[(size_t)k * n + c];
    T[c] = newton_T(m, g, u, T0[c], &st);
  }
  return st;
}

// p and c per cell.
int orc_primitives(const orc_mech_c* mc, int n, const double* U, const double* T, double* p, double* c) {
  Mech m = to_mech(mc);
  const int nv = nvar_of(m);
  for (int q = 0; q < n; ++q) {
    double u[16];
    for (int k = 0; k < nv; ++k) u[k] = U[(size_t)k * n + q];
    Prim<double> P = primitives(m, u, T[q]);
    p[q] = P.p;
    c[q] = P.c;
  }
  return 0;
}

int orc_production_rates(const orc_mech_c* mc, double T, const double* X, double* w) {
  Mech m = to_mech(mc);
  production_rates(m, T, X, w);
  return 0;
}

// S[ns-1] and J[(ns-1)^2] for one cell's conserved vector u[nv].
int orc_source_jacobian(const orc_mech_c* mc, const double* u, double T, double* S, double* J) {
  Mech m = to_mech(mc);
  if (m.ns - 1 > JAC_LANES) return -1;
  source_and_jacobian(m, u, T, S, J);
  return 0;
}

// Point-implicit update of n cells in place (U[nv][n]).
int orc_point_implicit(const orc_mech_c* mc, int n, double* U, const double* T, double dt) {
  Mech m = to_mech(mc);
  const int nv = nvar_of(m);
  int st = 0;
  for (int c = 0; c < n; ++c) {
    double u[16];
    for (int k = 0; k < nv; ++k) u[k] = U[(size_t)k * n + c];
    point_implicit(m, u, T[c], dt, &st);
    for (int k = 0; k < nv; ++k) U[(size_t)k * n + c] = u[k];
  }
  return st;
}

int orc_lu_solve(int n, double* A, double* b) { return lu_solve(n, A, b) ? 0 : ST_SINGULAR; }

// L(U) and, optionally, the face fluxes and the two LF speeds.
int orc_rhs(const orc_mech_c* mc, const orc_grid_c* gc, const double* U, const double* T, double* L,
            double* Fx, double* Gy, double* alpha) {
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<double> F;
  load_field(F, m, g, U, T);
  std::vector<double> Lv, Fxv, Gyv;
  double ax, ay;
  rhs(m, g, F, Lv, &Fxv, &Gyv, &ax, &ay);
  std::memcpy(L, Lv.data(), Lv.size() * sizeof(double));
  if (Fx) std::memcpy(Fx, Fxv.data(), Fxv.size() * sizeof(double));
  if (Gy) std::memcpy(Gy, Gyv.data(), Gyv.size() * sizeof(double));
  if (alpha) { alpha[0] = ax; alpha[1] = ay; }
  return 0;
}

double orc_cfl_dt(const orc_mech_c* mc, const orc_grid_c* gc, const double* U, const double* T, double cfl) {
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<double> F;
  load_field(F, m, g, U, T);
  return cfl_dt(m, g, F, cfl);
}

// n time steps in place. Exactly one of dt > 0 (fixed step) or cfl > 0.
// dt_log (may be null) receives the dt of every step.
// Right-hand side of an nx x ny field given with its 3 ghost layers
// (Up[nv][ny+6][nx+6], Tp[ny+6][nx+6]; corners ignored) and given LF speeds;
// the building block of a refined block's update, whose ghosts come from its
// neighbours. L: [nv][ny][nx].
int orc_rhs_ghosted(const orc_mech_c* mc, const orc_grid_c* gc, const double* Up, const double* Tp, double ax,
                    double ay, double* L) {
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<double> P;
  P.resize(nvar_of(m), g.nx + 6, g.ny + 6);
  std::memcpy(P.U.data(), Up, sizeof(double) * P.U.size());
  std::memcpy(P.T.data(), Tp, sizeof(double) * P.T.size());
  std::vector<double> Lv;
  rhs_ghosted(m, g, P, ax, ay, Lv);
  std::memcpy(L, Lv.data(), sizeof(double) * Lv.size());
  return 0;
}

// LF speeds (alpha_x, alpha_y) of Eq. 4.11 over n cells U[nv][n], T[n].
int orc_lf_alpha(const orc_mech_c* mc, int n, const double* U, const double* T, double* alpha) {
  Mech m = to_mech(mc);
  Field<double> F;
  F.resize(nvar_of(m), n, 1);
  std::memcpy(F.U.data(), U, sizeof(double) * F.U.size());
  std::memcpy(F.T.data(), T, sizeof(double) * F.T.size());
  double ax, ay;
  lf_alpha(m, F, &ax, &ay);
  alpha[0] = ax;
  alpha[1] = ay;
  return 0;
}

int orc_step(const orc_mech_c* mc, const orc_grid_c* gc, double* U, double* T, int nsteps, double dt,
             double cfl, int chem, double* t_out, double* dt_log) {
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<double> F;
  load_field(F, m, g, U, T);
  int st = 0;
  double t = 0.0;
  for (int n = 0; n < nsteps; ++n) {
    double h = dt > 0.0 ? dt : cfl_dt(m, g, F, cfl);
    st |= advance_one_step(m, g, F, h, chem);
    t += h;
    if (dt_log) dt_log[n] = h;
  }
  store_field(F, U, T);
  if (t_out) *t_out = t;
  return st;
}

// Tangent-linear model of n fixed-dt steps: (U, T) advance as in orc_step and
// (dU, dT) carry the directional derivative of the state along the input
// direction (dU, dT).
int orc_step_tangent(const orc_mech_c* mc, const orc_grid_c* gc, double* U, double* T, double* dU, double* dT,
                     int nsteps, double dt, int chem) {
  using D = Dual<double, 1>;
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<D> F;
  F.resize(nvar_of(m), g.nx, g.ny);
  for (size_t q = 0; q < F.U.size(); ++q) { F.U[q] = D(U[q]); F.U[q].d[0] = dU[q]; }
  for (size_t q = 0; q < F.T.size(); ++q) { F.T[q] = D(T[q]); F.T[q].d[0] = dT[q]; }
  int st = 0;
  for (int n = 0; n < nsteps; ++n) st |= advance_one_step(m, g, F, dt, chem);
  for (size_t q = 0; q < F.U.size(); ++q) { U[q] = F.U[q].v; dU[q] = F.U[q].d[0]; }
  for (size_t q = 0; q < F.T.size(); ++q) { T[q] = F.T[q].v; dT[q] = F.T[q].d[0]; }
  return st;
}

// Tangent of the right-hand side at (U, T) along dU: dL = (dL/dU) dU, with the
// temperature tangent made consistent by a Newton solve on dual numbers.
int orc_rhs_tangent(const orc_mech_c* mc, const orc_grid_c* gc, const double* U, const double* T, const double* dU,
                    double* dL) {
  using D = Dual<double, 1>;
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
  Field<D> F;
  F.resize(nvar_of(m), g.nx, g.ny);
  for (size_t q = 0; q < F.U.size(); ++q) { F.U[q] = D(U[q]); F.U[q].d[0] = dU[q]; }
  int st = 0;
  for (int j = 0; j < g.ny; ++j)
    for (int i = 0; i < g.nx; ++i) {
      D u[16];
      for (int k = 0; k < F.nv; ++k) u[k] = F.u(k, i, j);
      F.t(i, j) = newton_T(m, g, u, D(T[(size_t)j * g.nx + i]), &st);
    }
  std::vector<D> L;
  rhs(m, g, F, L);
  for (size_t q = 0; q < L.size(); ++q) dL[q] = L[q].d[0];
  return st;
}

int orc_trajectory_tangent8(const orc_mech_c* mc, const orc_grid_c* gc, const double* U, const double* T,
                            const double* dU0, int nl, int nsteps, double dt, int chem, double* dUN, double* loss) {
  if (nl == 1) return trajectory_tangent<1>(mc, gc, U, T, dU0, nl, nsteps, dt, chem, dUN, loss);
  return trajectory_tangent<8>(mc, gc, U, T, dU0, nl, nsteps, dt, chem, dUN, loss);
}

// Operation counts (add, mul, div, sqrt, exp, log) of the plain algorithm.
// part: 0 = one WENO5 reconstruction, 1 = rhs over the grid, 2 = Newton on
// every cell (warm start from T0), 3 = point-implicit chemistry on every
// cell, 4 = one full step (fixed dt).
int orc_opcount(const orc_mech_c* mc, const orc_grid_c* gc, int part, const double* U, const double* T,
                double dt, long long* out6) {
  Mech m = to_mech(mc);
  Grid g = to_grid(gc);
#ifdef _OPENMP
  int saved = omp_get_max_threads();
  omp_set_num_threads(1);
#endif
  g_ops = OpCount();
  int st = 0;
  if (part == 0) {
    Cnt r = weno5(Cnt(1.0), Cnt(2.0), Cnt(4.0), Cnt(3.0), Cnt(5.0), g.weno_eps);
    (void)r;
  } else {
    Field<Cnt> F;
    load_field(F, m, g, U, T);
    if (part == 1) {
      std::vector<Cnt> L;
      rhs(m, g, F, L);
    } else if (part == 2) {
      Field<Cnt> W = F;
      st |= update_T(m, g, F, W);
    } else if (part == 3) {
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
          Cnt u[16];
          for (int k = 0; k < F.nv; ++k) u[k] = F.u(k, i, j);
          point_implicit(m, u, F.t(i, j), dt, &st);
        }
    } else if (part == 4) {
      st |= advance_one_step(m, g, F, dt, true);
    }
  }
  out6[0] = g_ops.add;
  out6[1] = g_ops.mul;
  out6[2] = g_ops.div;
  out6[3] = g_ops.sqrt;
  out6[4] = g_ops.exp;
  out6[5] = g_ops.log;
#ifdef _OPENMP
  omp_set_num_threads(saved);
#endif
  return st;
}

}  // extern "C"
