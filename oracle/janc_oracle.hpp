// JANC reacting-flow step: plain CPU FP64 oracle (TEST INFRASTRUCTURE ONLY).
//
// This file is the reference against which the CUDA path is checked. Only the
// tests, the smoke check and the CPU-baseline leg of the benchmark may build,
// load or run it; the product path never does.
//
// It restates the method of arXiv 2504.13750 step by step, in the paper's
// order and notation, with no blocking, fusion or reordering:
//   Sec. 4.1  Eq. 4.1  reactive Euler system, U = [rho, rho u, rho v, E, rho Y_1..rho Y_{Ns-1}]
//             Eq. 4.2  thermally perfect EOS (p = rho R T, E = rho h - p + rho|u|^2/2)
//             Eq. 4.3-4.5 NASA-7 polynomials for cp, h, s
//             Eq. 4.6-4.9 finite-rate kinetics, Arrhenius + equilibrium reverse rate
//   Sec. 4.2  Eq. 4.10 conservative finite-difference flux difference
//             Eq. 4.11 global Lax-Friedrichs flux-vector splitting
//             WENO5 reconstruction with 3 ghost layers (text after Eq. 4.11)
//             3rd-order TVD Runge-Kutta for convection, Newton-Raphson T recovery
//             warm-started from the previous T (end of Sec. 4.2)
//             Eq. 4.12-4.13 first-order point-implicit chemistry, Jacobian over
//             rho Y_1..rho Y_{Ns-1} only
//   Sec. 4.3  advance_one_step = CFL, advance_flux (RK3), advance_source_term
//
// The code is templated on the scalar type so that the same text runs in
// plain double, in forward-mode dual numbers (tangent-linear checks and the
// chemistry Jacobian, which is by definition dS/d(rho Y)), and in an
// operation-counting scalar (algorithmic flop counts).
//
// Readings where the paper is silent or ambiguous (each one is applied the
// same way in the CUDA path and listed in the design notes):
//   * splitting order: flux(dt) then chemistry(dt), as advance_one_step is
//     written in Sec. 4.3 (Lie order); the Strang order the text of Sec. 4.3
//     names is the CHEM_STRANG variant (chemistry dt/2, flux dt, chemistry dt/2);
//   * alpha in Eq. 4.11: global max over interior cells, per direction
//     (|u|+c for x, |v|+c for y), recomputed from each RK stage's input;
//   * WENO5-JS (Jiang & Shu 1996) with epsilon = weno_eps and power 2,
//     applied component-wise to the split conserved fluxes;
//   * CFL: dt = CFL * min(dx, dy) / max(alpha_x, alpha_y) of the step's
//     starting state;
//   * slip wall = mirror ghost with the wall-normal momentum negated;
//     non-reflecting = zero-gradient copy of the edge cell; periodic = wrap;
//   * third-body factor = 1 for reactions without a third body;
//   * Newton stops when |dT| <= tol * T after the update, at most maxit
//     iterations;
//   * every state (U^n, U^1, U^2, U^*, U^{n+1}) carries the T obtained by
//     Newton from its own U, warm-started from the previous state's T;
//   * sound speed is the frozen c = sqrt(gamma R T), gamma = cp / cv.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace orc {

constexpr double RU = 8.314472;     // universal gas constant, J/(mol K), text after Eq. 4.5
constexpr double P_REF = 101325.0;  // reference pressure in Eq. 4.9, Pa

// Status bits (per cell, OR-ed together).
enum : int {
  ST_OK = 0,
  ST_NONFINITE = 1,
  ST_NONPOSITIVE = 2,     // rho, p or T <= 0
  ST_NEWTON_FAIL = 4,
  ST_SINGULAR = 8,
};

// --------------------------------------------------------------------------
// Scalar types.
// --------------------------------------------------------------------------
inline double val(double x) { return x; }
using std::exp;
using std::fabs;
using std::log;
using std::sqrt;

// Forward-mode dual number over a base scalar B with N tangent lanes.
template <class B, int N>
struct Dual {
  B v;
  B d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = B(0.0); }
  Dual(double c) : v(c) { for (int i = 0; i < N; ++i) d[i] = B(0.0); }
  explicit Dual(const B& c, int) : v(c) { for (int i = 0; i < N; ++i) d[i] = B(0.0); }
};
template <class B, int N> double val(const Dual<B, N>& x) { return val(x.v); }

#define ORC_DUAL_T template <class B, int N>
#define ORC_DUAL Dual<B, N>
ORC_DUAL_T ORC_DUAL operator+(const ORC_DUAL& a, const ORC_DUAL& b) {
  ORC_DUAL r(a.v + b.v, 0); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
ORC_DUAL_T ORC_DUAL operator-(const ORC_DUAL& a, const ORC_DUAL& b) {
  ORC_DUAL r(a.v - b.v, 0); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
ORC_DUAL_T ORC_DUAL operator-(const ORC_DUAL& a) {
  ORC_DUAL r(-a.v, 0); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
ORC_DUAL_T ORC_DUAL operator*(const ORC_DUAL& a, const ORC_DUAL& b) {
  ORC_DUAL r(a.v * b.v, 0); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
ORC_DUAL_T ORC_DUAL operator/(const ORC_DUAL& a, const ORC_DUAL& b) {
  B q = a.v / b.v; ORC_DUAL r(q, 0);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - q * b.d[i]) / b.v;
  return r;
}
ORC_DUAL_T ORC_DUAL operator+(const ORC_DUAL& a, double b) { return a + ORC_DUAL(b); }
ORC_DUAL_T ORC_DUAL operator+(double a, const ORC_DUAL& b) { return ORC_DUAL(a) + b; }
ORC_DUAL_T ORC_DUAL operator-(const ORC_DUAL& a, double b) { return a - ORC_DUAL(b); }
ORC_DUAL_T ORC_DUAL operator-(double a, const ORC_DUAL& b) { return ORC_DUAL(a) - b; }
ORC_DUAL_T ORC_DUAL operator*(const ORC_DUAL& a, double b) {
  ORC_DUAL r(a.v * b, 0); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
ORC_DUAL_T ORC_DUAL operator*(double a, const ORC_DUAL& b) { return b * a; }
ORC_DUAL_T ORC_DUAL operator/(const ORC_DUAL& a, double b) {
  ORC_DUAL r(a.v / b, 0); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / b;
  return r;
}
ORC_DUAL_T ORC_DUAL operator/(double a, const ORC_DUAL& b) { return ORC_DUAL(a) / b; }
ORC_DUAL_T ORC_DUAL& operator+=(ORC_DUAL& a, const ORC_DUAL& b) { a = a + b; return a; }
ORC_DUAL_T ORC_DUAL& operator-=(ORC_DUAL& a, const ORC_DUAL& b) { a = a - b; return a; }
ORC_DUAL_T ORC_DUAL exp(const ORC_DUAL& a) {
  using std::exp; B e = exp(a.v); ORC_DUAL r(e, 0);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * e;
  return r;
}
ORC_DUAL_T ORC_DUAL log(const ORC_DUAL& a) {
  using std::log; ORC_DUAL r(log(a.v), 0);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / a.v;
  return r;
}
ORC_DUAL_T ORC_DUAL sqrt(const ORC_DUAL& a) {
  using std::sqrt; B s = sqrt(a.v); ORC_DUAL r(s, 0);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * s);
  return r;
}
ORC_DUAL_T ORC_DUAL fabs(const ORC_DUAL& a) { return val(a) < 0.0 ? -a : a; }
#undef ORC_DUAL_T
#undef ORC_DUAL

// Operation-counting scalar: forwards to double and tallies each operation.
struct OpCount {
  long long add = 0, mul = 0, div = 0, sqrt = 0, exp = 0, log = 0;
};
extern thread_local OpCount g_ops;

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  explicit Cnt(double c) : v(c) {}
};
inline double val(const Cnt& x) { return x.v; }
inline Cnt operator+(const Cnt& a, const Cnt& b) { ++g_ops.add; return Cnt(a.v + b.v); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { ++g_ops.add; return Cnt(a.v - b.v); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { ++g_ops.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(const Cnt& a, const Cnt& b) { ++g_ops.div; return Cnt(a.v / b.v); }
inline Cnt operator+(const Cnt& a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, const Cnt& b) { return Cnt(a) + b; }
inline Cnt operator-(const Cnt& a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, const Cnt& b) { return Cnt(a) - b; }
inline Cnt operator*(const Cnt& a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, const Cnt& b) { return Cnt(a) * b; }
inline Cnt operator/(const Cnt& a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, const Cnt& b) { return Cnt(a) / b; }
inline Cnt& operator+=(Cnt& a, const Cnt& b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, const Cnt& b) { a = a - b; return a; }
inline Cnt exp(const Cnt& a) { ++g_ops.exp; return Cnt(std::exp(a.v)); }
inline Cnt log(const Cnt& a) { ++g_ops.log; return Cnt(std::log(a.v)); }
inline Cnt sqrt(const Cnt& a) { ++g_ops.sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt fabs(const Cnt& a) { return Cnt(std::fabs(a.v)); }

template <class S> inline S sq(const S& x) { return x * x; }

// Integer power by repeated multiplication (defined for negative bases, so no
// clipping of concentrations is needed).
template <class S> inline S ipow(const S& x, int n) {
  S r(1.0);
  for (int i = 0; i < n; ++i) r = r * x;
  return r;
}

// --------------------------------------------------------------------------
// Mechanism and grid descriptions.
// --------------------------------------------------------------------------
struct Mech {
  int ns = 0;                    // species; the last one is the Ns-th species (e.g. N2)
  int nr = 0;                    // reactions
  std::vector<double> M;         // [ns] molar mass, kg/mol
  std::vector<double> nasa;      // [ns][7] NASA-7 coefficients a_0..a_6 (single range)
  std::vector<double> A, b, Ea;  // [nr] Arrhenius: k_f = A T^b exp(-Ea/(Ru T)), SI units, Ea in J/mol
  std::vector<int> nuf, nub;     // [nr][ns] stoichiometric coefficients (reactants, products)
  std::vector<int> tb;           // [nr] 1 if the reaction carries a third-body factor
  std::vector<double> eff;       // [nr][ns] third-body coefficients a_ij
};

enum Bc : int { BC_WALL = 0, BC_ZEROGRAD = 1, BC_PERIODIC = 2 };

struct Grid {
  int nx = 0, ny = 0;
  double dx = 1.0, dy = 1.0;
  int bc[4] = {BC_WALL, BC_WALL, BC_WALL, BC_WALL};  // left, right, bottom, top
  double weno_eps = 1e-6;
  double newton_tol = 1e-12;
  int newton_maxit = 50;
};

inline int nvar_of(const Mech& m) { return 3 + m.ns; }  // 4 + (Ns - 1)

// --------------------------------------------------------------------------
// Thermodynamics (Eq. 4.3-4.5), dimensionless per species.
// --------------------------------------------------------------------------
// cp_k / (Ru/M_k), Eq. 4.3
template <class S> S cp_R(const Mech& m, int k, const S& T) {
  const double* a = &m.nasa[7 * k];
  return a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
}
// h_k / (Ru/M_k), Eq. 4.4
template <class S> S h_R(const Mech& m, int k, const S& T) {
  const double* a = &m.nasa[7 * k];
  return a[0] * T + a[1] / 2.0 * T * T + a[2] / 3.0 * T * T * T + a[3] / 4.0 * T * T * T * T +
         a[4] / 5.0 * T * T * T * T * T + a[5];
}
// s_k / (Ru/M_k), Eq. 4.5
template <class S> S s_R(const Mech& m, int k, const S& T) {
  const double* a = &m.nasa[7 * k];
  return a[0] * log(T) + a[1] * T + a[2] / 2.0 * T * T + a[3] / 3.0 * T * T * T +
         a[4] / 4.0 * T * T * T * T + a[6];
}

// Mass fractions of all Ns species from one cell's conserved vector u[0..nv).
// Y_Ns = 1 - sum of the others (Eq. 4.1 carries only Ns-1 species).
template <class S> void mass_fractions(const Mech& m, const S* u, S* Y) {
  S rho = u[0];
  S sum(0.0);
  for (int k = 0; k < m.ns - 1; ++k) {
    Y[k] = u[4 + k] / rho;
    sum = sum + Y[k];
  }
  Y[m.ns - 1] = 1.0 - sum;
}

// Mixture properties per unit mass (Eq. 4.2): R = Ru sum Y_k/M_k, h = sum Y_k h_k, cp = sum Y_k cp_k.
template <class S> S mix_R(const Mech& m, const S* Y) {
  S r(0.0);
  for (int k = 0; k < m.ns; ++k) r = r + Y[k] * (RU / m.M[k]);
  return r;
}
template <class S> S mix_h(const Mech& m, const S* Y, const S& T) {
  S h(0.0);
  for (int k = 0; k < m.ns; ++k) h = h + Y[k] * (RU / m.M[k]) * h_R(m, k, T);
  return h;
}
template <class S> S mix_cp(const Mech& m, const S* Y, const S& T) {
  S c(0.0);
  for (int k = 0; k < m.ns; ++k) c = c + Y[k] * (RU / m.M[k]) * cp_R(m, k, T);
  return c;
}

// Newton-Raphson T recovery from the energy (end of Sec. 4.2): solve
//   h(T) - R T = e,  e = E/rho - (u^2+v^2)/2   (from Eq. 4.2 with p = rho R T)
// with f' = cp - R = cv, warm-started from T0.
template <class S> S newton_T(const Mech& m, const Grid& g, const S* u, const S& T0, int* status) {
  const int ns = m.ns;
  S Y[16];
  mass_fractions(m, u, Y);
  S rho = u[0];
  S vx = u[1] / rho, vy = u[2] / rho;
  S e = u[3] / rho - 0.5 * (vx * vx + vy * vy);
  S R = mix_R(m, Y);
  S T = T0;
  (void)ns;
  for (int it = 0; it < g.newton_maxit; ++it) {
    S f = mix_h(m, Y, T) - R * T - e;
    S fp = mix_cp(m, Y, T) - R;
    S dT = -f / fp;
    T = T + dT;
    if (std::fabs(val(dT)) <= g.newton_tol * std::fabs(val(T))) return T;
  }
  *status |= ST_NEWTON_FAIL;
  return T;
}

// Primitive variables of one cell: p (Eq. 4.2), frozen sound speed.
template <class S> struct Prim {
  S rho, u, v, p, c;
};
template <class S> Prim<S> primitives(const Mech& m, const S* u, const S& T) {
  S Y[16];
  mass_fractions(m, u, Y);
  Prim<S> P;
  P.rho = u[0];
  P.u = u[1] / P.rho;
  P.v = u[2] / P.rho;
  S R = mix_R(m, Y);
  S cp = mix_cp(m, Y, T);
  S cv = cp - R;
  S gamma = cp / cv;
  P.p = P.rho * R * T;
  P.c = sqrt(gamma * R * T);
  return P;
}

// Conserved vector from primitive data (T, p, u, v, all Ns mass fractions), Eq. 4.2.
template <class S> void prim_to_cons(const Mech& m, const S& T, const S& p, const S& vx, const S& vy,
                                     const S* Yall, S* u) {
  S R = mix_R(m, Yall);
  S rho = p / (R * T);
  S h = mix_h(m, Yall, T);
  u[0] = rho;
  u[1] = rho * vx;
  u[2] = rho * vy;
  u[3] = rho * h - p + 0.5 * rho * (vx * vx + vy * vy);
  for (int k = 0; k < m.ns - 1; ++k) u[4 + k] = rho * Yall[k];
}

// --------------------------------------------------------------------------
// Chemistry (Eq. 4.6-4.9): production rates w_k (kg/m^3/s) from T and the
// molar concentrations X_j (mol/m^3) of all Ns species.
// --------------------------------------------------------------------------
template <class S> void production_rates(const Mech& m, const S& T, const S* X, S* w) {
  const int ns = m.ns;
  for (int k = 0; k < ns; ++k) w[k] = S(0.0);
  // g_j = s_j/(Ru/M_j) - h_j/(Ru T/M_j): the bracket of Eq. 4.9 per species.
  S gj[16];
  for (int j = 0; j < ns; ++j) gj[j] = s_R(m, j, T) - h_R(m, j, T) / T;
  for (int i = 0; i < m.nr; ++i) {
    const int* nf = &m.nuf[i * ns];
    const int* nb = &m.nub[i * ns];
    // Eq. 4.8: forward rate (T^b written as exp(b ln T))
    S kf = m.A[i] * exp(m.b[i] * log(T)) * exp(-m.Ea[i] / (RU * T));
    // Eq. 4.9: equilibrium constant
    S sum_g(0.0);
    int dnu = 0;
    for (int j = 0; j < ns; ++j) {
      int nu = nb[j] - nf[j];
      if (nu != 0) sum_g = sum_g + double(nu) * gj[j];
      dnu += nu;
    }
    S conc_ref = P_REF / (RU * T);
    S Keq = exp(sum_g);
    if (dnu >= 0) Keq = Keq * ipow(conc_ref, dnu);
    else Keq = Keq / ipow(conc_ref, -dnu);
    S kb = kf / Keq;
    // Eq. 4.7: law of mass action with the third-body factor
    S fwd = kf, bwd = kb;
    for (int j = 0; j < ns; ++j) {
      if (nf[j]) fwd = fwd * ipow(X[j], nf[j]);
      if (nb[j]) bwd = bwd * ipow(X[j], nb[j]);
    }
    S third(1.0);
    if (m.tb[i]) {
      third = S(0.0);
      for (int j = 0; j < ns; ++j) third = third + m.eff[i * ns + j] * X[j];
    }
    S q = third * (fwd - bwd);
    for (int k = 0; k < ns; ++k) {
      int nu = nb[k] - nf[k];
      if (nu != 0) w[k] = w[k] + m.M[k] * double(nu) * q;
    }
  }
}

// Molar concentrations of all Ns species from a conserved vector; the Ns-th
// species is what remains of rho after the carried partial densities.
template <class S> void concentrations(const Mech& m, const S* u, S* X) {
  S rest = u[0];
  for (int k = 0; k < m.ns - 1; ++k) {
    X[k] = u[4 + k] / m.M[k];
    rest = rest - u[4 + k];
  }
  X[m.ns - 1] = rest / m.M[m.ns - 1];
}

// Dense solve A x = b with LU factorisation and partial pivoting (first
// largest |pivot| wins on ties). A and b are overwritten; x returned in b.
template <class S> bool lu_solve(int n, S* A, S* b) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = std::fabs(val(A[c * n + c]));
    for (int r = c + 1; r < n; ++r) {
      double a = std::fabs(val(A[r * n + c]));
      if (a > best) { best = a; p = r; }
    }
    if (!(best > 0.0)) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[p * n + k]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < n; ++r) {
      S f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] = A[r * n + k] - f * A[c * n + k];
      b[r] = b[r] - f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    S s = b[r];
    for (int k = r + 1; k < n; ++k) s = s - A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return true;
}

constexpr int JAC_LANES = 8;  // tangent lanes for the chemistry Jacobian (Ns - 1 <= 8)

// Source vector S = [w_1..w_{Ns-1}] and its Jacobian J_kl = dS_k/d(rho Y_l)
// with T and rho held fixed (text after Eq. 4.13), by forward-mode
// differentiation of production_rates: the definition of the Jacobian.
template <class S> void source_and_jacobian(const Mech& m, const S* u, const S& T, S* Svec, S* J) {
  using D = Dual<S, JAC_LANES>;
  const int nsp = m.ns - 1;
  D ud[16];
  for (int k = 0; k < nvar_of(m); ++k) ud[k] = D(u[k], 0);
  for (int l = 0; l < nsp; ++l) ud[4 + l].d[l] = S(1.0);
  D X[16], w[16];
  concentrations(m, ud, X);
  production_rates(m, D(T, 0), X, w);
  for (int k = 0; k < nsp; ++k) {
    Svec[k] = w[k].v;
    for (int l = 0; l < nsp; ++l) J[k * nsp + l] = w[k].d[l];
  }
}

// First-order point-implicit update of one cell (Eq. 4.12-4.13):
//   (I - dt dS/dU) dU = S dt,  U_new = U + dU,  species components only.
template <class S> void point_implicit(const Mech& m, S* u, const S& T, double dt, int* status) {
  const int nsp = m.ns - 1;
  if (nsp <= 0 || m.nr == 0) return;
  S Svec[JAC_LANES], J[JAC_LANES * JAC_LANES];
  source_and_jacobian(m, u, T, Svec, J);
  S A[JAC_LANES * JAC_LANES], rhs[JAC_LANES];
  for (int k = 0; k < nsp; ++k) {
    for (int l = 0; l < nsp; ++l) A[k * nsp + l] = (k == l ? 1.0 : 0.0) - dt * J[k * nsp + l];
    rhs[k] = Svec[k] * dt;
  }
  if (!lu_solve(nsp, A, rhs)) { *status |= ST_SINGULAR; return; }
  for (int k = 0; k < nsp; ++k) u[4 + k] = u[4 + k] + rhs[k];
}

// --------------------------------------------------------------------------
// WENO5-JS reconstruction (Jiang & Shu 1996) of the value at the right face of
// the centre point f2 from the five point values f0..f4 = f_{i-2}..f_{i+2}.
// --------------------------------------------------------------------------
template <class S> S weno5(const S& f0, const S& f1, const S& f2, const S& f3, const S& f4, double eps) {
  S b0 = 13.0 / 12.0 * sq(f0 - 2.0 * f1 + f2) + 0.25 * sq(f0 - 4.0 * f1 + 3.0 * f2);
  S b1 = 13.0 / 12.0 * sq(f1 - 2.0 * f2 + f3) + 0.25 * sq(f1 - f3);
  S b2 = 13.0 / 12.0 * sq(f2 - 2.0 * f3 + f4) + 0.25 * sq(3.0 * f2 - 4.0 * f3 + f4);
  S a0 = 0.1 / sq(eps + b0);
  S a1 = 0.6 / sq(eps + b1);
  S a2 = 0.3 / sq(eps + b2);
  S s = a0 + a1 + a2;
  S q0 = (2.0 * f0 - 7.0 * f1 + 11.0 * f2) / 6.0;
  S q1 = (-f1 + 5.0 * f2 + 2.0 * f3) / 6.0;
  S q2 = (2.0 * f2 + 5.0 * f3 - f4) / 6.0;
  return (a0 * q0 + a1 * q1 + a2 * q2) / s;
}

// --------------------------------------------------------------------------
// Ghost cells (3 layers, text after Eq. 4.11): source index along one axis.
// Returns the interior index that feeds position i in [-3, n+3) and whether
// the wall-normal momentum is negated.
// --------------------------------------------------------------------------
inline int ghost_src(int i, int n, int bc_lo, int bc_hi, bool* flip) {
  *flip = false;
  if (i < 0) {
    if (bc_lo == BC_WALL) { *flip = true; return -1 - i; }
    if (bc_lo == BC_ZEROGRAD) return 0;
    return ((i % n) + n) % n;
  }
  if (i >= n) {
    if (bc_hi == BC_WALL) { *flip = true; return 2 * n - 1 - i; }
    if (bc_hi == BC_ZEROGRAD) return n - 1;
    return i % n;
  }
  return i;
}

// State arrays: U[nv][ny][nx] (x fastest), T[ny][nx].
template <class S> struct Field {
  int nv = 0, nx = 0, ny = 0;
  std::vector<S> U, T;
  void resize(int nv_, int nx_, int ny_) {
    nv = nv_; nx = nx_; ny = ny_;
    U.assign((size_t)nv * nx * ny, S(0.0));
    T.assign((size_t)nx * ny, S(0.0));
  }
  S& u(int k, int i, int j) { return U[((size_t)k * ny + j) * nx + i]; }
  const S& u(int k, int i, int j) const { return U[((size_t)k * ny + j) * nx + i]; }
  S& t(int i, int j) { return T[(size_t)j * nx + i]; }
  const S& t(int i, int j) const { return T[(size_t)j * nx + i]; }
};

// Global Lax-Friedrichs speeds of Eq. 4.11 over the interior cells.
template <class S> void lf_alpha(const Mech& m, const Field<S>& F, S* ax, S* ay) {
  const int nv = F.nv;
  S bx(0.0), by(0.0);
  bool first = true;
  for (int j = 0; j < F.ny; ++j)
    for (int i = 0; i < F.nx; ++i) {
      S u[16];
      for (int k = 0; k < nv; ++k) u[k] = F.u(k, i, j);
      Prim<S> P = primitives(m, u, F.t(i, j));
      S sx = fabs(P.u) + P.c;
      S sy = fabs(P.v) + P.c;
      // max with ties going to the first (lowest linear index) cell
      if (first || val(sx) > val(bx)) bx = sx;
      if (first || val(sy) > val(by)) by = sy;
      first = false;
    }
  *ax = bx;
  *ay = by;
}

// Right-hand side L(U) = -(F_{i+1/2}-F_{i-1/2})/dx - (G_{j+1/2}-G_{j-1/2})/dy
// (Eq. 4.10 without the source; the chemistry is split off) of a field whose
// ghost layers and LF speeds alpha_x, alpha_y (Eq. 4.11) are given: the flux
// split of Eq. 4.11 and WENO5 reconstruction of F+ and F- at every face.
// Optionally returns the face fluxes Fx[nv][ny][nx+1] (face i-1/2 at index i)
// and Gy[nv][ny+1][nx] (face j-1/2 at index j).
template <class S> void rhs_ghosted(const Mech& m, const Grid& g, const Field<S>& P, const S& ax, const S& ay,
                                    std::vector<S>& L, std::vector<S>* Fx_out = nullptr,
                                    std::vector<S>* Gy_out = nullptr) {
  // P is the field extended by 3 ghost cells on every side (P.nx = nx + 6,
  // P.ny = ny + 6; interior cell (i, j) at (i + 3, j + 3)). The x sweep reads
  // the ghost columns of the interior rows, the y sweep the ghost rows of the
  // interior columns; the corners are never read.
  const int nv = P.nv, nx = P.nx - 6, ny = P.ny - 6;
  L.assign((size_t)nv * nx * ny, S(0.0));
  std::vector<S> Fx((size_t)nv * ny * (nx + 1)), Gy((size_t)nv * (ny + 1) * nx);

  // x direction: one row at a time.
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    const int ne = nx + 6;
    std::vector<S> Fp((size_t)nv * ne), Fm((size_t)nv * ne);
    for (int ie = 0; ie < ne; ++ie) {
      S u[16];
      for (int k = 0; k < nv; ++k) u[k] = P.u(k, ie, j + 3);
      Prim<S> Q = primitives(m, u, P.t(ie, j + 3));
      // flux F of Eq. 4.1
      S f[16];
      f[0] = u[1];
      f[1] = u[1] * Q.u + Q.p;
      f[2] = u[2] * Q.u;
      f[3] = (u[3] + Q.p) * Q.u;
      for (int k = 4; k < nv; ++k) f[k] = u[k] * Q.u;
      for (int k = 0; k < nv; ++k) {
        Fp[(size_t)k * ne + ie] = 0.5 * (f[k] + ax * u[k]);
        Fm[(size_t)k * ne + ie] = 0.5 * (f[k] - ax * u[k]);
      }
    }
    for (int k = 0; k < nv; ++k) {
      const S* p = &Fp[(size_t)k * ne];
      const S* q = &Fm[(size_t)k * ne];
      for (int fi = 0; fi <= nx; ++fi) {
        // face between cells fi-1 and fi; extended index of cell i is i+3
        int c = fi - 1 + 3;  // left cell of the face
        S hp = weno5(p[c - 2], p[c - 1], p[c], p[c + 1], p[c + 2], g.weno_eps);
        S hm = weno5(q[c + 3], q[c + 2], q[c + 1], q[c], q[c - 1], g.weno_eps);
        Fx[((size_t)k * ny + j) * (nx + 1) + fi] = hp + hm;
      }
    }
  }
  // y direction: one column at a time.
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < nx; ++i) {
    const int ne = ny + 6;
    std::vector<S> Gp((size_t)nv * ne), Gm((size_t)nv * ne);
    for (int je = 0; je < ne; ++je) {
      S u[16];
      for (int k = 0; k < nv; ++k) u[k] = P.u(k, i + 3, je);
      Prim<S> Q = primitives(m, u, P.t(i + 3, je));
      S f[16];
      f[0] = u[2];
      f[1] = u[1] * Q.v;
      f[2] = u[2] * Q.v + Q.p;
      f[3] = (u[3] + Q.p) * Q.v;
      for (int k = 4; k < nv; ++k) f[k] = u[k] * Q.v;
      for (int k = 0; k < nv; ++k) {
        Gp[(size_t)k * ne + je] = 0.5 * (f[k] + ay * u[k]);
        Gm[(size_t)k * ne + je] = 0.5 * (f[k] - ay * u[k]);
      }
    }
    for (int k = 0; k < nv; ++k) {
      const S* p = &Gp[(size_t)k * ne];
      const S* q = &Gm[(size_t)k * ne];
      for (int fj = 0; fj <= ny; ++fj) {
        int c = fj - 1 + 3;
        S hp = weno5(p[c - 2], p[c - 1], p[c], p[c + 1], p[c + 2], g.weno_eps);
        S hm = weno5(q[c + 3], q[c + 2], q[c + 1], q[c], q[c - 1], g.weno_eps);
        Gy[((size_t)k * (ny + 1) + fj) * nx + i] = hp + hm;
      }
    }
  }
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k < nv; ++k)
      for (int i = 0; i < nx; ++i) {
        S dfx = Fx[((size_t)k * ny + j) * (nx + 1) + i + 1] - Fx[((size_t)k * ny + j) * (nx + 1) + i];
        S dgy = Gy[((size_t)k * (ny + 1) + j + 1) * nx + i] - Gy[((size_t)k * (ny + 1) + j) * nx + i];
        L[((size_t)k * ny + j) * nx + i] = -dfx / g.dx - dgy / g.dy;
      }
  if (Fx_out) *Fx_out = Fx;
  if (Gy_out) *Gy_out = Gy;
}

// The field extended by the 3 ghost layers of the physical boundaries (text
// after Eq. 4.11): ghost_src along each axis; a wall mirror negates the
// wall-normal momentum. Corners are left at zero (never read).
template <class S> Field<S> pad_physical(const Grid& g, const Field<S>& F) {
  Field<S> P;
  P.resize(F.nv, F.nx + 6, F.ny + 6);
  for (int j = 0; j < F.ny; ++j)
    for (int ie = 0; ie < F.nx + 6; ++ie) {
      bool flip;
      int si = ghost_src(ie - 3, F.nx, g.bc[0], g.bc[1], &flip);
      for (int k = 0; k < F.nv; ++k) P.u(k, ie, j + 3) = F.u(k, si, j);
      if (flip) P.u(1, ie, j + 3) = -P.u(1, ie, j + 3);
      P.t(ie, j + 3) = F.t(si, j);
    }
  for (int i = 0; i < F.nx; ++i)
    for (int je = 0; je < F.ny + 6; ++je) {
      if (je >= 3 && je < F.ny + 3) continue;
      bool flip;
      int sj = ghost_src(je - 3, F.ny, g.bc[2], g.bc[3], &flip);
      for (int k = 0; k < F.nv; ++k) P.u(k, i + 3, je) = F.u(k, i, sj);
      if (flip) P.u(2, i + 3, je) = -P.u(2, i + 3, je);
      P.t(i + 3, je) = F.t(i, sj);
    }
  return P;
}

// Right-hand side L(U) = -(dF/dx + dG/dy) of the semi-discrete equation
// (Eq. 4.10 without the source; the chemistry is split off), with the flux
// split of Eq. 4.11 and WENO5 reconstruction of F+ and F- at every face:
// the physical ghost layers, the global LF speeds of the interior cells, then
// rhs_ghosted. Optionally returns the face fluxes Fx[nv][ny][nx+1] (face
// i-1/2 at index i) and Gy[nv][ny+1][nx] (face j-1/2 at index j).
template <class S> void rhs(const Mech& m, const Grid& g, const Field<S>& F, std::vector<S>& L,
                            std::vector<S>* Fx_out = nullptr, std::vector<S>* Gy_out = nullptr,
                            S* ax_out = nullptr, S* ay_out = nullptr) {
  S ax, ay;
  lf_alpha(m, F, &ax, &ay);
  if (ax_out) *ax_out = ax;
  if (ay_out) *ay_out = ay;
  rhs_ghosted(m, g, pad_physical(g, F), ax, ay, L, Fx_out, Gy_out);
}

// Newton T for every cell of `out`, warm-started from `warm`'s T.
template <class S> int update_T(const Mech& m, const Grid& g, Field<S>& out, const Field<S>& warm) {
  int st_all = 0;
  #pragma omp parallel for schedule(static) reduction(| : st_all)
  for (int j = 0; j < out.ny; ++j)
    for (int i = 0; i < out.nx; ++i) {
      S u[16];
      for (int k = 0; k < out.nv; ++k) u[k] = out.u(k, i, j);
      int st = 0;
      out.t(i, j) = newton_T(m, g, u, warm.t(i, j), &st);
      st_all |= st;
    }
  return st_all;
}

// Physical admissibility of a state (status word only; nothing is clipped).
template <class S> int check_state(const Mech& m, const Field<S>& F) {
  int st = 0;
  for (int j = 0; j < F.ny; ++j)
    for (int i = 0; i < F.nx; ++i) {
      S u[16];
      for (int k = 0; k < F.nv; ++k) {
        u[k] = F.u(k, i, j);
        if (!std::isfinite(val(u[k]))) st |= ST_NONFINITE;
      }
      double T = val(F.t(i, j));
      if (!std::isfinite(T)) st |= ST_NONFINITE;
      if (!(val(u[0]) > 0.0) || !(T > 0.0)) st |= ST_NONPOSITIVE;
    }
  (void)m;
  return st;
}

// CFL time step (cfl() of Sec. 4.3) from the state's LF speeds.
template <class S> double cfl_dt(const Mech& m, const Grid& g, const Field<S>& F, double cfl) {
  S ax, ay;
  lf_alpha(m, F, &ax, &ay);
  double amax = std::max(val(ax), val(ay));
  return cfl * std::min(g.dx, g.dy) / amax;
}

// The point-implicit chemistry step (Eq. 4.12-4.13) over dt applied to every
// cell of F, followed by the Newton T of the new state warm-started from the
// old one.
template <class S> int chemistry_step(const Mech& m, const Grid& g, Field<S>& F, double dt) {
  int st = 0;
  Field<S> Un = F;
  #pragma omp parallel for schedule(static) reduction(| : st)
  for (int j = 0; j < F.ny; ++j)
    for (int i = 0; i < F.nx; ++i) {
      S u[16];
      for (int k = 0; k < F.nv; ++k) u[k] = F.u(k, i, j);
      int s = 0;
      point_implicit(m, u, F.t(i, j), dt, &s);
      for (int k = 0; k < F.nv; ++k) Un.u(k, i, j) = u[k];
      st |= s;
    }
  st |= update_T(m, g, Un, F);
  F = Un;
  return st;
}

// Splitting of the chemistry and flux operators within one step.
enum : int {
  CHEM_OFF = 0,       // flux terms only (the explicit variant without sources)
  CHEM_LIE = 1,       // flux(dt) then chemistry(dt): advance_one_step as coded in Sec. 4.3
  CHEM_STRANG = 2,    // chemistry(dt/2), flux(dt), chemistry(dt/2): the Strang
                      // splitting named in the text of Sec. 4.3
  CHEM_EXPLICIT = 3,  // no splitting: the production rates are a source term of
                      // the semi-discrete equation, advanced by the same TVD-RK3
                      // as the fluxes (the user source_terms path of Sec. 4.3)
};

// L += S(U): the mass production rates of the carried species (Eq. 4.7-4.9)
// at each cell's T, added to the rows rho Y_1 .. rho Y_{ns-1}.
template <class S> void add_sources(const Mech& m, const Field<S>& F, std::vector<S>& L) {
  const int ns = m.ns;
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < F.ny; ++j)
    for (int i = 0; i < F.nx; ++i) {
      S X[16], w[16];
      S rest = F.u(0, i, j);
      for (int k = 0; k < ns - 1; ++k) {
        X[k] = F.u(4 + k, i, j) / m.M[k];
        rest = rest - F.u(4 + k, i, j);
      }
      X[ns - 1] = rest / m.M[ns - 1];
      production_rates(m, F.t(i, j), X, w);
      for (int k = 0; k < ns - 1; ++k) {
        S& l = L[((size_t)(4 + k) * F.ny + j) * F.nx + i];
        l = l + w[k];
      }
    }
}

// One time step (advance_one_step of Sec. 4.3): TVD-RK3 of the flux terms
// (Shu-Osher form) and the point-implicit chemistry (Eq. 4.12-4.13) in the
// order given by chem (CHEM_*; a bool true means CHEM_LIE). dt is the step's
// (from the CFL of its starting state when the caller asks for it). F holds
// U^n and its T on entry and U^{n+1} and its T on exit.
template <class S> int advance_one_step(const Mech& m, const Grid& g, Field<S>& F, double dt, int chem) {
  const size_t N = F.U.size();
  int st = 0;
  const bool reacting = m.nr > 0 && m.ns > 1;
  if (chem == CHEM_STRANG && reacting) st |= chemistry_step(m, g, F, 0.5 * dt);
  std::vector<S> L;
  Field<S> U1 = F, U2 = F;
  const bool explicit_src = chem == CHEM_EXPLICIT && reacting;
  // stage 1: U1 = U^n + dt L(U^n)
  rhs(m, g, F, L);
  if (explicit_src) add_sources(m, F, L);
  for (size_t q = 0; q < N; ++q) U1.U[q] = F.U[q] + dt * L[q];
  st |= update_T(m, g, U1, F);
  // stage 2: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1))
  rhs(m, g, U1, L);
  if (explicit_src) add_sources(m, U1, L);
  for (size_t q = 0; q < N; ++q) U2.U[q] = 0.75 * F.U[q] + 0.25 * (U1.U[q] + dt * L[q]);
  st |= update_T(m, g, U2, U1);
  // stage 3: U* = 1/3 U^n + 2/3 (U2 + dt L(U2))
  rhs(m, g, U2, L);
  if (explicit_src) add_sources(m, U2, L);
  Field<S> Us = F;
  for (size_t q = 0; q < N; ++q) Us.U[q] = (1.0 / 3.0) * F.U[q] + (2.0 / 3.0) * (U2.U[q] + dt * L[q]);
  st |= update_T(m, g, Us, U2);
  if (chem == CHEM_LIE && reacting) st |= chemistry_step(m, g, Us, dt);
  if (chem == CHEM_STRANG && reacting) st |= chemistry_step(m, g, Us, 0.5 * dt);
  F = Us;
  st |= check_state(m, F);
  return st;
}

}  // namespace orc
