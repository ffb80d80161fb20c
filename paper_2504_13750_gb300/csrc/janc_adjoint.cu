// Discrete adjoint of the step (advance_one_step, Sec. 4.3 of arXiv
// 2504.13750): the transpose of everything the forward kernels compute, for
// gradients of a trajectory loss with respect to the initial state, with
// checkpoint-and-recompute over the trajectory.
//
//  * Right-hand side L(U) (Eq. 4.10-4.11, WENO5, ghost layers): the
//    vector-Jacobian product is taken face by face (the reverse of the
//    reconstruction formula for both split signs) into a face-contribution
//    buffer, then gathered per cell over the faces whose stencils touch it,
//    ghost images included and folded back with the wall flips; the chain
//    through u, v and p(T(U)) uses the implicit derivative of the Newton T
//    recovery. The global LF speeds alpha (Eq. 4.11) receive the summed
//    cotangent, which flows to the cell that attains the maximum (ties:
//    lowest linear index).
//  * Point-implicit chemistry (Eq. 4.12-4.13): the 12 x 12 local Jacobian of
//    the cell map U* -> U^{n+1} (through T* = T(U*), rates, Jacobian and the
//    LU solve) by forward-mode dual numbers, 4 lanes per pass, then its
//    transpose times the cotangent.
//  * TVD-RK3: the Shu-Osher stages reversed.
// No atomics touch state cotangents: every cell gathers its own.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/janc.h"
#include "janc_adjoint.cuh"
#include "janc_device.cuh"
#include "janc_internal.h"

namespace janc {

// ---------------------------------------------------------------------------
// RHS vector-Jacobian product.
// ---------------------------------------------------------------------------
constexpr int AF = 10;  // face contributions: 5 for F+, 5 for F-

// Face pass. Thread = (variable, face). mu: cotangent of L [nv][ny][nx].
// CF[k][face][10]: cotangents of the split fluxes at the stencil cells.
template <int NV>
__global__ void k_adj_faces(StateView S, const double* __restrict__ alpha2, const double* __restrict__ mu,
                            double* __restrict__ CF, GridDev g, int xdir) {
  const long long n = g.n;
  const int nx = g.nx, ny = g.ny;
  const int nfl = xdir ? nx + 1 : ny + 1;   // faces per line
  const int nlines = xdir ? ny : nx;
  const long long per_var = (long long)nfl * nlines;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= per_var * NV) return;
  const int k = (int)(q / per_var);
  const long long rem = q % per_var;
  int f, line;
  if (xdir) { line = (int)(rem / nfl); f = (int)(rem % nfl); }
  else { f = (int)(rem / nlines); line = (int)(rem % nlines); }
  const int ncell = xdir ? nx : ny;
  const int bc_lo = xdir ? g.bc[0] : g.bc[2], bc_hi = xdir ? g.bc[1] : g.bc[3];
  const int nmom = xdir ? 1 : 2;
  const double ha = 0.5 * alpha2[xdir ? 0 : 1];
  const double* Uk = S.plane(k, n);
  const double* up = S.plane(xdir ? NV + 1 : NV + 2, n);
  const double* pp = S.plane(NV + 3, n);
  double Fp[6], Fm[6];
#pragma unroll
  for (int w = 0; w < 6; ++w) {
    bool flip;
    const int src = ghost_src(f - 3 + w, ncell, bc_lo, bc_hi, flip);
    const long long idx = xdir ? (long long)line * nx + src : (long long)src * nx + line;
    double un = up[idx];
    if (flip) un = -un;
    double U = Uk[idx];
    if (flip && k == nmom) U = -U;
    const double hp = 0.5 * pp[idx];
    const double lp = fma(0.5, un, ha), lm = fma(0.5, un, -ha);
    if (k == nmom) { Fp[w] = fma(lp, U, hp); Fm[w] = fma(lm, U, hp); }
    else if (k == 3) { Fp[w] = fma(lp, U, hp * un); Fm[w] = fma(lm, U, hp * un); }
    else { Fp[w] = lp * U; Fm[w] = lm * U; }
  }
  // cotangent of the face flux: L(i) = -(F(i+1/2) - F(i-1/2)) / h
  const double rh = xdir ? g.rdx : g.rdy;
  auto mu_at = [&](int c) -> double {
    if (c < 0 || c >= ncell) return 0.0;
    const long long idx = xdir ? (long long)line * nx + c : (long long)c * nx + line;
    return mu[(long long)k * n + idx];
  };
  const double phi = rh * (mu_at(f) - mu_at(f - 1));
  double* out = CF + ((long long)k * per_var + (xdir ? (long long)line * nfl + f : (long long)f * nlines + line)) * AF;
  double gp[5], gm[5];
  weno_face_vjp<false>(Fp, g.eps4, phi, gp);   // window cells f-3 .. f+1
  weno_face_vjp<true>(Fm + 1, g.eps4, phi, gm);  // window cells f-2 .. f+2
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    out[m] = gp[m];
    out[5 + m] = gm[m];
  }
}

// Cell pass: cotangents of U, u_n and p of cell c from the faces, with the
// ghost positions that copy cell c folded back. Returns via references.
template <int NV>
__device__ __forceinline__ void gather_dir(const StateView& S, const double* __restrict__ CF, const GridDev& g,
                                           double ha, int xdir, int i, int j, double* aU, double& a_un, double& a_p,
                                           double& a_alpha) {
  const long long n = g.n;
  const int nx = g.nx, ny = g.ny;
  const int nfl = xdir ? nx + 1 : ny + 1;
  const int nlines = xdir ? ny : nx;
  const long long per_var = (long long)nfl * nlines;
  const int ncell = xdir ? nx : ny;
  const int c = xdir ? i : j;
  const int line = xdir ? j : i;
  const int bc_lo = xdir ? g.bc[0] : g.bc[2], bc_hi = xdir ? g.bc[1] : g.bc[3];
  const int nmom = xdir ? 1 : 2;
  const long long idx = (long long)j * nx + i;
  const double un0 = S.plane(xdir ? NV + 1 : NV + 2, n)[idx];
  const double hp = 0.5 * S.plane(NV + 3, n)[idx];
  double Uc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) Uc[k] = S.plane(k, n)[idx];
  // positions that read cell c: c itself and the ghost images that map to it
  int pos[7];
  bool fl[7];
  int np = 0;
  pos[np] = c; fl[np++] = false;
  for (int e = -3; e <= -1; ++e) {
    bool flip;
    if (ghost_src(e, ncell, bc_lo, bc_hi, flip) == c) { pos[np] = e; fl[np++] = flip; }
  }
  for (int e = ncell; e <= ncell + 2; ++e) {
    bool flip;
    if (ghost_src(e, ncell, bc_lo, bc_hi, flip) == c) { pos[np] = e; fl[np++] = flip; }
  }
  for (int t = 0; t < np; ++t) {
    const int e = pos[t];
    const bool flip = fl[t];
    const double un = flip ? -un0 : un0;
    const double lp = fma(0.5, un, ha), lm = fma(0.5, un, -ha);
    double aLp = 0.0, aLm = 0.0, a_hp = 0.0, a_hpu = 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double U = (flip && k == nmom) ? -Uc[k] : Uc[k];
      double fp = 0.0, fm = 0.0;
      for (int f = e - 1; f <= e + 3; ++f) {
        if (f < 0 || f >= nfl) continue;
        fp += CF[((long long)k * per_var + (xdir ? (long long)line * nfl + f : (long long)f * nlines + line)) * AF +
                 (e - f + 3)];
      }
      for (int f = e - 2; f <= e + 2; ++f) {
        if (f < 0 || f >= nfl) continue;
        fm += CF[((long long)k * per_var + (xdir ? (long long)line * nfl + f : (long long)f * nlines + line)) * AF +
                 5 + (e - f + 2)];
      }
      const double aUk = lp * fp + lm * fm;
      aU[k] += (flip && k == nmom) ? -aUk : aUk;
      aLp = fma(U, fp, aLp);
      aLm = fma(U, fm, aLm);
      if (k == nmom) a_hp += fp + fm;
      if (k == 3) a_hpu += fp + fm;
    }
    // F+- = lambda+- U (+ hp on the normal momentum, + hp u_n on the energy)
    const double a_un_e = 0.5 * (aLp + aLm) + hp * a_hpu;
    a_alpha += 0.5 * (aLp - aLm);
    a_p += 0.5 * (a_hp + un * a_hpu);
    a_un += flip ? -a_un_e : a_un_e;
  }
}

template <int NS>
__global__ void k_adj_cells(StateView S, const double* __restrict__ alpha2, const double* __restrict__ CFx,
                            const double* __restrict__ CFy, double* __restrict__ nu, double* adj_alpha, GridDev g,
                            const MechDev* __restrict__ mech) {
  constexpr int NV = NS + 3;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double ax = 0.0, ay = 0.0;
  if (i < g.nx && j < g.ny) {
    const long long n = g.n;
    const long long idx = (long long)j * g.nx + i;
    double aU[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) aU[k] = 0.0;
    double a_u = 0.0, a_v = 0.0, a_p = 0.0;
    gather_dir<NV>(S, CFx, g, 0.5 * alpha2[0], 1, i, j, aU, a_u, a_p, ax);
    gather_dir<NV>(S, CFy, g, 0.5 * alpha2[1], 0, i, j, aU, a_v, a_p, ay);
    double u[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[idx];
    const double T = S.plane(NV, n)[idx];
    const double rrho = 1.0 / u[0];
    const double vx = u[1] * rrho, vy = u[2] * rrho;
    CellThermo<NS> ct;
    cell_thermo<NS>(u, T, *mech, ct);
    double dT[NV], dp[NV];
    dT_dp_dU<NS>(u, T, *mech, ct, dT, dp);
    aU[0] += -(vx * a_u + vy * a_v) * rrho;
    aU[1] += a_u * rrho;
    aU[2] += a_v * rrho;
#pragma unroll
    for (int k = 0; k < NV; ++k) nu[(long long)k * n + idx] = fma(dp[k], a_p, aU[k]);
  }
  // block sums of the alpha cotangents
  __shared__ double rx[256], ry[256];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  rx[tid] = ax;
  ry[tid] = ay;
  __syncthreads();
  for (int s = blockDim.x * blockDim.y / 2; s > 0; s >>= 1) {
    if (tid < s) { rx[tid] += rx[tid + s]; ry[tid] += ry[tid + s]; }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(adj_alpha, rx[0]);
    atomicAdd(adj_alpha + 1, ry[0]);
  }
}

// Arg-max of |u|+c (d = 0) and |v|+c (d = 1) over the cells; ties go to the
// lowest linear index. pass 0: max bits; pass 1: lowest index with the max.
template <int NS>
__global__ void k_speed_argmax(StateView S, GridDev g, const MechDev* __restrict__ mech, unsigned long long* mx,
                               int* idx_out, int pass) {
  constexpr int NV = NS + 3;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.n) return;
  const long long n = g.n;
  double u[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[q];
  const double c = sound_speed<NS>(u, S.plane(NV, n)[q], *mech);
  const double rr = rcp(u[0]);
  const unsigned long long sx = dbits(dabs(u[1] * rr) + c), sy = dbits(dabs(u[2] * rr) + c);
  if (pass == 0) {
    atomicMax(mx, sx);
    atomicMax(mx + 1, sy);
  } else {
    if (sx == mx[0]) atomicMin(idx_out, (int)q);
    if (sy == mx[1]) atomicMin(idx_out + 1, (int)q);
  }
}

// The alpha cotangents flow to the arg-max cells: d(|u_d| + c)/dU.
template <int NS>
__global__ void k_adj_alpha(StateView S, GridDev g, const MechDev* __restrict__ mech, const int* idx,
                            const double* adj_alpha, double* nu) {
  constexpr int NV = NS + 3;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const long long n = g.n;
  for (int d = 0; d < 2; ++d) {
    const int cidx = idx[d];
    if (cidx < 0 || cidx >= g.n) continue;
    const double a = adj_alpha[d];
    double u[NV];
    for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[cidx];
    const double T = S.plane(NV, n)[cidx];
    const MechDev& m = *mech;
    CellThermo<NS> ct;
    cell_thermo<NS>(u, T, m, ct);
    double dT[NV], dp[NV];
    dT_dp_dU<NS>(u, T, m, ct, dT, dp);
    const double rho = u[0];
    const double p = RU * ct.W * T;
    const double Cv = ct.Cv, Cp = ct.Cv + ct.W;
    const double c = sqrt(Cp * p / (Cv * rho));
    const double vel = u[1 + d] / rho;
    const double sgn = vel < 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < NV; ++k) {
      // dz-weighted cv sums for dCv/dU
      double dz_cv = 0.0, dW = 0.0;
      if (k == 0) { dz_cv = ct.cvR[NS - 1] * m.invM[NS - 1]; dW = m.invM[NS - 1]; }
      else if (k >= 4) {
        dz_cv = ct.cvR[k - 4] * m.invM[k - 4] - ct.cvR[NS - 1] * m.invM[NS - 1];
        dW = m.invM[k - 4] - m.invM[NS - 1];
      }
      const double dCv = dz_cv + ct.dCv * dT[k];
      const double dCp = dCv + dW;
      const double drho = k == 0 ? 1.0 : 0.0;
      const double dc = 0.5 * c * (dCp / Cp + dp[k] / p - dCv / Cv - drho / rho);
      double dvel = 0.0;
      if (k == 0) dvel = -vel / rho;
      if (k == 1 + d) dvel = 1.0 / rho;
      nu[(long long)k * n + cidx] += a * (sgn * dvel + dc);
    }
  }
}

// ---------------------------------------------------------------------------
// Chemistry: forward-mode duals with L lanes.
// ---------------------------------------------------------------------------
template <int L>
struct Dn {
  double v;
  double d[L];
};
template <int L> __device__ __forceinline__ Dn<L> dconst(double x) {
  Dn<L> r; r.v = x;
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = 0.0;
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> dadd(const Dn<L>& a, const Dn<L>& b) {
  Dn<L> r; r.v = a.v + b.v;
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = a.d[l] + b.d[l];
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> dsub(const Dn<L>& a, const Dn<L>& b) {
  Dn<L> r; r.v = a.v - b.v;
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = a.d[l] - b.d[l];
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> dmul(const Dn<L>& a, const Dn<L>& b) {
  Dn<L> r; r.v = a.v * b.v;
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = fma(a.d[l], b.v, a.v * b.d[l]);
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> dscale(const Dn<L>& a, double s) {
  Dn<L> r; r.v = a.v * s;
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = a.d[l] * s;
  return r;
}
// a * b + c
template <int L> __device__ __forceinline__ Dn<L> dfma(const Dn<L>& a, const Dn<L>& b, const Dn<L>& c) {
  Dn<L> r; r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = fma(a.d[l], b.v, fma(a.v, b.d[l], c.d[l]));
  return r;
}
// s * a + c with a double s
template <int L> __device__ __forceinline__ Dn<L> dsfma(double s, const Dn<L>& a, const Dn<L>& c) {
  Dn<L> r; r.v = fma(s, a.v, c.v);
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = fma(s, a.d[l], c.d[l]);
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> drcp(const Dn<L>& a) {
  Dn<L> r; r.v = rcp(a.v);
  const double q = -r.v * r.v;
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = q * a.d[l];
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> dexp(const Dn<L>& a) {
  Dn<L> r; r.v = exp_t(a.v);
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = r.v * a.d[l];
  return r;
}
template <int L> __device__ __forceinline__ Dn<L> dlog(const Dn<L>& a) {
  Dn<L> r; r.v = log(a.v);
  const double q = rcp(a.v);
#pragma unroll
  for (int l = 0; l < L; ++l) r.d[l] = q * a.d[l];
  return r;
}

// Cotangent of U* from the cotangent of U^{n+1} for one cell, lanes
// [lane0, lane0 + L) of the input. The map: T* = T(U*) (Newton, from the
// stored value), then the point-implicit update of the species.
template <int NS, int L>
__device__ void chem_vjp_lanes(const double* uval, double Tval, const MechDev& m, double dt, const double* lam,
                               int lane0, double* out) {
  constexpr int NSP = NS - 1;
  constexpr int NV = NS + 3;
  Dn<L> u[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    u[k] = dconst<L>(uval[k]);
#pragma unroll
    for (int l = 0; l < L; ++l) u[k].d[l] = (k == lane0 + l) ? 1.0 : 0.0;
  }
  // Newton T on duals from the converged value (the value part stays put,
  // the tangent part becomes the implicit derivative).
  Dn<L> z[NS];
  Dn<L> rest = u[0];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    z[k] = dscale<L>(u[4 + k], m.invM[k]);
    rest = dsub<L>(rest, u[4 + k]);
  }
  z[NSP] = dscale<L>(rest, m.invM[NSP]);
  Dn<L> W = z[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) W = dadd<L>(W, z[k]);
  Dn<L> h[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    Dn<L> s = dscale<L>(z[0], m.hc[0][q]);
#pragma unroll
    for (int k = 1; k < NS; ++k) s = dsfma<L>(m.hc[k][q], z[k], s);
    h[q] = s;
  }
  const Dn<L> rrho = drcp<L>(u[0]);
  const Dn<L> ke = dfma<L>(u[1], u[1], dmul<L>(u[2], u[2]));
  const Dn<L> rhoe = dsub<L>(u[3], dscale<L>(dmul<L>(rrho, ke), 0.5));
  const Dn<L> K0 = dsub<L>(h[5], dscale<L>(rhoe, 1.0 / RU));
  const Dn<L> K1 = dsub<L>(h[0], W);
  Dn<L> T = dconst<L>(Tval);
  for (int it = 0; it < 2; ++it) {
    Dn<L> F = dfma<L>(T, h[4], h[3]);
    F = dfma<L>(T, F, h[2]);
    F = dfma<L>(T, F, h[1]);
    F = dfma<L>(T, F, K1);
    F = dfma<L>(T, F, K0);
    Dn<L> Fp = dfma<L>(T, dscale<L>(h[4], 5.0), dscale<L>(h[3], 4.0));
    Fp = dfma<L>(T, Fp, dscale<L>(h[2], 3.0));
    Fp = dfma<L>(T, Fp, dscale<L>(h[1], 2.0));
    Fp = dfma<L>(T, Fp, K1);
    T = dsub<L>(T, dmul<L>(F, drcp<L>(Fp)));
  }
  // rates (Eq. 4.7-4.9) on duals
  Dn<L> X[NS];
#pragma unroll
  for (int k = 0; k < NSP; ++k) X[k] = dscale<L>(u[4 + k], m.invM[k]);
  X[NSP] = z[NSP];
  Dn<L> Ctot = X[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) Ctot = dadd<L>(Ctot, X[k]);
  const Dn<L> lnT = dlog<L>(T);
  const Dn<L> rT = drcp<L>(T);
  Dn<L> eG[NS], reG[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* c = m.gc[k];
    Dn<L> G = dsfma<L>(c[4], T, dconst<L>(c[3]));
    G = dfma<L>(T, G, dconst<L>(c[2]));
    G = dfma<L>(T, G, dconst<L>(c[1]));
    G = dfma<L>(T, G, dconst<L>(c[6]));
    G = dsfma<L>(c[5], rT, G);
    G = dsfma<L>(c[0], lnT, G);
    eG[k] = dexp<L>(G);
    reG[k] = drcp<L>(eG[k]);
  }
  const Dn<L> cref = dscale<L>(rT, P_REF / RU);
  const Dn<L> rcref = dscale<L>(T, RU / P_REF);
  Dn<L> wd[NSP];
  Dn<L> J[NSP][NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    wd[k] = dconst<L>(0.0);
#pragma unroll
    for (int l = 0; l < NSP; ++l) J[k][l] = dconst<L>(0.0);
  }
  for (int i = 0; i < m.nr; ++i) {
    const int nre = m.nre[i], npr = m.npr[i];
    const Dn<L> kf = dexp<L>(dsfma<L>(m.b[i], lnT, dsfma<L>(-m.EaR[i], rT, dconst<L>(m.lnA[i]))));
    Dn<L> kb = kf;
    for (int r = 0; r < nre; ++r)
      for (int q = 0; q < m.rnu[i][r]; ++q) kb = dmul<L>(kb, eG[m.rsp[i][r]]);
    for (int r = 0; r < npr; ++r)
      for (int q = 0; q < m.pnu[i][r]; ++q) kb = dmul<L>(kb, reG[m.psp[i][r]]);
    for (int q = 0; q < m.dnu[i]; ++q) kb = dmul<L>(kb, rcref);
    for (int q = 0; q < -m.dnu[i]; ++q) kb = dmul<L>(kb, cref);
    Dn<L> xr[MAX_SIDE], xp[MAX_SIDE];
    Dn<L> fwd = kf, bwd = kb;
    for (int r = 0; r < nre; ++r) {
      xr[r] = X[m.rsp[i][r]];
      for (int q = 0; q < m.rnu[i][r]; ++q) fwd = dmul<L>(fwd, xr[r]);
    }
    for (int r = 0; r < npr; ++r) {
      xp[r] = X[m.psp[i][r]];
      for (int q = 0; q < m.pnu[i][r]; ++q) bwd = dmul<L>(bwd, xp[r]);
    }
    Dn<L> Mi = dconst<L>(1.0);
    if (m.tb[i]) {
      Mi = Ctot;
      for (int e = 0; e < m.neff[i]; ++e) Mi = dsfma<L>(m.effv[i][e], X[m.effsp[i][e]], Mi);
    }
    const Dn<L> net = dsub<L>(fwd, bwd);
    const Dn<L> q = dmul<L>(Mi, net);
    for (int r = 0; r < nre; ++r) {
      const int k = m.rsp[i][r];
      if (k < NSP) wd[k] = dsfma<L>(-m.rnud[i][r], q, wd[k]);
    }
    for (int r = 0; r < npr; ++r) {
      const int k = m.psp[i][r];
      if (k < NSP) wd[k] = dsfma<L>(m.pnud[i][r], q, wd[k]);
    }
    Dn<L> dq[2 * MAX_SIDE];
    int dsp[2 * MAX_SIDE];
    int nd = 0;
    for (int r = 0; r < nre; ++r) {
      Dn<L> dd = dscale<L>(kf, m.rnud[i][r]);
      for (int s = 0; s < nre; ++s) {
        const int pw = m.rnu[i][s] - (s == r ? 1 : 0);
        for (int t = 0; t < pw; ++t) dd = dmul<L>(dd, xr[s]);
      }
      dq[nd] = dmul<L>(Mi, dd);
      dsp[nd++] = m.rsp[i][r];
    }
    for (int r = 0; r < npr; ++r) {
      Dn<L> dd = dscale<L>(kb, m.pnud[i][r]);
      for (int s = 0; s < npr; ++s) {
        const int pw = m.pnu[i][s] - (s == r ? 1 : 0);
        for (int t = 0; t < pw; ++t) dd = dmul<L>(dd, xp[s]);
      }
      dq[nd] = dscale<L>(dmul<L>(Mi, dd), -1.0);
      dsp[nd++] = m.psp[i][r];
    }
    for (int side = 0; side < 2; ++side) {
      const int cnt = side ? npr : nre;
      for (int r = 0; r < cnt; ++r) {
        const int k = side ? m.psp[i][r] : m.rsp[i][r];
        if (k >= NSP) continue;
        const double nu = side ? m.pnud[i][r] : -m.rnud[i][r];
        for (int d = 0; d < nd; ++d) {
          const int jj = dsp[d];
          if (jj < NSP) {
            J[k][jj] = dsfma<L>(nu, dq[d], J[k][jj]);
          } else {
            const Dn<L> v = dscale<L>(dq[d], nu);
            for (int l = 0; l < NSP; ++l) J[k][l] = dsfma<L>(-m.mratio[l], v, J[k][l]);
          }
        }
        if (m.tb[i]) {
          const Dn<L> v = dscale<L>(net, nu);
          for (int l = 0; l < NSP; ++l) J[k][l] = dsfma<L>(m.ceff[i][l], v, J[k][l]);
        }
      }
    }
  }
  // (I - dt J) dx = dt wd, LU with partial pivoting on the values
  Dn<L> b[NSP];
  for (int k = 0; k < NSP; ++k) {
    b[k] = dscale<L>(wd[k], dt);
    for (int l = 0; l < NSP; ++l) {
      J[k][l] = dscale<L>(J[k][l], -dt);
      if (k == l) J[k][l].v += 1.0;
    }
  }
  for (int c = 0; c < NSP; ++c) {
    int piv = c;
    double best = fabs(J[c][c].v);
    for (int r = c + 1; r < NSP; ++r)
      if (fabs(J[r][c].v) > best) { best = fabs(J[r][c].v); piv = r; }
    if (piv != c) {
      for (int k = 0; k < NSP; ++k) { Dn<L> t = J[c][k]; J[c][k] = J[piv][k]; J[piv][k] = t; }
      Dn<L> t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    const Dn<L> ip = drcp<L>(J[c][c]);
    for (int r = c + 1; r < NSP; ++r) {
      const Dn<L> f = dmul<L>(J[r][c], ip);
      for (int k = c + 1; k < NSP; ++k) J[r][k] = dsub<L>(J[r][k], dmul<L>(f, J[c][k]));
      b[r] = dsub<L>(b[r], dmul<L>(f, b[c]));
    }
  }
  for (int r = NSP - 1; r >= 0; --r) {
    Dn<L> s = b[r];
    for (int k = r + 1; k < NSP; ++k) s = dsub<L>(s, dmul<L>(J[r][k], b[k]));
    b[r] = dmul<L>(s, drcp<L>(J[r][r]));
  }
  // d(U^{n+1})/d(U*_lane) = identity + d(M_k dx_k) on the species rows
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const int lane = lane0 + l;
    if (lane >= NV) continue;
    double s = lam[lane];
    for (int k = 0; k < NSP; ++k) s = fma(lam[4 + k], m.M[k] * b[k].d[l], s);
    out[lane] = s;
  }
}

constexpr int CHEM_L = 4;

template <int NS>
__global__ void k_adj_chem(StateView Sstar, GridDev g, const MechDev* __restrict__ mech, double dt,
                           const double* __restrict__ lam, double* __restrict__ out, int lane0) {
  constexpr int NV = NS + 3;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.n) return;
  const long long n = g.n;
  double u[NV], l[NV], o[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    u[k] = Sstar.plane(k, n)[q];
    l[k] = lam[(long long)k * n + q];
    o[k] = 0.0;
  }
  chem_vjp_lanes<NS, CHEM_L>(u, Sstar.plane(NV, n)[q], *mech, dt, l, lane0, o);
  for (int k = lane0; k < lane0 + CHEM_L && k < NV; ++k) out[(long long)k * n + q] = o[k];
}

// ---------------------------------------------------------------------------
// Small kernels: linear combinations, loss terms, primitive T derivative.
// ---------------------------------------------------------------------------
// out = a x + b y (y may be null)
__global__ void k_lincomb(long long count, double* out, double a, const double* x, double b, const double* y) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double v = a * x[q];
  if (y) v = fma(b, y[q], v);
  out[q] = v;
}
// out += a x + b y (y may be null)
__global__ void k_lincomb_acc(long long count, double* out, double a, const double* x, double b, const double* y) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double v = fma(a, x[q], out[q]);
  if (y) v = fma(b, y[q], v);
  out[q] = v;
}

// loss += w * sum_j p(nx-1, j) (one block)
template <int NS>
__global__ void k_loss_endwall(StateView S, GridDev g, double w, double* loss) {
  constexpr int NV = NS + 3;
  __shared__ double red[256];
  double s = 0.0;
  for (int j = threadIdx.x; j < g.ny; j += blockDim.x) s += S.plane(NV + 3, g.n)[(long long)j * g.nx + g.nx - 1];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] += w * red[0];
}

// lam += w dp/dU at the end-wall cells (nx-1, j)
template <int NS>
__global__ void k_seed_endwall(StateView S, GridDev g, const MechDev* __restrict__ mech, double w, double* lam) {
  constexpr int NV = NS + 3;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.ny) return;
  const long long n = g.n;
  const long long idx = (long long)j * g.nx + g.nx - 1;
  double u[NV];
  for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[idx];
  const double T = S.plane(NV, n)[idx];
  CellThermo<NS> ct;
  cell_thermo<NS>(u, T, *mech, ct);
  double dT[NV], dp[NV];
  dT_dp_dU<NS>(u, T, *mech, ct, dT, dp);
  for (int k = 0; k < NV; ++k) lam[(long long)k * n + idx] += w * dp[k];
}

// loss = sum seed * U (one block per 256-chunk, atomic sum)
__global__ void k_dot(long long count, const double* a, const double* b, double* out) {
  __shared__ double red[256];
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  red[threadIdx.x] = q < count ? a[q] * b[q] : 0.0;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// dL/dT of the primitive initialisation U(T, p, u, v, Y) (Eq. 4.2) at fixed
// p, u, v, Y: rho = p/(R T), E = rho h - p + rho |u|^2/2, rho Y_k.
template <int NS>
__global__ void k_prim_T_vjp(const double* __restrict__ T, const double* __restrict__ p,
                             const double* __restrict__ vx, const double* __restrict__ vy,
                             const double* __restrict__ Y, const double* __restrict__ dLdU, double* __restrict__ out,
                             GridDev g, const MechDev* __restrict__ mech) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.n) return;
  const long long n = g.n;
  const MechDev& m = *mech;
  const double t = T[q];
  double Wm = 0.0, h = 0.0, cp = 0.0;  // per mass / Ru
  double Yk[NS];
  for (int k = 0; k < NS; ++k) {
    Yk[k] = Y[(long long)k * n + q];
    const double* c = m.hc[k];
    const double hk = fma(t, fma(t, fma(t, fma(t, fma(t, c[4], c[3]), c[2]), c[1]), c[0]), c[5]);
    const double cpk = fma(t, fma(t, fma(t, fma(t, 5.0 * c[4], 4.0 * c[3]), 3.0 * c[2]), 2.0 * c[1]), c[0]);
    Wm += Yk[k] * m.invM[k];
    h += Yk[k] * m.invM[k] * hk;
    cp += Yk[k] * m.invM[k] * cpk;
  }
  const double rho = p[q] / (RU * Wm * t);
  const double drho = -rho / t;
  const double ke = 0.5 * (vx[q] * vx[q] + vy[q] * vy[q]);
  double s = dLdU[q] * drho + dLdU[n + q] * vx[q] * drho + dLdU[2 * n + q] * vy[q] * drho;
  s += dLdU[3 * n + q] * (drho * (RU * h + ke) + rho * RU * cp);
  for (int k = 0; k < NS - 1; ++k) s += dLdU[(long long)(4 + k) * n + q] * Yk[k] * drho;
  out[q] = s;
}

// ---------------------------------------------------------------------------
// Launch helpers.
// ---------------------------------------------------------------------------
static unsigned nblk(long long count, int thr) { return (unsigned)((count + thr - 1) / thr); }

template <int NS>
static cudaError_t rhs_vjp_t(const StateView& S, const double* alpha2_dev, const double* mu, double* nu, double* CFx,
                             double* CFy, double* scratch /* 2 doubles + 2 u64 + 2 int */, const GridDev& g,
                             const MechDev* mech, cudaStream_t st) {
  constexpr int NV = NS + 3;
  double* adj_alpha = scratch;
  unsigned long long* mx = (unsigned long long*)(scratch + 2);
  int* idx = (int*)(scratch + 4);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 4 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(idx, 0x7f, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long fx = (long long)NV * g.ny * (g.nx + 1), fy = (long long)NV * (g.ny + 1) * g.nx;
  k_adj_faces<NV><<<nblk(fx, 128), 128, 0, st>>>(S, alpha2_dev, mu, CFx, g, 1);
  k_adj_faces<NV><<<nblk(fy, 128), 128, 0, st>>>(S, alpha2_dev, mu, CFy, g, 0);
  dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  k_adj_cells<NS><<<grd, blk, 0, st>>>(S, alpha2_dev, CFx, CFy, nu, adj_alpha, g, mech);
  k_speed_argmax<NS><<<nblk(g.n, 256), 256, 0, st>>>(S, g, mech, mx, idx, 0);
  k_speed_argmax<NS><<<nblk(g.n, 256), 256, 0, st>>>(S, g, mech, mx, idx, 1);
  k_adj_alpha<NS><<<1, 32, 0, st>>>(S, g, mech, idx, adj_alpha, nu);
  return cudaGetLastError();
}

cudaError_t launch_rhs_vjp(int ns, const StateView& S, const double* alpha2_dev, const double* mu, double* nu,
                           double* CFx, double* CFy, double* scratch, const GridDev& g, const MechDev* mech,
                           cudaStream_t st) {
  switch (ns) {
    case 1: return rhs_vjp_t<1>(S, alpha2_dev, mu, nu, CFx, CFy, scratch, g, mech, st);
    case 3: return rhs_vjp_t<3>(S, alpha2_dev, mu, nu, CFx, CFy, scratch, g, mech, st);
    case 9: return rhs_vjp_t<9>(S, alpha2_dev, mu, nu, CFx, CFy, scratch, g, mech, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chem_vjp(int ns, const StateView& Sstar, const GridDev& g, const MechDev* mech, double dt,
                            const double* lam, double* out, cudaStream_t st) {
  const int nv = ns + 3;
  for (int lane0 = 0; lane0 < nv; lane0 += CHEM_L) {
    switch (ns) {
      case 3: k_adj_chem<3><<<nblk(g.n, 64), 64, 0, st>>>(Sstar, g, mech, dt, lam, out, lane0); break;
      case 9: k_adj_chem<9><<<nblk(g.n, 64), 64, 0, st>>>(Sstar, g, mech, dt, lam, out, lane0); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_lincomb(long long count, double* out, double a, const double* x, double b, const double* y,
                           bool accumulate, cudaStream_t st) {
  if (accumulate) k_lincomb_acc<<<nblk(count, 256), 256, 0, st>>>(count, out, a, x, b, y);
  else k_lincomb<<<nblk(count, 256), 256, 0, st>>>(count, out, a, x, b, y);
  return cudaGetLastError();
}

cudaError_t launch_loss_endwall(int ns, const StateView& S, const GridDev& g, double w, double* loss,
                                cudaStream_t st) {
  switch (ns) {
    case 1: k_loss_endwall<1><<<1, 256, 0, st>>>(S, g, w, loss); break;
    case 3: k_loss_endwall<3><<<1, 256, 0, st>>>(S, g, w, loss); break;
    case 9: k_loss_endwall<9><<<1, 256, 0, st>>>(S, g, w, loss); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_seed_endwall(int ns, const StateView& S, const GridDev& g, const MechDev* mech, double w,
                                double* lam, cudaStream_t st) {
  switch (ns) {
    case 1: k_seed_endwall<1><<<nblk(g.ny, 128), 128, 0, st>>>(S, g, mech, w, lam); break;
    case 3: k_seed_endwall<3><<<nblk(g.ny, 128), 128, 0, st>>>(S, g, mech, w, lam); break;
    case 9: k_seed_endwall<9><<<nblk(g.ny, 128), 128, 0, st>>>(S, g, mech, w, lam); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_dot(long long count, const double* a, const double* b, double* out, cudaStream_t st) {
  k_dot<<<nblk(count, 256), 256, 0, st>>>(count, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_prim_T_vjp(int ns, const double* T, const double* p, const double* u, const double* v,
                              const double* Y, const double* dLdU, double* out, const GridDev& g,
                              const MechDev* mech, cudaStream_t st) {
  switch (ns) {
    case 1: k_prim_T_vjp<1><<<nblk(g.n, 256), 256, 0, st>>>(T, p, u, v, Y, dLdU, out, g, mech); break;
    case 3: k_prim_T_vjp<3><<<nblk(g.n, 256), 256, 0, st>>>(T, p, u, v, Y, dLdU, out, g, mech); break;
    case 9: k_prim_T_vjp<9><<<nblk(g.n, 256), 256, 0, st>>>(T, p, u, v, Y, dLdU, out, g, mech); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace janc
