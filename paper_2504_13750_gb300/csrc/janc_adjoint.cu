// Discrete adjoint of the step (advance_one_step, Sec. 4.3 of arXiv
// 2504.13750): the transpose of everything the forward kernels compute, for
// gradients of a trajectory loss with respect to the initial state, with
// checkpoint-and-recompute over the trajectory.
//
//  * Right-hand side L(U) (Eq. 4.10-4.11, WENO5, ghost layers): the
//    vector-Jacobian product takes the derivative of both split signs'
//    reconstructions with respect to their window differences face by face
//    (formed here, or kept by the forward in the face-derivative store), in
//    tiles that slide along grid lines like the forward kernel, and sums the
//    split-flux cotangents per stencil position (ghost positions included);
//    each cell then reads the sums of its own position and of the ghost
//    images that copy it, folded back with the wall flips. The chain through u, v and p(T(U)) uses the implicit
//    derivative of the Newton T recovery. The global LF speeds alpha
//    (Eq. 4.11) receive the summed cotangent, which flows to the cell that
//    attains the maximum (ties: lowest linear index).
//  * Point-implicit chemistry (Eq. 4.12-4.13): one transposed solve with the
//    LU factors of the forward system, then the gradient of a scalar
//    (sum over reactions of the weighted rate and its derivative along the
//    solution) in reverse mode, chained through T* = T(U*) (see
//    chem_vjp_rev; chem_vjp_stored starts from the factors the forward kept).
//  * TVD-RK3: the Shu-Osher stages reversed; each stage's RHS VJP writes the
//    stage's linear combinations of the cotangents itself.
// No atomics touch state cotangents: every cell gathers its own. (The
// per-position split-flux sums take at most two atomic additions per slot
// onto zero, whose result does not depend on their order.)
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/janc.h"
#include "janc_adjoint.cuh"
#include "janc_device.cuh"
#include "janc_internal.h"
#include "janc_mech_policy.cuh"
#include "janc_weno.cuh"

namespace janc {

// ---------------------------------------------------------------------------
// RHS vector-Jacobian product.
// ---------------------------------------------------------------------------
// Face pass, tiled like the forward face-flux kernel. A block takes
// VLINES grid lines by VFACES (16, or 8 on small grids) consecutive faces
// along them (x tiles first, then y tiles) and stages the cotangent mu of L
// for them; every thread owns one (variable, line) and walks its faces. At
// face t, L_i = -(F_{i+1/2} - F_{i-1/2}) / h gives the face value the
// cotangent phi = (mu_i - mu_{i-1}) / h, and each of the two reconstructions
// W (F+ and F-) passes it on as phi dW/dF_j to the five split-flux values of
// its window.
//
// dW/dF_j comes from the partials with respect to the window differences
// D_m = F_m - F_{m-1} (weno_face_dD) plus the centre F2's weight one. The
// walk sums phi dW/dD_m per difference ("edge" q between positions q-1 and
// q), and a position's sum is complete once the faces have passed both of
// its edges: edge q minus edge q+1 plus the phi of the face whose window it
// centres. Each complete position, ghost positions -3 .. ncell + 2 included,
// is added to GF (zeroed beforehand): position e of a line holds
// (dL/dF+_e, dL/dF-_e); GF layout x faces [k][j][i + 3][2], y faces
// [k][j + 3][i][2]. A position is touched by the faces of at most two tiles,
// so each slot receives at most two additions onto zero, whose result does
// not depend on their order.
//
// Two forms: k_adj_faces recomputes the reconstructions from the staged
// cells; k_adj_faces_lin reads the derivatives the forward stored
// (launch_face_flux_lin) and only forms the sums.
constexpr int VLINES = 8;

// The per-position sums of one (variable, line) as its faces pass.
struct EdgeSums {
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;  // F+ edges t+1 .. t+4 at face t
  double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;  // F- edges t+2 .. t+5
  double pp = 0.0, pm = 0.0;                      // the last completed F+ / F- edge (t, t+1)
  double ph1 = 0.0, ph2 = 0.0;                    // phi of faces t-1 and t-2
  // After face t's partials are in: positions t (F+) and t+1 (F-) are
  // complete; add them to slot pair `s` (+0) and the next pair (+1).
  __device__ __forceinline__ void finish_face(double phi, double* gs, long long pstride) {
    atomicAdd(gs, (pp - p0) + ph2);
    atomicAdd(gs + pstride + 1, (pm - m0) + ph2);
    pp = p0; p0 = p1; p1 = p2; p2 = p3; p3 = 0.0;
    pm = m0; m0 = m1; m1 = m2; m2 = m3; m3 = 0.0;
    ph2 = ph1; ph1 = phi;
  }
  // After the tile's last face (nf faces): positions nf .. nf+3 (F+) and
  // nf+1 .. nf+4 (F-), starting at slot pair `s` of position nf.
  __device__ __forceinline__ void flush(double* gs, long long pstride) {
    atomicAdd(gs, (pp - p0) + ph2);
    atomicAdd(gs + pstride, (p0 - p1) + ph1);
    atomicAdd(gs + 2 * pstride, p1 - p2);
    atomicAdd(gs + 3 * pstride, p2);
    atomicAdd(gs + pstride + 1, (pm - m0) + ph2);
    atomicAdd(gs + 2 * pstride + 1, (m0 - m1) + ph1);
    atomicAdd(gs + 3 * pstride + 1, m1 - m2);
    atomicAdd(gs + 4 * pstride + 1, m2);
  }
};

// Tile geometry shared by both face-pass forms.
struct VjpTile {
  bool xdir;
  int f0, l0, nlines, nfaces, ncell, bc_lo, bc_hi, nmom;
  __device__ __forceinline__ VjpTile(const GridDev& g, int blk, int nbx, int ntx_x, int ntx_y, int vfaces) {
    xdir = blk < nbx;
    const int tile = xdir ? blk : blk - nbx;
    const int ntl = xdir ? ntx_x : ntx_y;
    const int ta = tile % ntl, tb = tile / ntl;
    f0 = xdir ? ta * vfaces : tb * vfaces;
    l0 = xdir ? tb * VLINES : ta * VLINES;
    nlines = xdir ? g.ny : g.nx;
    nfaces = (xdir ? g.nx : g.ny) + 1;
    ncell = xdir ? g.nx : g.ny;
    bc_lo = xdir ? g.bc[0] : g.bc[2];
    bc_hi = xdir ? g.bc[1] : g.bc[3];
    nmom = xdir ? 1 : 2;
  }
};

// Stages mu of cells f0-1 .. f0+VFACES-1 of the tile's lines (zero outside).
template <int NV, int VFACES>
__device__ __forceinline__ void stage_mu(const VjpTile& T, const double* __restrict__ mu, const GridDev& g,
                                         double (*sMu)[VLINES][VFACES + 1]) {
  const long long n = g.n;
  for (int q = threadIdx.x; q < VLINES * (VFACES + 1); q += blockDim.x) {
    int line, w;
    if (T.xdir) { line = q / (VFACES + 1); w = q % (VFACES + 1); } else { w = q / VLINES; line = q % VLINES; }
    const int lg = T.l0 + line;
    const int c = T.f0 - 1 + w;
    const bool in = lg < T.nlines && c >= 0 && c < T.ncell;
    const long long idx = T.xdir ? (long long)lg * g.nx + c : (long long)c * g.nx + lg;
#pragma unroll
    for (int k = 0; k < NV; ++k) sMu[k][line][w] = in ? mu[(long long)k * n + idx] : 0.0;
  }
}

// Slot pair of tile position 0 (cell f0 - 3) of (var, lg), and the pair stride.
__device__ __forceinline__ double* gf_base(const VjpTile& T, double* GFx, double* GFy, const GridDev& g, int var,
                                           int lg, long long& pstride) {
  if (T.xdir) {
    pstride = 2;
    return GFx + (((long long)var * g.ny + lg) * (g.nx + 6) + T.f0) * 2;
  }
  pstride = 2LL * g.nx;
  return GFy + (((long long)var * (g.ny + 6) + T.f0) * g.nx + lg) * 2;
}

template <int NV, int VFACES>
__global__ void __launch_bounds__(VLINES * NV) k_adj_faces(StateView S, const double* __restrict__ alpha2,
                                                           const double* __restrict__ mu, double mu_scale,
                                                           double* __restrict__ GFx, double* __restrict__ GFy,
                                                           GridDev g, int nbx, int ntx_x, int ntx_y) {
  constexpr int VWIN = VFACES + 5;
  __shared__ double sU[NV][VLINES][VWIN];
  __shared__ double sLp[VLINES][VWIN], sLm[VLINES][VWIN], sHp[VLINES][VWIN], sHpu[VLINES][VWIN];
  __shared__ double sMu[NV][VLINES][VFACES + 1];
  const VjpTile T(g, blockIdx.x, nbx, ntx_x, ntx_y, VFACES);
  const long long n = g.n;
  const int nx = g.nx;
  const double ha = 0.5 * alpha2[T.xdir ? 0 : 1];
  const double rh = (T.xdir ? g.rdx : g.rdy) * mu_scale;
  const double* uplane = S.plane(T.xdir ? NV + 1 : NV + 2, n);
  const double* pplane = S.plane(NV + 3, n);

  // ---- stage: cells f0-3 .. f0+VFACES+1 of every line, and mu ----
  for (int q = threadIdx.x; q < VLINES * VWIN; q += blockDim.x) {
    int line, w;
    if (T.xdir) { line = q / VWIN; w = q % VWIN; } else { w = q / VLINES; line = q % VLINES; }
    int lg = T.l0 + line;
    if (lg >= T.nlines) lg = T.nlines - 1;  // inactive line: any valid cell
    int cg = T.f0 - 3 + w;
    if (cg > T.ncell + 2) cg = T.ncell + 2;
    bool flip;
    const int src = ghost_src(cg, T.ncell, T.bc_lo, T.bc_hi, flip);
    const long long idx = T.xdir ? (long long)lg * nx + src : (long long)src * nx + lg;
    double un = uplane[idx];
    if (flip) un = -un;
    const double hp = 0.5 * pplane[idx];
    sLp[line][w] = fma(0.5, un, ha);
    sLm[line][w] = fma(0.5, un, -ha);
    sHp[line][w] = hp;
    sHpu[line][w] = hp * un;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double v = S.plane(k, n)[idx];
      if (flip && k == T.nmom) v = -v;
      sU[k][line][w] = v;
    }
  }
  stage_mu<NV, VFACES>(T, mu, g, sMu);
  __syncthreads();

  const int var = threadIdx.x / VLINES;
  const int line = threadIdx.x % VLINES;
  const int lg = T.l0 + line;
  if (lg >= T.nlines) return;
  const int nf = min(VFACES, T.nfaces - T.f0);
  const double* Ul = sU[var][line];
  const double* lp = sLp[line];
  const double* lm = sLm[line];
  const double* pt = (var == T.nmom) ? sHp[line] : (var == 3 ? sHpu[line] : nullptr);
  const double* ml = sMu[var][line];
  auto Fp = [&](int w) -> double { return pt ? fma(lp[w], Ul[w], pt[w]) : lp[w] * Ul[w]; };
  auto Fm = [&](int w) -> double { return pt ? fma(lm[w], Ul[w], pt[w]) : lm[w] * Ul[w]; };
  long long pstride;
  double* gbase = gf_base(T, GFx, GFy, g, var, lg, pstride);
  const double rh4 = 4.0 * rh;
  Win P, M;
  P.init(Fp(0), Fp(1), Fp(2), Fp(3), Fp(4), g.eps4);
  M.init(Fm(1), Fm(2), Fm(3), Fm(4), Fm(5), g.eps4);
  EdgeSums E;
  for (int t = 0; t < nf; ++t) {
    const double dmu = ml[t + 1] - ml[t];
    weno_face_dD<false, true>(P, rh4 * dmu, nullptr, E.p0, E.p1, E.p2, E.p3);
    weno_face_dD<true, true>(M, rh4 * dmu, nullptr, E.m0, E.m1, E.m2, E.m3);
    E.finish_face(rh * dmu, gbase + (long long)t * pstride, pstride);
    if (t + 1 < nf) {
      P.push(Fp(t + 5), g.eps4);
      M.push(Fm(t + 6), g.eps4);
    }
  }
  E.flush(gbase + (long long)nf * pstride, pstride);
}

template <int NV, int VFACES>
__global__ void __launch_bounds__(VLINES * NV) k_adj_faces_lin(const double* __restrict__ lin,
                                                               const double* __restrict__ mu, double mu_scale,
                                                               double* __restrict__ GFx, double* __restrict__ GFy,
                                                               GridDev g, int nbx, int ntx_x, int ntx_y) {
  __shared__ double sMu[NV][VLINES][VFACES + 1];
  const VjpTile T(g, blockIdx.x, nbx, ntx_x, ntx_y, VFACES);
  stage_mu<NV, VFACES>(T, mu, g, sMu);
  __syncthreads();
  const int var = threadIdx.x / VLINES;
  const int line = threadIdx.x % VLINES;
  const int lg = T.l0 + line;
  if (lg >= T.nlines) return;
  const int nf = min(VFACES, T.nfaces - T.f0);
  const double rh = (T.xdir ? g.rdx : g.rdy) * mu_scale;
  const double* ml = sMu[var][line];
  // the store's layout (face_flux_tile<..., LIN>): x faces [8][NV][nx+1][ny], then y faces [8][NV][ny+1][nx]
  const long long nfx = g.nx + 1, nfy = g.ny + 1;
  const double* lb;
  long long cstride;
  if (T.xdir) { lb = lin + ((long long)var * nfx + T.f0) * g.ny + lg; cstride = (long long)NV * nfx * g.ny; }
  else { lb = lin + 8LL * NV * nfx * g.ny + ((long long)var * nfy + T.f0) * g.nx + lg; cstride = (long long)NV * nfy * g.nx; }
  const long long fstride = T.nlines;
  long long pstride;
  double* gbase = gf_base(T, GFx, GFy, g, var, lg, pstride);
  EdgeSums E;
  const double rh4 = 4.0 * rh;  // the store holds a quarter of each partial
#pragma unroll 4
  for (int t = 0; t < nf; ++t) {
    const double* l = lb + (long long)t * fstride;
    double d[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) d[c] = __ldg(l + c * cstride);
    const double dmu = ml[t + 1] - ml[t];
    const double p4 = rh4 * dmu;
    E.p0 = fma(p4, d[0], E.p0); E.p1 = fma(p4, d[1], E.p1); E.p2 = fma(p4, d[2], E.p2); E.p3 = fma(p4, d[3], E.p3);
    E.m0 = fma(p4, d[4], E.m0); E.m1 = fma(p4, d[5], E.m1); E.m2 = fma(p4, d[6], E.m2); E.m3 = fma(p4, d[7], E.m3);
    E.finish_face(rh * dmu, gbase + (long long)t * pstride, pstride);
  }
  E.flush(gbase + (long long)nf * pstride, pstride);
}

// Cell pass: cotangents of U, u_n and p of cell c from the per-position sums
// of k_adj_faces, with the ghost positions that copy cell c folded back.
// Returns via references.
template <int NV>
__device__ __forceinline__ void gather_dir(const StateView& S, double* __restrict__ GF, const GridDev& g,
                                           double ha, int xdir, int i, int j, double* aU, double& a_un, double& a_p,
                                           double& a_alpha) {
  const long long n = g.n;
  const int nx = g.nx, ny = g.ny;
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
    // all loads first, then the zeroing (each slot is read by exactly one
    // cell: the sums are left zero for the next face pass), so the loads are
    // not held behind the stores
    double* gf0 = GF + 2 * (xdir ? ((long long)line) * (nx + 6) + (e + 3) : ((long long)(e + 3)) * nx + line);
    const long long kstride = 2 * (xdir ? (long long)ny * (nx + 6) : (long long)(ny + 6) * nx);
    double fpk[NV], fmk[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      fpk[k] = gf0[k * kstride];
      fmk[k] = gf0[k * kstride + 1];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      gf0[k * kstride] = 0.0;
      gf0[k * kstride + 1] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double U = (flip && k == nmom) ? -Uc[k] : Uc[k];
      const double fp = fpk[k], fm = fmk[k];
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

// A mass-action monomial prod_s X_{sp(s)}^{a(s)} over n <= MAX_SIDE distinct
// species (sp, a: accessors of the reaction side): the value, the gradient
// g_s, the derivative along e (D), and the gradient of D
// (h_s = sum_t e_t d2/dX_t dX_s).
template <class SP, class A>
__device__ __forceinline__ void monomial(const double* X, SP sp, A a, int n, const double* e, double& val, double* g,
                                         double& D, double* h) {
  double P[MAX_SIDE], P1[MAX_SIDE], P2[MAX_SIDE];
#pragma unroll
  for (int s = 0; s < n; ++s) {
    const double x = X[sp(s)];
    double pw = 1.0;
#pragma unroll
    for (int q = 0; q < a(s) - 2; ++q) pw *= x;  // x^(a-2)
    P2[s] = a(s) >= 2 ? a(s) * (a(s) - 1) * pw : 0.0;
    const double pw1 = a(s) >= 2 ? pw * x : 1.0;  // x^(a-1)
    P1[s] = a(s) * pw1;
    P[s] = pw1 * x;
  }
  val = 1.0;
#pragma unroll
  for (int s = 0; s < n; ++s) val *= P[s];
  D = 0.0;
#pragma unroll
  for (int s = 0; s < n; ++s) {
    double ex = P1[s];
#pragma unroll
    for (int t = 0; t < n; ++t)
      if (t != s) ex *= P[t];
    g[s] = ex;
    D = fma(e[sp(s)], ex, D);
  }
#pragma unroll
  for (int s = 0; s < n; ++s) {
    double hs = 0.0;
#pragma unroll
    for (int t = 0; t < n; ++t) {
      double v;
      if (t == s) {
        v = P2[s];
#pragma unroll
        for (int w = 0; w < n; ++w)
          if (w != s) v *= P[w];
      } else {
        v = P1[s] * P1[t];
#pragma unroll
        for (int w = 0; w < n; ++w)
          if (w != s && w != t) v *= P[w];
      }
      hs = fma(e[sp(t)], v, hs);
    }
    h[s] = hs;
  }
}

// Explicit source S(U): rho Y_k rows receive M_k wdot_k(T(U), X(U)). Its VJP
// (dS/dU)^T mu is the gradient of g = sum_i m_i q_i with
// m_i = sum_k nu_ki w_k, w_k = M_k mu_{4+k}, in (T, X) per reaction; the cell
// pass chains it through X(U) and the implicit dT/dU. keep: k_f and k_b of
// the stage input kept by the forward (entries 2i, 2i+1 of cell q), or null
// to form them again.
template <int NS>
__device__ __forceinline__ void src_grad(const double* u, double T, const MechDev& m, const double* w,
                                         const double* __restrict__ keep, long long n, long long q, double& gT_out,
                                         double* gX) {
  constexpr int NSP = NS - 1;
  double X[NS];
  double rest = u[0];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    X[k] = u[4 + k] * m.invM[k];
    rest -= u[4 + k];
  }
  X[NSP] = rest * m.invM[NSP];
  double Ctot = X[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) Ctot += X[k];
  const double rT = rcp(T);
  const double rT2 = rT * rT;
  // with `keep` the forward's k_f and k_b are read back and exp(G_k) is not needed
  const double lnT = keep ? 0.0 : log(T);
  double eG[NS], reG[NS], dG[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* c = m.gc[k];
    if (!keep) {
      eG[k] = exp_t(fma(c[0], lnT, fma(c[5], rT, fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), c[6]))));
      reG[k] = rcp(eG[k]);
    }
    dG[k] = fma(c[0], rT, fma(-c[5], rT2, fma(T, fma(T, fma(T, 4.0 * c[4], 3.0 * c[3]), 2.0 * c[2]), c[1])));
  }
  const double cref = (P_REF / RU) * rT;
  const double rcref = (RU / P_REF) * T;
  double zero[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) zero[k] = 0.0;
  double gT = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) gX[k] = 0.0;
  for (int i = 0; i < m.nr; ++i) {
    const int nre = m.nre[i], npr = m.npr[i];
    double mi = 0.0;
    for (int r = 0; r < nre; ++r)
      if (m.rsp[i][r] < NSP) mi = fma(-m.rnud[i][r], w[m.rsp[i][r]], mi);
    for (int r = 0; r < npr; ++r)
      if (m.psp[i][r] < NSP) mi = fma(m.pnud[i][r], w[m.psp[i][r]], mi);
    const double dlkf = fma(m.b[i], rT, m.EaR[i] * rT2);
    double kf, kb, dlkb = dlkf;
    for (int r = 0; r < nre; ++r)
      for (int qq = 0; qq < m.rnu[i][r]; ++qq) dlkb += dG[m.rsp[i][r]];
    for (int r = 0; r < npr; ++r)
      for (int qq = 0; qq < m.pnu[i][r]; ++qq) dlkb -= dG[m.psp[i][r]];
    const int dn = m.dnu[i];
    dlkb = fma((double)dn, rT, dlkb);
    if (keep) {
      kf = __ldg(keep + (2LL * i) * n + q);
      kb = __ldg(keep + (2LL * i + 1) * n + q);
    } else {
      kf = exp_t(fma(m.b[i], lnT, fma(-m.EaR[i], rT, m.lnA[i])));
      kb = kf;
      for (int r = 0; r < nre; ++r)
        for (int qq = 0; qq < m.rnu[i][r]; ++qq) kb *= eG[m.rsp[i][r]];
      for (int r = 0; r < npr; ++r)
        for (int qq = 0; qq < m.pnu[i][r]; ++qq) kb *= reG[m.psp[i][r]];
      for (int qq = 0; qq < dn; ++qq) kb *= rcref;
      for (int qq = 0; qq < -dn; ++qq) kb *= cref;
    }
    double F, gF[MAX_SIDE], DF, hF[MAX_SIDE], B, gB[MAX_SIDE], DB, hB[MAX_SIDE];
    monomial(X, [&](int s_) { return m.rsp[i][s_]; }, [&](int s_) { return m.rnu[i][s_]; }, nre, zero, F, gF, DF, hF);
    monomial(X, [&](int s_) { return m.psp[i][s_]; }, [&](int s_) { return m.pnu[i][s_]; }, npr, zero, B, gB, DB, hB);
    double Mi = 1.0;
    if (m.tb[i]) {
      Mi = Ctot;
      for (int e = 0; e < m.neff[i]; ++e) Mi = fma(m.effv[i][e], X[m.effsp[i][e]], Mi);
    }
    const double net = fma(kf, F, -kb * B);
    gT = fma(mi * Mi, fma(kf * dlkf, F, -kb * dlkb * B), gT);
    for (int r = 0; r < nre; ++r) gX[m.rsp[i][r]] = fma(mi * Mi * kf, gF[r], gX[m.rsp[i][r]]);
    for (int r = 0; r < npr; ++r) gX[m.psp[i][r]] = fma(-mi * Mi * kb, gB[r], gX[m.psp[i][r]]);
    if (m.tb[i])
      for (int j = 0; j < NS; ++j) gX[j] = fma(1.0 + m.effm1[i][j], mi * net, gX[j]);
  }
  gT_out = gT;
}

// Lexicographic arg-max step: the larger speed (non-negative doubles as
// bits), on equal speeds the lower linear index.
__device__ __forceinline__ void argmax_merge(unsigned long long& m, int& i, unsigned long long m2, int i2) {
  if (m2 > m || (m2 == m && i2 < i)) { m = m2; i = i2; }
}

// Cell pass of the RHS VJP (256 threads per block). Besides the gathered
// cotangents it leaves, per block, the block sums of the alpha cotangents
// (atomically added) and the arg-max of |u|+c and |v|+c over its cells in
// part_mx / part_id [2 * block + direction].
// SRC (the explicit source-term form): the cell also adds the VJP of the
// source S(U) at this stage state, (dS/dU)^T mu (src_grad, with the rate
// constants from src_keep when the forward kept them).
template <int NS, bool SRC>
__global__ void k_adj_cells(StateView S, const double* __restrict__ alpha2, double* __restrict__ GFx,
                            double* __restrict__ GFy, VjpIO io, double* adj_alpha, GridDev g,
                            const MechDev* __restrict__ mech, unsigned long long* __restrict__ part_mx,
                            int* __restrict__ part_id, const double* __restrict__ src_keep) {
  constexpr int NV = NS + 3;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double ax = 0.0, ay = 0.0;
  unsigned long long sx = 0, sy = 0;
  int cid = 0x7fffffff;
  if (i < g.nx && j < g.ny) {
    const long long n = g.n;
    const long long idx = (long long)j * g.nx + i;
    double aU[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) aU[k] = 0.0;
    double a_u = 0.0, a_v = 0.0, a_p = 0.0;
    gather_dir<NV>(S, GFx, g, 0.5 * alpha2[0], 1, i, j, aU, a_u, a_p, ax);
    gather_dir<NV>(S, GFy, g, 0.5 * alpha2[1], 0, i, j, aU, a_v, a_p, ay);
    double u[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[idx];
    const double T = S.plane(NV, n)[idx];
    const double rrho = rcp(u[0]);
    const double vx = u[1] * rrho, vy = u[2] * rrho;
    CellThermo<NS> ct;
    cell_thermo<NS>(u, T, *mech, ct);
    double dT[NV], dp[NV];
    dT_dp_dU<NS>(u, T, *mech, ct, dT, dp);
    aU[0] += -(vx * a_u + vy * a_v) * rrho;
    aU[1] += a_u * rrho;
    aU[2] += a_v * rrho;
    if constexpr (SRC) {
      constexpr int NSP = NS - 1;
      const MechDev& m = *mech;
      double w[NSP];
#pragma unroll
      for (int k = 0; k < NSP; ++k) w[k] = m.M[k] * (io.mu_scale * io.lam[(long long)(4 + k) * n + idx]);
      double gT, gX[NS];
      src_grad<NS>(u, T, m, w, src_keep, n, idx, gT, gX);
      const double gN = gX[NSP] * m.invM[NSP];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double d = gT * dT[k];
        if (k == 0) d += gN;
        if (k >= 4) d += fma(gX[k - 4], m.invM[k - 4], -gN);
        aU[k] += d;
      }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const long long kq = (long long)k * n + idx;
      double va = fma(dp[k], a_p, aU[k]);  // nu
      if (io.acc_a) va += io.a[kq];
      if (io.xa) va = fma(io.ca, io.xa[kq], va);
      io.a[kq] = va;
      if (io.b) {
        const double vb = io.cb * io.xb[kq];
        io.b[kq] = io.acc_b ? io.b[kq] + vb : vb;
      }
    }
    // the LF speeds of this cell, as the forward's alpha max formed them
    const double c = sound_speed<NS>(u, T, *mech);
    const double rr = rcp(u[0]);
    sx = dbits(dabs(u[1] * rr) + c);
    sy = dbits(dabs(u[2] * rr) + c);
    cid = (int)idx;
  }
  // block sums of the alpha cotangents and block arg-max of the speeds
  __shared__ double rx[256], ry[256];
  __shared__ unsigned long long mx[2][256];
  __shared__ int id[2][256];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  rx[tid] = ax;
  ry[tid] = ay;
  mx[0][tid] = sx;
  mx[1][tid] = sy;
  id[0][tid] = cid;
  id[1][tid] = cid;
  __syncthreads();
  for (int s = blockDim.x * blockDim.y / 2; s > 0; s >>= 1) {
    if (tid < s) {
      rx[tid] += rx[tid + s];
      ry[tid] += ry[tid + s];
#pragma unroll
      for (int d = 0; d < 2; ++d) argmax_merge(mx[d][tid], id[d][tid], mx[d][tid + s], id[d][tid + s]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(adj_alpha, rx[0]);
    atomicAdd(adj_alpha + 1, ry[0]);
    const int b = blockIdx.x + gridDim.x * blockIdx.y;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      part_mx[2 * b + d] = mx[d][0];
      part_id[2 * b + d] = id[d][0];
    }
  }
}

// The alpha cotangents flow to the arg-max cells: d(|u_d| + c)/dU. One block
// of 256 threads: the arg-max over the nb block partials of k_adj_cells
// (ties: lowest linear index), then thread 0 applies the two cotangents.
template <int NS>
__global__ void k_adj_alpha(StateView S, GridDev g, const MechDev* __restrict__ mech,
                            const unsigned long long* __restrict__ part_mx, const int* __restrict__ part_id, int nb,
                            double* adj_alpha, double* nu) {
  constexpr int NV = NS + 3;
  __shared__ unsigned long long mx[2][256];
  __shared__ int id[2][256];
  const int tid = threadIdx.x;
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    unsigned long long m = 0;
    int i = 0x7fffffff;
    for (int b = tid; b < nb; b += blockDim.x) argmax_merge(m, i, part_mx[2 * b + d], part_id[2 * b + d]);
    mx[d][tid] = m;
    id[d][tid] = i;
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
#pragma unroll
      for (int d = 0; d < 2; ++d) argmax_merge(mx[d][tid], id[d][tid], mx[d][tid + s], id[d][tid + s]);
    }
    __syncthreads();
  }
  // Warp 0: lane k < NV takes component k of d(|u_0| + c)/dU at the x
  // arg-max cell, lane 16 + k the same component of d(|v| + c)/dU at the y
  // arg-max cell; lane k then adds both (x first), so a cell that is the
  // arg-max of both directions receives them in that order.
  static_assert(NV <= 16, "one half-warp per direction");
  if (tid >= 32) return;
  const int d = tid >> 4, k = tid & 15;
  const long long n = g.n;
  const int cidx = id[d][0];
  double contrib = 0.0;
  if (k < NV && cidx >= 0 && cidx < g.n) {
    const double a = adj_alpha[d];
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = S.plane(q, n)[cidx];
    const double T = S.plane(NV, n)[cidx];
    const MechDev& m = *mech;
    CellThermo<NS> ct;
    cell_thermo<NS>(u, T, m, ct);
    const double rho = u[0];
    // component k of dT/dU and dp/dU (as dT_dp_dU forms them)
    const double rrho = 1.0 / rho;
    const double vx = u[1] * rrho, vy = u[2] * rrho;
    const double fN = (ct.hR[NS - 1] - T) * m.invM[NS - 1];
    double dF, dWk = 0.0, dz_cv = 0.0;
    if (k == 0) {
      dF = fN - 0.5 * (vx * vx + vy * vy) * (1.0 / RU);
      dWk = m.invM[NS - 1];
      dz_cv = ct.cvR[NS - 1] * m.invM[NS - 1];
    } else if (k == 1) {
      dF = vx * (1.0 / RU);
    } else if (k == 2) {
      dF = vy * (1.0 / RU);
    } else if (k == 3) {
      dF = -1.0 / RU;
    } else {
      dF = (ct.hR[k - 4] - T) * m.invM[k - 4] - fN;
      dWk = m.invM[k - 4] - m.invM[NS - 1];
      dz_cv = ct.cvR[k - 4] * m.invM[k - 4] - ct.cvR[NS - 1] * m.invM[NS - 1];
    }
    const double rCv = 1.0 / ct.Cv;
    const double dTk = -dF * rCv;
    const double dpk = RU * (T * dWk + ct.W * dTk);
    const double p = RU * ct.W * T;
    const double Cv = ct.Cv, Cp = ct.Cv + ct.W;
    const double c = sqrt(Cp * p / (Cv * rho));
    const double vel = u[1 + d] / rho;
    const double sgn = vel < 0.0 ? -1.0 : 1.0;
    const double dCv = dz_cv + ct.dCv * dTk;
    const double dCp = dCv + dWk;
    const double drho = k == 0 ? 1.0 : 0.0;
    const double dc = 0.5 * c * (dCp / Cp + dpk / p - dCv / Cv - drho / rho);
    double dvel = 0.0;
    if (k == 0) dvel = -vel / rho;
    if (k == 1 + d) dvel = 1.0 / rho;
    contrib = a * (sgn * dvel + dc);
  }
  const double cy = __shfl_down_sync(0xffffffffu, contrib, 16);
  if (d == 0 && k < NV) {
    const int cx = id[0][0], cyi = id[1][0];
    if (cx >= 0 && cx < g.n) nu[(long long)k * n + cx] += contrib;
    if (cyi >= 0 && cyi < g.n) nu[(long long)k * n + cyi] += cy;
  }
  // the cotangents are consumed: leave them zero for the next cell pass
  __syncwarp();
  if (tid == 0) {
    adj_alpha[0] = 0.0;
    adj_alpha[1] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Chemistry VJP in reverse mode.
//
// The point-implicit update (Eq. 4.12-4.13) is rho Y_k += M_k x_k with
// A x = dt wd, A = I - dt J'', all at (T*, X(U*)), T* = T(U*). For the
// cotangent lam of U^{n+1}, with r_k = M_k lam_{4+k} and mu = A^{-T} r,
//   lam^T dU^{n+1} = lam^T dU* + mu^T (dt dwd + dt dJ'' x),
// and J'' x is the derivative of wd along x_eff = (x_0..x_{ns-2},
// -sum_l (M_l/M_ns) x_l) in concentration space. So the VJP is lam plus the
// gradient with respect to U* of
//   psi = dt sum_i m_i (q_i + Dq_i[x_eff]),  m_i = sum_k nu_ki mu_k,
// at fixed mu and x. psi depends on T only through k_f and k_b, and on the
// concentrations through the third-body sum (linear) and the mass-action
// monomials; its gradient in (T, X) is written out per reaction below and
// chained to U* through X(U*) and the implicit dT/dU* of the Newton recovery.
// ---------------------------------------------------------------------------

// The forward pass keeps k_f, k_b and their log-T derivatives of every
// reaction for the reverse pass: in local arrays for the run-time table, in
// shared memory (one column of 4 NR doubles per thread, every index a
// constant) for the compiled structure.
struct LocalRateCache {
  double kf[MAX_NR], kb[MAX_NR], dkf[MAX_NR], dkb[MAX_NR];
  __device__ __forceinline__ void put(int i, double a, double b, double c, double d) {
    kf[i] = a; kb[i] = b; dkf[i] = c; dkb[i] = d;
  }
  __device__ __forceinline__ double k_f(int i) const { return kf[i]; }
  __device__ __forceinline__ double k_b(int i) const { return kb[i]; }
  template <class Rx>
  __device__ __forceinline__ double dk_f(const Rx& R) const { return dkf[R.idx()]; }
  template <class Rx>
  __device__ __forceinline__ double dk_b(const Rx& R) const { return dkb[R.idx()]; }
};
struct SharedRateCache {
  double* col;  // this thread's column: entry q at col[q * stride]
  int stride;
  __device__ __forceinline__ void put(int i, double a, double b, double c, double d) {
    col[(4 * i) * stride] = a;
    col[(4 * i + 1) * stride] = b;
    col[(4 * i + 2) * stride] = c;
    col[(4 * i + 3) * stride] = d;
  }
  __device__ __forceinline__ double k_f(int i) const { return col[(4 * i) * stride]; }
  __device__ __forceinline__ double k_b(int i) const { return col[(4 * i + 1) * stride]; }
  template <class Rx>
  __device__ __forceinline__ double dk_f(const Rx& R) const { return col[(4 * R.idx() + 2) * stride]; }
  template <class Rx>
  __device__ __forceinline__ double dk_b(const Rx& R) const { return col[(4 * R.idx() + 3) * stride]; }
};
// The rate constants the segment recompute's chemistry kept (k_chem_lin:
// k_f, k_b of reaction i at entries 2i, 2i+1 of cell q) and their log-T
// derivatives formed here, as the forward pass of chem_vjp_rev forms them:
// d ln k_f/dT = b/T + Ea/(R T^2), d ln k_b/dT = d ln k_f/dT + sum over the
// reactants of dG - sum over the products of dG + dnu/T.
template <int NS>
struct StoredRateCache {
  const double* clin;
  long long n, q;
  double rT, rT2;
  const double* dG;
  const MechDev& m;
  __device__ __forceinline__ double k_f(int i) const { return __ldg(clin + (2LL * i) * n + q); }
  __device__ __forceinline__ double k_b(int i) const { return __ldg(clin + (2LL * i + 1) * n + q); }
  template <class Rx>
  __device__ __forceinline__ double dk_f(const Rx& R) const {
    const int i = R.idx();
    return fma(m.b[i], rT, m.EaR[i] * rT2);
  }
  template <class Rx>
  __device__ __forceinline__ double dk_b(const Rx& R) const {
    double d = dk_f(R);
#pragma unroll
    for (int r = 0; r < R.nre(); ++r)
#pragma unroll
      for (int k = 0; k < R.rnu(r); ++k) d += dG[R.rsp(r)];
#pragma unroll
    for (int r = 0; r < R.npr(); ++r)
#pragma unroll
      for (int k = 0; k < R.pnu(r); ++k) d -= dG[R.psp(r)];
    return fma((double)R.dnu(), rT, d);
  }
};

// Reverse pass over the reactions (shared by both chemistry VJPs): the
// gradient (gT, gX) of psi = dt sum_i m_i (q_i + Dq_i[x_eff]) in (T, X),
// m_i = sum_k nu_ki mu_k, with the rate constants and their log-T
// derivatives from `cache`.
template <int NS, bool FIXED, class Cache>
__device__ __forceinline__ void chem_reverse_reactions(const MechDev& m, const double* X, const double* xe, double Ctot,
                                                       const double* mu, double dt, const Cache& cache, double& gT_out,
                                                       double* gX) {
  constexpr int NSP = NS - 1;
  double gT = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) gX[k] = 0.0;
  for_reactions<FIXED>(m, [&](auto R) {
    const int i = R.idx();
    const int nre = R.nre(), npr = R.npr();
    double mi = 0.0;
#pragma unroll
    for (int r = 0; r < nre; ++r)
      if (R.rsp(r) < NSP) mi = fma(-R.rnud(r), mu[R.rsp(r)], mi);
#pragma unroll
    for (int r = 0; r < npr; ++r)
      if (R.psp(r) < NSP) mi = fma(R.pnud(r), mu[R.psp(r)], mi);
    const double w = dt * mi;
    const double kf = cache.k_f(i), kb = cache.k_b(i);
    double F, gF[MAX_SIDE], DF, hF[MAX_SIDE], B, gB[MAX_SIDE], DB, hB[MAX_SIDE];
    monomial(X, [&](int s_) { return R.rsp(s_); }, [&](int s_) { return R.rnu(s_); }, nre, xe, F, gF, DF, hF);
    monomial(X, [&](int s_) { return R.psp(s_); }, [&](int s_) { return R.pnu(s_); }, npr, xe, B, gB, DB, hB);
    const double net = fma(kf, F, -kb * B);
    const double Dnet = fma(kf, DF, -kb * DB);
    double Mi = 1.0, DMi = 0.0;
    if (R.tb()) {
      Mi = Ctot;
#pragma unroll
      for (int e = 0; e < R.neff(); ++e) Mi = fma(m.effv[i][e], X[R.effsp(e)], Mi);
#pragma unroll
      for (int j = 0; j < NS; ++j) DMi = fma(1.0 + m.effm1[i][j], xe[j], DMi);
    }
    const double MD = Mi + DMi;
    const double kfp = kf * cache.dk_f(R), kbp = kb * cache.dk_b(R);
    gT = fma(w, fma(MD, fma(kfp, F, -kbp * B), Mi * fma(kfp, DF, -kbp * DB)), gT);
#pragma unroll
    for (int r = 0; r < nre; ++r) {
      const int j = R.rsp(r);
      gX[j] = fma(w * kf, fma(MD, gF[r], Mi * hF[r]), gX[j]);
    }
#pragma unroll
    for (int r = 0; r < npr; ++r) {
      const int j = R.psp(r);
      gX[j] = fma(-w * kb, fma(MD, gB[r], Mi * hB[r]), gX[j]);
    }
    if (R.tb()) {
      const double v = w * (net + Dnet);
#pragma unroll
      for (int j = 0; j < NS; ++j) gX[j] = fma(1.0 + m.effm1[i][j], v, gX[j]);
    }
  });
  gT_out = gT;
}

// Chain of the chemistry VJP to U*: X(U*) and the implicit dT/dU* of the
// Newton recovery; out = lam + (d(T, X)/dU*)^T (gT, gX).
template <int NS>
__device__ __forceinline__ void chem_vjp_out(const double* u, double T, const MechDev& m, const double* lam, double gT,
                                             const double* gX, double* out) {
  constexpr int NSP = NS - 1;
  constexpr int NV = NS + 3;
  CellThermo<NS> ct;
  cell_thermo<NS>(u, T, m, ct);
  double dT[NV], dp[NV];
  dT_dp_dU<NS>(u, T, m, ct, dT, dp);
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = fma(gT, dT[q], lam[q]);
  const double gN = gX[NSP] * m.invM[NSP];
  out[0] += gN;
#pragma unroll
  for (int k = 0; k < NSP; ++k) out[4 + k] += fma(gX[k], m.invM[k], -gN);
}

template <int NS, bool FIXED, class Cache>
__device__ void chem_vjp_rev(const double* u, double T, const MechDev& m, double dt, const double* lam, double* out,
                             Cache& cache) {
  constexpr int NSP = NS - 1;
  constexpr int NV = NS + 3;
  double X[NS];
  double rest = u[0];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    X[k] = u[4 + k] * m.invM[k];
    rest -= u[4 + k];
  }
  X[NSP] = rest * m.invM[NSP];
  double Ctot = X[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) Ctot += X[k];
  const double lnT = log(T);
  const double rT = rcp(T);
  const double rT2 = rT * rT;
  double eG[NS], reG[NS], dG[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* c = m.gc[k];
    const double G = fma(c[0], lnT, fma(c[5], rT, fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), c[6])));
    eG[k] = exp_t(G);
    reG[k] = rcp(eG[k]);
    dG[k] = fma(c[0], rT, fma(-c[5], rT2, fma(T, fma(T, fma(T, 4.0 * c[4], 3.0 * c[3]), 2.0 * c[2]), c[1])));
  }
  const double cref = (P_REF / RU) * rT;
  const double rcref = (RU / P_REF) * T;

  // ---- forward: rates, J'' and the caches of the reverse pass ----
  double wd[NSP], A[NSP][NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    wd[k] = 0.0;
#pragma unroll
    for (int l = 0; l < NSP; ++l) A[k][l] = 0.0;
  }
  for_reactions<FIXED>(m, [&](auto R) {
    const int i = R.idx();
    const int nre = R.nre(), npr = R.npr();
    const double kf = exp_t(fma(m.b[i], lnT, fma(-m.EaR[i], rT, m.lnA[i])));
    const double dlkf = fma(m.b[i], rT, m.EaR[i] * rT2);
    double kb = kf, dlkb = dlkf;
#pragma unroll
    for (int r = 0; r < nre; ++r)
#pragma unroll
      for (int q = 0; q < R.rnu(r); ++q) { kb *= eG[R.rsp(r)]; dlkb += dG[R.rsp(r)]; }
#pragma unroll
    for (int r = 0; r < npr; ++r)
#pragma unroll
      for (int q = 0; q < R.pnu(r); ++q) { kb *= reG[R.psp(r)]; dlkb -= dG[R.psp(r)]; }
    const int dn = R.dnu();
#pragma unroll
    for (int q = 0; q < dn; ++q) kb *= rcref;
#pragma unroll
    for (int q = 0; q < -dn; ++q) kb *= cref;
    dlkb = fma((double)dn, rT, dlkb);
    cache.put(i, kf, kb, dlkf, dlkb);
    double xr[MAX_SIDE], xp[MAX_SIDE];
    double fwd = kf, bwd = kb;
#pragma unroll
    for (int r = 0; r < nre; ++r) {
      xr[r] = X[R.rsp(r)];
#pragma unroll
      for (int q = 0; q < R.rnu(r); ++q) fwd *= xr[r];
    }
#pragma unroll
    for (int r = 0; r < npr; ++r) {
      xp[r] = X[R.psp(r)];
#pragma unroll
      for (int q = 0; q < R.pnu(r); ++q) bwd *= xp[r];
    }
    double Mi = 1.0;
    if (R.tb()) {
      Mi = Ctot;
#pragma unroll
      for (int e = 0; e < R.neff(); ++e) Mi = fma(m.effv[i][e], X[R.effsp(e)], Mi);
    }
    const double net = fwd - bwd;
    const double q = Mi * net;
    double dq[2 * MAX_SIDE];
    int dsp[2 * MAX_SIDE];
    int nd = 0;
#pragma unroll
    for (int r = 0; r < nre; ++r) {
      double dd = kf * R.rnud(r);
#pragma unroll
      for (int s2 = 0; s2 < nre; ++s2) {
        const int pw = R.rnu(s2) - (s2 == r ? 1 : 0);
#pragma unroll
        for (int t = 0; t < pw; ++t) dd *= xr[s2];
      }
      dq[nd] = Mi * dd;
      dsp[nd++] = R.rsp(r);
    }
#pragma unroll
    for (int r = 0; r < npr; ++r) {
      double dd = kb * R.pnud(r);
#pragma unroll
      for (int s2 = 0; s2 < npr; ++s2) {
        const int pw = R.pnu(s2) - (s2 == r ? 1 : 0);
#pragma unroll
        for (int t = 0; t < pw; ++t) dd *= xp[s2];
      }
      dq[nd] = -Mi * dd;
      dsp[nd++] = R.psp(r);
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int cnt = side ? npr : nre;
#pragma unroll
      for (int r = 0; r < cnt; ++r) {
        const int k = side ? R.psp(r) : R.rsp(r);
        if (k >= NSP) continue;
        const double nu = side ? R.pnud(r) : -R.rnud(r);
        wd[k] = fma(nu, q, wd[k]);
#pragma unroll
        for (int d = 0; d < nre + npr; ++d) {
          const int jj = dsp[d];
          if (jj < NSP) {
            A[k][jj] = fma(nu, dq[d], A[k][jj]);
          } else {
            const double v = dq[d] * nu;
#pragma unroll
            for (int l = 0; l < NSP; ++l) A[k][l] = fma(-m.mratio[l], v, A[k][l]);
          }
        }
        if (R.tb()) {
          const double v = net * nu;
#pragma unroll
          for (int l = 0; l < NSP; ++l) A[k][l] = fma(m.ceff[i][l], v, A[k][l]);
        }
      }
    }
  });
  // A = I - dt J'', factored P A = L U in place (partial pivoting on
  // values). Row swaps and the final un-permutation are selects over the
  // candidate rows, so every index stays a constant.
  double x[NSP];
  int perm[NSP];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    x[k] = dt * wd[k];
#pragma unroll
    for (int l = 0; l < NSP; ++l) A[k][l] = fma(-dt, A[k][l], k == l ? 1.0 : 0.0);
  }
#pragma unroll
  for (int c = 0; c < NSP; ++c) {
    int piv = c;
    double best = fabs(A[c][c]);
#pragma unroll
    for (int r = c + 1; r < NSP; ++r)
      if (fabs(A[r][c]) > best) { best = fabs(A[r][c]); piv = r; }
    perm[c] = piv;
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      const double ac = A[c][k];
      double v = ac;
#pragma unroll
      for (int r = c + 1; r < NSP; ++r) v = (piv == r) ? A[r][k] : v;
#pragma unroll
      for (int r = c + 1; r < NSP; ++r) A[r][k] = (piv == r) ? ac : A[r][k];
      A[c][k] = v;
    }
    {
      const double xc = x[c];
      double v = xc;
#pragma unroll
      for (int r = c + 1; r < NSP; ++r) v = (piv == r) ? x[r] : v;
#pragma unroll
      for (int r = c + 1; r < NSP; ++r) x[r] = (piv == r) ? xc : x[r];
      x[c] = v;
    }
    const double ip = rcp(A[c][c]);
#pragma unroll
    for (int r = c + 1; r < NSP; ++r) {
      const double f = A[r][c] * ip;
      A[r][c] = f;  // L
#pragma unroll
      for (int k = c + 1; k < NSP; ++k) A[r][k] = fma(-f, A[c][k], A[r][k]);
      x[r] = fma(-f, x[c], x[r]);
    }
  }
#pragma unroll
  for (int r = NSP - 1; r >= 0; --r) {
    double s = x[r];
#pragma unroll
    for (int k = r + 1; k < NSP; ++k) s = fma(-A[r][k], x[k], s);
    x[r] = s * rcp(A[r][r]);
  }
  // mu = A^{-T} r: U^T z = r, L^T w = z, then undo the row swaps
  double mu[NSP];
#pragma unroll
  for (int c = 0; c < NSP; ++c) {
    double s = m.M[c] * lam[4 + c];
#pragma unroll
    for (int k = 0; k < c; ++k) s = fma(-A[k][c], mu[k], s);
    mu[c] = s * rcp(A[c][c]);
  }
#pragma unroll
  for (int c = NSP - 1; c >= 0; --c) {
    double s = mu[c];
#pragma unroll
    for (int k = c + 1; k < NSP; ++k) s = fma(-A[k][c], mu[k], s);
    mu[c] = s;
  }
#pragma unroll
  for (int c = NSP - 1; c >= 0; --c) {
    const int p = perm[c];
    const double mc = mu[c];
    double v = mc;
#pragma unroll
    for (int r = c + 1; r < NSP; ++r) v = (p == r) ? mu[r] : v;
#pragma unroll
    for (int r = c + 1; r < NSP; ++r) mu[r] = (p == r) ? mc : mu[r];
    mu[c] = v;
  }
  double xe[NS];
  double xN = 0.0;
#pragma unroll
  for (int l = 0; l < NSP; ++l) {
    xe[l] = x[l];
    xN = fma(-m.mratio[l], x[l], xN);
  }
  xe[NSP] = xN;

  // ---- reverse: gradient of psi in (T, X) ----
  double gT, gX[NS];
  chem_reverse_reactions<NS, FIXED>(m, X, xe, Ctot, mu, dt, cache, gT, gX);
  chem_vjp_out<NS>(u, T, m, lam, gT, gX, out);
}

// Chemistry VJP from the factors the segment recompute kept (k_chem_lin):
// no rates, Jacobian or factorisation are formed again. The transposed solve
// A^T mu = r runs on the LU factors in elimination order: with
// A = P_1 L_1 P_2 L_2 ... P_{n-1} L_{n-1} U (P_c the row swap of step c, L_c
// the multipliers of step c in the rows' positions at that step),
// mu = P_1 L_1^{-T} ... P_{n-1} L_{n-1}^{-T} U^{-T} r.
template <int NS, bool FIXED>
__device__ void chem_vjp_stored(const double* u, double T, const MechDev& m, double dt, const double* lam, double* out,
                                const double* __restrict__ clin, long long n, long long q) {
  constexpr int NSP = NS - 1;
  double X[NS];
  double rest = u[0];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    X[k] = u[4 + k] * m.invM[k];
    rest -= u[4 + k];
  }
  X[NSP] = rest * m.invM[NSP];
  double Ctot = X[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) Ctot += X[k];
  const double rT = rcp(T);
  const double rT2 = rT * rT;
  double dG[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* c = m.gc[k];
    dG[k] = fma(c[0], rT, fma(-c[5], rT2, fma(T, fma(T, fma(T, 4.0 * c[4], 3.0 * c[3]), 2.0 * c[2]), c[1])));
  }
  const long long lu0 = 2LL * m.nr;
  auto LU = [&](int r, int k) { return __ldg(clin + (lu0 + r * NSP + k) * n + q); };
  double xe[NS];
  double xN = 0.0;
#pragma unroll
  for (int l = 0; l < NSP; ++l) {
    xe[l] = __ldg(clin + (lu0 + NSP * NSP + 1 + l) * n + q);
    xN = fma(-m.mratio[l], xe[l], xN);
  }
  xe[NSP] = xN;
  const unsigned long long pivs = __ldg(reinterpret_cast<const unsigned long long*>(clin) + (lu0 + NSP * NSP) * n + q);
  // U^T z = r, r_k = M_k lam_{4+k} (the diagonal entries hold 1/U_kk)
  double mu[NSP];
#pragma unroll
  for (int c = 0; c < NSP; ++c) {
    double s = m.M[c] * lam[4 + c];
#pragma unroll
    for (int k = 0; k < c; ++k) s = fma(-LU(k, c), mu[k], s);
    mu[c] = s * LU(c, c);
  }
  // then, from the last step to the first: L_c^{-T}, then the swap P_c
#pragma unroll
  for (int c = NSP - 1; c >= 0; --c) {
    double s = mu[c];
#pragma unroll
    for (int r = c + 1; r < NSP; ++r) s = fma(-LU(r, c), mu[r], s);
    const int p = (int)((pivs >> (4 * c)) & 15ull);
    double v = s;
#pragma unroll
    for (int r = c + 1; r < NSP; ++r) v = (p == r) ? mu[r] : v;
#pragma unroll
    for (int r = c + 1; r < NSP; ++r) mu[r] = (p == r) ? s : mu[r];
    mu[c] = v;
  }
  const StoredRateCache<NS> cache{clin, n, q, rT, rT2, dG, m};
  double gT, gX[NS];
  chem_reverse_reactions<NS, FIXED>(m, X, xe, Ctot, mu, dt, cache, gT, gX);
  chem_vjp_out<NS>(u, T, m, lam, gT, gX, out);
}

template <int NS, bool FIXED>
__global__ void __launch_bounds__(128) k_adj_chem_lin(StateView Sstar, GridDev g, const MechDev* __restrict__ mech,
                                                      double dt, const double* __restrict__ lam,
                                                      double* __restrict__ out, const double* __restrict__ clin) {
  constexpr int NV = NS + 3;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.n) return;
  const long long n = g.n;
  double u[NV], l[NV], o[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    u[k] = Sstar.plane(k, n)[q];
    l[k] = lam[(long long)k * n + q];
  }
  chem_vjp_stored<NS, FIXED>(u, Sstar.plane(NV, n)[q], *mech, dt, l, o, clin, n, q);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[(long long)k * n + q] = o[k];
}

template <int NS, bool FIXED>
__global__ void __launch_bounds__(128) k_adj_chem_rev(StateView Sstar, GridDev g, const MechDev* __restrict__ mech,
                                                      double dt, const double* __restrict__ lam,
                                                      double* __restrict__ out) {
  constexpr int NV = NS + 3;
  extern __shared__ double rate_cols[];  // FIXED: 4 NR doubles per thread, thread-major columns
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.n) return;
  const long long n = g.n;
  double u[NV], l[NV], o[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    u[k] = Sstar.plane(k, n)[q];
    l[k] = lam[(long long)k * n + q];
  }
  if constexpr (FIXED) {
    SharedRateCache cache{rate_cols + threadIdx.x, (int)blockDim.x};
    chem_vjp_rev<NS, true>(u, Sstar.plane(NV, n)[q], *mech, dt, l, o, cache);
  } else {
    LocalRateCache cache;
    chem_vjp_rev<NS, false>(u, Sstar.plane(NV, n)[q], *mech, dt, l, o, cache);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) out[(long long)k * n + q] = o[k];
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

// Cell-pass blocks of 32 x 8 cells.
static int adj_cell_blocks(const GridDev& g) { return ((g.nx + 31) / 32) * ((g.ny + 7) / 8); }

size_t rhs_vjp_scratch_bytes(const GridDev& g) {
  return 256 + (((size_t)adj_cell_blocks(g) * 2 * (sizeof(unsigned long long) + sizeof(int)) + 255) & ~(size_t)255);
}

template <int NS>
static cudaError_t rhs_vjp_t(const StateView& S, const double* alpha2_dev, const VjpIO& io, double* CFx, double* CFy,
                             double* scratch, const GridDev& g, const MechDev* mech, const double* lin, bool fresh,
                             bool src, const double* src_keep, cudaStream_t st) {
  constexpr int NV = NS + 3;
  const int nb = adj_cell_blocks(g);
  double* adj_alpha = scratch;
  unsigned long long* part_mx = (unsigned long long*)((char*)scratch + 256);
  int* part_id = (int*)(part_mx + 2 * nb);
  const double* mu = io.lam;
  const double ms = io.mu_scale;
  if (fresh) {
    // CFx / CFy hold the per-position sums (GF of k_adj_faces); the cell
    // pass and k_adj_alpha leave them and the alpha cotangents zero
    cudaError_t e = cudaMemsetAsync(adj_alpha, 0, 2 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(CFx, 0, sizeof(double) * 2 * (size_t)NV * g.ny * (g.nx + 6), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(CFy, 0, sizeof(double) * 2 * (size_t)NV * (g.ny + 6) * g.nx, st);
    if (e != cudaSuccess) return e;
  }
  // tiles of 16 faces while that gives at least 8 blocks per SM, else 8
  const int sms = sm_count();
  auto tiles = [&](int vf, int* nbx, int* ntx_x, int* ntx_y) {
    *ntx_x = (g.nx + 1 + vf - 1) / vf;
    *ntx_y = (g.nx + VLINES - 1) / VLINES;
    *nbx = *ntx_x * ((g.ny + VLINES - 1) / VLINES);
    return *nbx + *ntx_y * ((g.ny + 1 + vf - 1) / vf);
  };
  int nbx, ntx_x, ntx_y;
  int total = tiles(16, &nbx, &ntx_x, &ntx_y);
  if (total >= 8 * sms) {
    if (lin) k_adj_faces_lin<NV, 16><<<total, VLINES * NV, 0, st>>>(lin, mu, ms, CFx, CFy, g, nbx, ntx_x, ntx_y);
    else k_adj_faces<NV, 16><<<total, VLINES * NV, 0, st>>>(S, alpha2_dev, mu, ms, CFx, CFy, g, nbx, ntx_x, ntx_y);
  } else {
    total = tiles(8, &nbx, &ntx_x, &ntx_y);
    if (lin) k_adj_faces_lin<NV, 8><<<total, VLINES * NV, 0, st>>>(lin, mu, ms, CFx, CFy, g, nbx, ntx_x, ntx_y);
    else k_adj_faces<NV, 8><<<total, VLINES * NV, 0, st>>>(S, alpha2_dev, mu, ms, CFx, CFy, g, nbx, ntx_x, ntx_y);
  }
  dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  bool done = false;
  if constexpr (NS > 1) {
    if (src) {
      k_adj_cells<NS, true><<<grd, blk, 0, st>>>(S, alpha2_dev, CFx, CFy, io, adj_alpha, g, mech, part_mx, part_id,
                                                  src_keep);
      done = true;
    }
  }
  if (!done)
    k_adj_cells<NS, false><<<grd, blk, 0, st>>>(S, alpha2_dev, CFx, CFy, io, adj_alpha, g, mech, part_mx, part_id,
                                                 nullptr);
  k_adj_alpha<NS><<<1, 256, 0, st>>>(S, g, mech, part_mx, part_id, nb, adj_alpha, io.a);
  return cudaGetLastError();
}

cudaError_t launch_rhs_vjp(int ns, const StateView& S, const double* alpha2_dev, const VjpIO& io, double* CFx,
                           double* CFy, double* scratch, const GridDev& g, const MechDev* mech, const double* lin,
                           bool fresh, bool src, const double* src_keep, cudaStream_t st) {
  switch (ns) {
    case 1: return rhs_vjp_t<1>(S, alpha2_dev, io, CFx, CFy, scratch, g, mech, lin, fresh, src, src_keep, st);
    case 3: return rhs_vjp_t<3>(S, alpha2_dev, io, CFx, CFy, scratch, g, mech, lin, fresh, src, src_keep, st);
    case 9: return rhs_vjp_t<9>(S, alpha2_dev, io, CFx, CFy, scratch, g, mech, lin, fresh, src, src_keep, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chem_vjp(int ns, const StateView& Sstar, const GridDev& g, const MechDev* mech, double dt,
                            const double* lam, double* out, const double* clin, cudaStream_t st) {
  if (clin) {
    switch (ns) {
      case 3: k_adj_chem_lin<3, false><<<nblk(g.n, 128), 128, 0, st>>>(Sstar, g, mech, dt, lam, out, clin); break;
      case 9:
        if (g.chem_fixed) k_adj_chem_lin<9, true><<<nblk(g.n, 128), 128, 0, st>>>(Sstar, g, mech, dt, lam, out, clin);
        else k_adj_chem_lin<9, false><<<nblk(g.n, 128), 128, 0, st>>>(Sstar, g, mech, dt, lam, out, clin);
        break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (ns) {
    case 3: k_adj_chem_rev<3, false><<<nblk(g.n, 128), 128, 0, st>>>(Sstar, g, mech, dt, lam, out); break;
    case 9:
      if (g.chem_fixed) {
        const int smem = (int)(sizeof(double) * 4 * fixed_h2air::NR * 128);
        static std::atomic<unsigned long long> attr_done{0};
        const cudaError_t e = set_attr_once((const void*)k_adj_chem_rev<9, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, smem, &attr_done);
        if (e != cudaSuccess) return e;
        k_adj_chem_rev<9, true><<<nblk(g.n, 128), 128, smem, st>>>(Sstar, g, mech, dt, lam, out);
      } else {
        k_adj_chem_rev<9, false><<<nblk(g.n, 128), 128, 0, st>>>(Sstar, g, mech, dt, lam, out);
      }
      break;
    default: return cudaErrorInvalidValue;
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
