// First-order point-implicit chemistry (arXiv 2504.13750, Eq. 4.12-4.13) on
// every cell, after the flux RK3 of the step (advance_source_term, Sec. 4.3).
//
// Per cell: molar concentrations X_j (the ns-th species takes what is left of
// rho), forward rates k_f = A T^b exp(-Ea/(Ru T)) (Eq. 4.8), reverse rates
// through the equilibrium constant of Eq. 4.9, rates of progress with the
// third-body factor (Eq. 4.7), and the analytic Jacobian of the carried
// sources with respect to rho Y_1..rho Y_{ns-1} at fixed T and rho (text after
// Eq. 4.13). The linear system is solved in molar unknowns
// dx_l = d(rho Y_l) / M_l, where it reads
//   (I - dt J'') dx = dt wdot,  J''_kl = dWk/dX_l - (M_l / M_ns) dWk/dX_ns,
// (row k of the mass-based system divided by M_k), with an unrolled LU
// factorisation and partial pivoting whose search and row swaps are integer
// compares and selects. Then Newton T for the new state, aux planes and the
// alpha max for the next step.
//
// exp(G_k) is formed once per species so that each reverse rate costs a few
// multiplications instead of a second exponential per reaction; the
// exponentials use the table-driven exp_t (about half the FP64 instructions
// of the library exp).
//
// The reaction loop is written once over a structure policy: DynRx reads each
// reaction's species, coefficients and third-body data from the run-time
// table, FixRx<I> returns them as compile-time constants of the shipped H2-air
// mechanism (janc_mech_fixed.cuh). Both run the same operations in the same
// order (the compiler may still contract multiply-adds differently in the
// two, so their results agree to rounding, each within the oracle's bars);
// with FixRx every index of the per-cell arrays (concentrations, exp(G_k),
// production rates, Jacobian) is a constant and the arrays live in registers
// instead of local memory.
#include <utility>

#include "janc_device.cuh"
#include "janc_internal.h"
#include "janc_mech_fixed.cuh"
#include "janc_mech_policy.cuh"

namespace janc {

constexpr int CHEM_THREADS = 128;

// One CHEM_THREADS block `blk` of cells; shared by the single-grid and the
// batched kernels. STORE (the discrete adjoint's segment recompute): also
// keep, per cell, what the chemistry VJP reuses (chem_lin_entries doubles,
// entry e of cell q at clin[e * n + q]): k_f and k_b of every reaction
// (2i, 2i+1), then at 2 nr the LU factors of A = I - dt J'' in elimination
// order (row r, column k at 2 nr + r (ns-1) + k: the multiplier of row r at
// elimination step k for r > k, U for r < k, 1/U_kk on the diagonal), the
// pivot row of every step (4 bits each, one 64-bit word) and the solution x.
template <int NS, bool FIXED, bool STORE = false>
__device__ __forceinline__ void chem_block(const StateView& S, const GridDev& g, const MechDev* __restrict__ mech,
                                           const StepCtl& ctl, const unsigned long long* __restrict__ alpha_step,
                                           unsigned long long* alpha_out, int* status, long long blk,
                                           double* __restrict__ clin = nullptr) {
  constexpr int NSP = NS - 1;
  constexpr int NV = NS + 3;
  const MechDev& m = *mech;
  const long long n = g.n;
  const long long idx = blk * blockDim.x + threadIdx.x;
  const double dt = step_dt(ctl, alpha_step) * ctl.chem_frac;
  unsigned long long sx = 0, sy = 0;
  int st = 0;
  if (idx < n) {
    double u[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[idx];
    const double T = S.plane(NV, n)[idx];

    // concentrations (Eq. 4.7 uses molar concentrations X_j)
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
    // exp(G_k) and exp(-G_k), G_k = s_k/R - h_k/(RT) (Eq. 4.9 bracket)
    double eG[NS], reG[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double* c = m.gc[k];
      const double G = fma(c[0], lnT, fma(c[5], rT, fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), c[6])));
      eG[k] = exp_t(G);
      reG[k] = rcp(eG[k]);
    }
    const double cref = (P_REF / RU) * rT;   // P_ref / (Ru T)
    const double rcref = (RU / P_REF) * T;

    double wd[NSP];        // molar production rates of the carried species
    double J[NSP][NSP];    // J'' of the header comment
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      wd[k] = 0.0;
#pragma unroll
      for (int l = 0; l < NSP; ++l) J[k][l] = 0.0;
    }

    for_reactions<FIXED>(m, [&](auto R) {
      const int i = R.idx();
      const int nre = R.nre(), npr = R.npr();
      const double kf = exp_t(fma(m.b[i], lnT, fma(-m.EaR[i], rT, m.lnA[i])));
      // k_b = k_f / K_eq,  K_eq = prod_j exp(G_j)^{nu_j} (P_ref/(Ru T))^{dnu}
      double kb = kf;
#pragma unroll
      for (int r = 0; r < nre; ++r)
#pragma unroll
        for (int q = 0; q < R.rnu(r); ++q) kb *= eG[R.rsp(r)];
#pragma unroll
      for (int r = 0; r < npr; ++r)
#pragma unroll
        for (int q = 0; q < R.pnu(r); ++q) kb *= reG[R.psp(r)];
      const int dn = R.dnu();
#pragma unroll
      for (int q = 0; q < dn; ++q) kb *= rcref;
#pragma unroll
      for (int q = 0; q < -dn; ++q) kb *= cref;
      if (STORE) {
        clin[(2LL * i) * n + idx] = kf;
        clin[(2LL * i + 1) * n + idx] = kb;
      }
      // law of mass action and its derivatives with respect to each participant
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
      // sources: wdot_k += nu_ki q
#pragma unroll
      for (int r = 0; r < nre; ++r) {
        const int k = R.rsp(r);
        if (k < NSP) wd[k] = fma(-R.rnud(r), q, wd[k]);
      }
#pragma unroll
      for (int r = 0; r < npr; ++r) {
        const int k = R.psp(r);
        if (k < NSP) wd[k] = fma(R.pnud(r), q, wd[k]);
      }
      // dq/dX_j for the participants (third-body factor held fixed here)
      double dq[2 * MAX_SIDE];
      int dsp[2 * MAX_SIDE];
      int nd = 0;
#pragma unroll
      for (int r = 0; r < nre; ++r) {
        double d = R.rnu(r) == 1 ? kf : kf * R.rnud(r);
#pragma unroll
        for (int s = 0; s < nre; ++s) {
          const int pw = R.rnu(s) - (s == r ? 1 : 0);
#pragma unroll
          for (int t = 0; t < pw; ++t) d *= xr[s];
        }
        dq[nd] = Mi * d;
        dsp[nd++] = R.rsp(r);
      }
#pragma unroll
      for (int r = 0; r < npr; ++r) {
        double d = R.pnu(r) == 1 ? kb : kb * R.pnud(r);
#pragma unroll
        for (int s = 0; s < npr; ++s) {
          const int pw = R.pnu(s) - (s == r ? 1 : 0);
#pragma unroll
          for (int t = 0; t < pw; ++t) d *= xp[s];
        }
        dq[nd] = -Mi * d;
        dsp[nd++] = R.psp(r);
      }
      // rows: every carried species with nonzero net coefficient
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int cnt = side ? npr : nre;
#pragma unroll
        for (int r = 0; r < cnt; ++r) {
          const int k = side ? R.psp(r) : R.rsp(r);
          if (k >= NSP) continue;
          const double nu = side ? R.pnud(r) : -R.rnud(r);
#pragma unroll
          for (int d = 0; d < nre + npr; ++d) {
            const int j = dsp[d];
            if (j < NSP) {
              J[k][j] = fma(nu, dq[d], J[k][j]);
            } else {
              const double v = nu * dq[d];
#pragma unroll
              for (int l = 0; l < NSP; ++l) J[k][l] = fma(-m.mratio[l], v, J[k][l]);
            }
          }
          if (R.tb()) {
            const double v = nu * net;
#pragma unroll
            for (int l = 0; l < NSP; ++l) J[k][l] = fma(v, m.ceff[i][l], J[k][l]);
          }
        }
      }
    });

    // (I - dt J'') dx = dt wd
    double A[NSP][NSP], b[NSP], ip[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      b[k] = dt * wd[k];
#pragma unroll
      for (int l = 0; l < NSP; ++l) A[k][l] = fma(-dt, J[k][l], k == l ? 1.0 : 0.0);
    }
    bool singular = false;
    const long long lu0 = 2LL * m.nr;  // STORE: first LU entry
    unsigned long long pivs = 0;
#pragma unroll
    for (int c = 0; c < NSP; ++c) {
      int piv = c;
      unsigned long long best = dbits(A[c][c]) & 0x7fffffffffffffffull;
#pragma unroll
      for (int r = c + 1; r < NSP; ++r) {
        const unsigned long long v = dbits(A[r][c]) & 0x7fffffffffffffffull;
        if (v > best) { best = v; piv = r; }
      }
      // row swap c <-> piv as selects: row c takes the pivot row's values and
      // the pivot row row c's old ones (nothing moves when piv == c). Written
      // as one gather and one scatter per column so that every index stays a
      // constant and the matrix stays in registers.
#pragma unroll
      for (int k = c; k < NSP; ++k) {
        const double ac = A[c][k];
        double v = ac;
#pragma unroll
        for (int r = c + 1; r < NSP; ++r) v = (piv == r) ? A[r][k] : v;
#pragma unroll
        for (int r = c + 1; r < NSP; ++r) A[r][k] = (piv == r) ? ac : A[r][k];
        A[c][k] = v;
      }
      {
        const double bc = b[c];
        double v = bc;
#pragma unroll
        for (int r = c + 1; r < NSP; ++r) v = (piv == r) ? b[r] : v;
#pragma unroll
        for (int r = c + 1; r < NSP; ++r) b[r] = (piv == r) ? bc : b[r];
        b[c] = v;
      }
      if (best == 0ull) singular = true;
      ip[c] = rcp(A[c][c]);
      if (STORE) pivs |= (unsigned long long)piv << (4 * c);
#pragma unroll
      for (int r = c + 1; r < NSP; ++r) {
        const double f = A[r][c] * ip[c];
        if (STORE) clin[(lu0 + r * NSP + c) * n + idx] = f;
#pragma unroll
        for (int k = c + 1; k < NSP; ++k) A[r][k] = fma(-f, A[c][k], A[r][k]);
        b[r] = fma(-f, b[c], b[r]);
      }
    }
    if (STORE) {
#pragma unroll
      for (int r = 0; r < NSP; ++r) {
        clin[(lu0 + r * NSP + r) * n + idx] = ip[r];
#pragma unroll
        for (int k = r + 1; k < NSP; ++k) clin[(lu0 + r * NSP + k) * n + idx] = A[r][k];
      }
      reinterpret_cast<unsigned long long*>(clin)[(lu0 + NSP * NSP) * n + idx] = pivs;
    }
#pragma unroll
    for (int r = NSP - 1; r >= 0; --r) {
      double s = b[r];
#pragma unroll
      for (int k = r + 1; k < NSP; ++k) s = fma(-A[r][k], b[k], s);
      b[r] = s * ip[r];
    }
    if (STORE) {
#pragma unroll
      for (int k = 0; k < NSP; ++k) clin[(lu0 + NSP * NSP + 1 + k) * n + idx] = b[k];
    }
    if (singular) {
      st |= ST_SINGULAR;
    } else {
#pragma unroll
      for (int k = 0; k < NSP; ++k) u[4 + k] = fma(m.M[k], b[k], u[4 + k]);
    }
#pragma unroll
    for (int k = 4; k < NV; ++k) S.plane(k, n)[idx] = u[k];
    double Tn, p, c, rrho;
    st |= newton_cell<NS>(u, T, m, g.newton_tol, g.newton_maxit, Tn, p, c, rrho);
    const double vx = u[1] * rrho, vy = u[2] * rrho;
    S.plane(NV, n)[idx] = Tn;
    S.plane(NV + 1, n)[idx] = vx;
    S.plane(NV + 2, n)[idx] = vy;
    S.plane(NV + 3, n)[idx] = p;
    sx = dbits(dabs(vx) + c);
    sy = dbits(dabs(vy) + c);
  }
  block_reduce_alpha_status(sx, sy, st, alpha_out, status);
}

template <int NS, bool FIXED>
__global__ void __launch_bounds__(CHEM_THREADS) k_chem(StateView S, GridDev g, const MechDev* __restrict__ mech,
                                                       StepCtl ctl, const unsigned long long* __restrict__ alpha_step,
                                                       unsigned long long* alpha_out, int* status) {
  chem_block<NS, FIXED>(S, g, mech, ctl, alpha_step, alpha_out, status, blockIdx.x);
}

// k_chem that also keeps the chemistry VJP's factors (chem_block, STORE).
template <int NS, bool FIXED>
__global__ void __launch_bounds__(CHEM_THREADS) k_chem_lin(StateView S, GridDev g, const MechDev* __restrict__ mech,
                                                           StepCtl ctl,
                                                           const unsigned long long* __restrict__ alpha_step,
                                                           unsigned long long* alpha_out, int* status,
                                                           double* __restrict__ clin) {
  chem_block<NS, FIXED, true>(S, g, mech, ctl, alpha_step, alpha_out, status, blockIdx.x, clin);
}

// Batched chemistry over the flattened (request, block) list: in place on
// each request's S[0], output alpha in slot 4.
template <int NS, bool FIXED>
__global__ void __launch_bounds__(CHEM_THREADS) k_chem_batch(const BatchReq* __restrict__ reqs,
                                                             const int* __restrict__ first, int nreq) {
  const int total = first[nreq];
  for (int e = blockIdx.x; e < total; e += gridDim.x) {
    const int r = batch_owner(first, nreq, e);
    const BatchReq& q = reqs[r];
    chem_block<NS, FIXED>(q.S[0], q.g, q.mech, q.ctl, q.alpha, q.alpha + 8, q.status, e - first[r]);
    __syncthreads();
  }
}

bool fixed_structure(const janc_mechanism* m) {
  using namespace fixed_h2air;
  if (!m || m->ns != NS || m->nr != NR || !m->nuf || !m->nub || !m->tb || !m->eff) return false;
  for (int i = 0; i < NR; ++i) {
    if ((m->tb[i] ? 1 : 0) != kTb[i]) return false;
    for (int j = 0; j < NS; ++j) {
      if (m->nuf[i * NS + j] != kNuf[i * NS + j] || m->nub[i * NS + j] != kNub[i * NS + j]) return false;
      if (kTb[i] && (m->eff[i * NS + j] != 1.0 ? 1 : 0) != kEffNe1[i * NS + j]) return false;
    }
  }
  return true;
}

cudaError_t launch_chem_batch(int ns, const BatchReq* reqs, const int* first, int nreq, int total, bool fixed,
                              cudaStream_t st) {
  const int sms = sm_count();
  const int grid = total < sms * 16 ? total : sms * 16;
  if (grid <= 0) return cudaSuccess;
  switch (ns) {
    case 3: k_chem_batch<3, false><<<grid, CHEM_THREADS, 0, st>>>(reqs, first, nreq); break;
    case 9:
      if (fixed) k_chem_batch<9, true><<<grid, CHEM_THREADS, 0, st>>>(reqs, first, nreq);
      else k_chem_batch<9, false><<<grid, CHEM_THREADS, 0, st>>>(reqs, first, nreq);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int chem_blocks(const GridDev& g) { return (int)((g.n + CHEM_THREADS - 1) / CHEM_THREADS); }

// Threads per block: CHEM_THREADS while that gives at least 4 blocks per SM,
// else 64 or 32, so that a small grid's cells spread over all SMs (each
// cell is one long dependent FP64 chain; a launch of a few blocks per SM is
// latency-bound).
static int chem_threads(long long n) {
  const int sms = sm_count();
  for (int t = CHEM_THREADS; t > 32; t /= 2)
    if ((n + t - 1) / t >= 4LL * sms) return t;
  return 32;
}

cudaError_t launch_chem(int ns, const StateView& S, const GridDev& g, const MechDev* mech, const StepCtl& ctl,
                        const unsigned long long* alpha_step, unsigned long long* alpha_out, int* status,
                        cudaStream_t st) {
  const int thr = chem_threads(g.n);
  const unsigned blocks = (unsigned)((g.n + thr - 1) / thr);
  switch (ns) {
    case 3: k_chem<3, false><<<blocks, thr, 0, st>>>(S, g, mech, ctl, alpha_step, alpha_out, status); break;
    case 9:
      if (g.chem_fixed) k_chem<9, true><<<blocks, thr, 0, st>>>(S, g, mech, ctl, alpha_step, alpha_out, status);
      else k_chem<9, false><<<blocks, thr, 0, st>>>(S, g, mech, ctl, alpha_step, alpha_out, status);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t chem_lin_entries(int ns, int nr) { return 2 * (size_t)nr + (size_t)(ns - 1) * (ns - 1) + 1 + (ns - 1); }

cudaError_t launch_chem_lin(int ns, const StateView& S, const GridDev& g, const MechDev* mech, const StepCtl& ctl,
                            const unsigned long long* alpha_step, unsigned long long* alpha_out, int* status,
                            double* clin, cudaStream_t st) {
  const int thr = chem_threads(g.n);
  const unsigned blocks = (unsigned)((g.n + thr - 1) / thr);
  switch (ns) {
    case 3: k_chem_lin<3, false><<<blocks, thr, 0, st>>>(S, g, mech, ctl, alpha_step, alpha_out, status, clin); break;
    case 9:
      if (g.chem_fixed)
        k_chem_lin<9, true><<<blocks, thr, 0, st>>>(S, g, mech, ctl, alpha_step, alpha_out, status, clin);
      else
        k_chem_lin<9, false><<<blocks, thr, 0, st>>>(S, g, mech, ctl, alpha_step, alpha_out, status, clin);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace janc
