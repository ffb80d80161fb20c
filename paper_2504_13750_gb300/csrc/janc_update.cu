// Per-cell kernels of the step (arXiv 2504.13750, Sec. 4.2-4.3): the TVD-RK3
// stage update from the face fluxes (Eq. 4.10), the Newton T recovery that
// every new state gets (end of Sec. 4.2), the auxiliary planes (u, v, p) the
// next flux evaluation reads, and the block max of |u|+c, |v|+c that becomes
// the next stage's alpha (Eq. 4.11). Also the state set-up kernels.
#include "janc_device.cuh"
#include "janc_internal.h"

namespace janc {

constexpr int UPD_BX = 32, UPD_BY = 8;

// Writes T, aux planes and returns the cell's (|u|+c, |v|+c) as bits.
template <int NS>
__device__ __forceinline__ void finish_cell(const StateView& S, long long n, long long idx, const double* u, double T,
                                            double p, double c, double rrho, unsigned long long& sx,
                                            unsigned long long& sy) {
  constexpr int NV = NS + 3;
  const double vx = u[1] * rrho, vy = u[2] * rrho;
  S.plane(NV, n)[idx] = T;
  S.plane(NV + 1, n)[idx] = vx;
  S.plane(NV + 2, n)[idx] = vy;
  S.plane(NV + 3, n)[idx] = p;
  sx = dbits(dabs(vx) + c);
  sy = dbits(dabs(vy) + c);
}

// One block (bx, by) of blockDim.x x blockDim.y cells of the stage update; shared by the
// single-grid and the batched kernels.
template <int NS, int STAGE, bool SRC = false>
__device__ __forceinline__ void rk_update_block(const StateView& Sin, const StateView& S0, const StateView& Sout,
                                                const double* __restrict__ Fx, const double* __restrict__ Gy,
                                                const GridDev& g, const MechDev* __restrict__ mech,
                                                const StepCtl& ctl, const unsigned long long* __restrict__ alpha_step,
                                                unsigned long long* alpha_out, int* status, double* clock2, int bx,
                                                int by, double* __restrict__ src_keep = nullptr) {
  constexpr int NV = NS + 3;
  const int i = bx * blockDim.x + threadIdx.x;
  const int j = by * blockDim.y + threadIdx.y;
  const long long n = g.n;
  const double dt = step_dt(ctl, alpha_step);
  if (STAGE == 1 && clock2 && bx == 0 && by == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    clock2[0] += dt;  // simulated time
    clock2[1] = dt;   // last dt
  }
  unsigned long long sx = 0, sy = 0;
  int st = 0;
  if (i < g.nx && j < g.ny) {
    const long long idx = (long long)j * g.nx + i;
    const int nx1 = g.nx + 1;
    const double cx = dt * g.rdx, cy = dt * g.rdy;
    double u[NV];
    double src[NV > 4 ? NV - 4 : 1];
    if (SRC) {  // explicit source term: production rates at the stage input
      double uin[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) uin[k] = Sin.plane(k, n)[idx];
      carried_rates<NS>(uin, Sin.plane(NV, n)[idx], *mech, src, src_keep, n, idx);
#pragma unroll
      for (int k = 0; k < NS - 1; ++k) src[k] *= mech->M[k];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double dF = Fx[((long long)k * g.ny + j) * nx1 + i + 1] - Fx[((long long)k * g.ny + j) * nx1 + i];
      const double dG = Gy[((long long)k * (g.ny + 1) + j + 1) * g.nx + i] - Gy[((long long)k * (g.ny + 1) + j) * g.nx + i];
      // U + dt L(U) with L = -(dF/dx + dG/dy) (+ the source), dt folded into
      // the face-difference factors: two FMAs per variable
      const double uin = Sin.plane(k, n)[idx];
      double t = fma(-cx, dF, fma(-cy, dG, uin));
      if (SRC && k >= 4) t = fma(dt, src[k - 4], t);
      if (STAGE == 1) {
        u[k] = t;
      } else {
        const double u0 = S0.plane(k, n)[idx];
        u[k] = (STAGE == 2) ? fma(0.75, u0, 0.25 * t) : fma(1.0 / 3.0, u0, (2.0 / 3.0) * t);
      }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) Sout.plane(k, n)[idx] = u[k];
    double T, p, c, rrho;
    st = newton_cell<NS>(u, Sin.plane(NV, n)[idx], *mech, g.newton_tol, g.newton_maxit, T, p, c, rrho);
    finish_cell<NS>(Sout, n, idx, u, T, p, c, rrho, sx, sy);
  }
  block_reduce_alpha_status(sx, sy, st, alpha_out, status);
}

template <int NS, int STAGE, bool SRC>
__global__ void __launch_bounds__(UPD_BX* UPD_BY) k_rk_update(StateView Sin, StateView S0, StateView Sout,
                                                              const double* __restrict__ Fx,
                                                              const double* __restrict__ Gy, GridDev g,
                                                              const MechDev* __restrict__ mech, StepCtl ctl,
                                                              const unsigned long long* __restrict__ alpha_step,
                                                              unsigned long long* alpha_out, int* status,
                                                              double* clock2, double* src_keep) {
  rk_update_block<NS, STAGE, SRC>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, alpha_step, alpha_out, status, clock2,
                                  blockIdx.x, blockIdx.y, src_keep);
}

// Batched stage update over the flattened (request, block) list. Stage s
// reads S[s-1] (s = 1, 2) or S[2] (s = 3) and writes S[s] (S[0] for s = 3);
// the output alpha goes to slot s, or slot 4 for stage 3 without chemistry.
template <int NS, int STAGE>
__global__ void __launch_bounds__(UPD_BX* UPD_BY) k_rk_update_batch(const BatchReq* __restrict__ reqs,
                                                                    const int* __restrict__ first, int nreq,
                                                                    int chem) {
  const int total = first[nreq];
  for (int e = blockIdx.x; e < total; e += gridDim.x) {
    const int r = batch_owner(first, nreq, e);
    const BatchReq& q = reqs[r];
    const int local = e - first[r];
    const int out = STAGE == 3 ? 0 : STAGE;
    const int aslot = STAGE == 3 ? (chem ? 3 : 4) : STAGE;
    rk_update_block<NS, STAGE>(q.S[STAGE - 1], q.S[0], q.S[out], q.Fx, q.Gy, q.g, q.mech, q.ctl, q.alpha,
                               q.alpha + 2 * aslot, q.status, STAGE == 1 ? q.clock2 : nullptr, local % q.ubx,
                               local / q.ubx);
    __syncthreads();
  }
}

// Start of a batched step: for every request, the previous step's final
// alpha becomes the step's starting alpha (except on its first step, whose
// alpha was set when the state was loaded), and slots 1..4 are cleared.
__global__ void k_batch_prep(BatchReq* reqs, int nreq) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nreq) return;
  unsigned long long* a = reqs[r].alpha;
  if (!reqs[r].fresh) {
    a[0] = a[8];
    a[1] = a[9];
  }
  for (int k = 2; k < 10; ++k) a[k] = 0ull;
  reqs[r].fresh = 0;
}

template <int NS>
static cudaError_t launch_rk_update_batch_t(int stage, const BatchReq* reqs, const int* first, int nreq, int total,
                                            int chem, cudaStream_t st) {
  const int sms = sm_count();
  const int grid = total < sms * 8 ? total : sms * 8;
  if (grid <= 0) return cudaSuccess;
  dim3 blk(UPD_BX, UPD_BY);
  if (stage == 1) k_rk_update_batch<NS, 1><<<grid, blk, 0, st>>>(reqs, first, nreq, chem);
  else if (stage == 2) k_rk_update_batch<NS, 2><<<grid, blk, 0, st>>>(reqs, first, nreq, chem);
  else k_rk_update_batch<NS, 3><<<grid, blk, 0, st>>>(reqs, first, nreq, chem);
  return cudaGetLastError();
}

cudaError_t launch_rk_update_batch(int ns, int stage, const BatchReq* reqs, const int* first, int nreq, int total,
                                   int chem, cudaStream_t st) {
  switch (ns) {
    case 1: return launch_rk_update_batch_t<1>(stage, reqs, first, nreq, total, chem, st);
    case 3: return launch_rk_update_batch_t<3>(stage, reqs, first, nreq, total, chem, st);
    case 9: return launch_rk_update_batch_t<9>(stage, reqs, first, nreq, total, chem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_prep(BatchReq* reqs, int nreq, cudaStream_t st) {
  if (nreq <= 0) return cudaSuccess;
  k_batch_prep<<<(nreq + 127) / 128, 128, 0, st>>>(reqs, nreq);
  return cudaGetLastError();
}

void update_blocks(const GridDev& g, int* ubx, int* uby) {
  *ubx = (g.nx + UPD_BX - 1) / UPD_BX;
  *uby = (g.ny + UPD_BY - 1) / UPD_BY;
}

template <int NS>
static cudaError_t launch_rk_update_t(int stage, const StateView& Sin, const StateView& S0, const StateView& Sout,
                                      const double* Fx, const double* Gy, const GridDev& g, const MechDev* mech,
                                      const StepCtl& ctl, const unsigned long long* a_step, unsigned long long* a_out,
                                      int* status, double* clock2, cudaStream_t st, double* keep) {
  // UPD_BX x UPD_BY blocks while that gives at least 4 blocks per SM; on
  // smaller grids shorter blocks (UPD_BX x 4, 2, 1) spread the cells over
  // all SMs.
  const int sms = sm_count();
  const long long bxs = (g.nx + UPD_BX - 1) / UPD_BX;
  int by = UPD_BY;
  while (by > 1 && bxs * ((g.ny + by - 1) / by) < 4LL * sms) by /= 2;
  dim3 blk(UPD_BX, by), grd((unsigned)bxs, (g.ny + by - 1) / by);
  if (ctl.source && NS > 1) {
    if (stage == 1)
      k_rk_update<NS, 1, true><<<grd, blk, 0, st>>>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, keep);
    else if (stage == 2)
      k_rk_update<NS, 2, true><<<grd, blk, 0, st>>>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, keep);
    else
      k_rk_update<NS, 3, true><<<grd, blk, 0, st>>>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, keep);
  } else {
    if (stage == 1)
      k_rk_update<NS, 1, false><<<grd, blk, 0, st>>>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, keep);
    else if (stage == 2)
      k_rk_update<NS, 2, false><<<grd, blk, 0, st>>>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, keep);
    else
      k_rk_update<NS, 3, false><<<grd, blk, 0, st>>>(Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, keep);
  }
  return cudaGetLastError();
}

cudaError_t launch_rk_update(int ns, int stage, const StateView& Sin, const StateView& S0, const StateView& Sout,
                             const double* Fx, const double* Gy, const GridDev& g, const MechDev* mech,
                             const StepCtl& ctl, const unsigned long long* a_step, unsigned long long* a_out,
                             int* status, double* clock2, cudaStream_t st, double* src_keep) {
  switch (ns) {
    case 1: return launch_rk_update_t<1>(stage, Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, st,
                                         src_keep);
    case 3: return launch_rk_update_t<3>(stage, Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, st,
                                         src_keep);
    case 9: return launch_rk_update_t<9>(stage, Sin, S0, Sout, Fx, Gy, g, mech, ctl, a_step, a_out, status, clock2, st,
                                         src_keep);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// State set-up.
// ---------------------------------------------------------------------------
// Conserved state from T, p, u, v and all mass fractions (Eq. 4.2):
// rho = p / (R T), E = rho h - p + rho |u|^2 / 2, rho Y_k.
template <int NS>
__global__ void k_set_primitive(StateView S, const double* __restrict__ T, const double* __restrict__ p,
                                const double* __restrict__ vx, const double* __restrict__ vy,
                                const double* __restrict__ Y, GridDev g, const MechDev* __restrict__ mech,
                                unsigned long long* alpha_out, int* status) {
  constexpr int NV = NS + 3;
  const MechDev& m = *mech;
  const long long n = g.n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long sx = 0, sy = 0;
  int st = 0;
  if (idx < n) {
    const double t = T[idx], pr = p[idx], a = vx[idx], b = vy[idx];
    double W = 0.0, H = 0.0;  // sum Y_k / M_k and sum Y_k h_k / Ru
    double Yk[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      Yk[k] = Y[(long long)k * n + idx];
      const double zk = Yk[k] * m.invM[k];
      W += zk;
      const double hk = fma(t, fma(t, fma(t, fma(t, fma(t, m.hc[k][4], m.hc[k][3]), m.hc[k][2]), m.hc[k][1]),
                                   m.hc[k][0]), m.hc[k][5]);
      H = fma(zk, hk, H);
    }
    const double rho = pr * rcp(RU * W * t);
    double u[NV];
    u[0] = rho;
    u[1] = rho * a;
    u[2] = rho * b;
    u[3] = fma(rho * RU, H, -pr) + 0.5 * rho * fma(a, a, b * b);
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) u[4 + k] = rho * Yk[k];
#pragma unroll
    for (int k = 0; k < NV; ++k) S.plane(k, n)[idx] = u[k];
    // T as given; p, c from the same mixture formulas the step uses.
    double Tn, pn, c, rrho;
    st = newton_cell<NS>(u, t, m, g.newton_tol, g.newton_maxit, Tn, pn, c, rrho);
    finish_cell<NS>(S, n, idx, u, t, RU * W * rho * t, c, rrho, sx, sy);
  }
  block_reduce_alpha_status(sx, sy, st, alpha_out, status);
}

// Newton T for a loaded conserved state (warm start T0, or 1000 K).
template <int NS>
__global__ void k_set_conserved(StateView S, const double* __restrict__ T0, GridDev g,
                                const MechDev* __restrict__ mech, unsigned long long* alpha_out, int* status) {
  constexpr int NV = NS + 3;
  const long long n = g.n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long sx = 0, sy = 0;
  int st = 0;
  if (idx < n) {
    double u[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[idx];
    const double tw = T0 ? T0[idx] : 1000.0;
    double T, p, c, rrho;
    st = newton_cell<NS>(u, tw, *mech, g.newton_tol, g.newton_maxit, T, p, c, rrho);
    finish_cell<NS>(S, n, idx, u, T, p, c, rrho, sx, sy);
  }
  block_reduce_alpha_status(sx, sy, st, alpha_out, status);
}

cudaError_t launch_set_primitive(int ns, const StateView& S, const double* T, const double* p, const double* u,
                                 const double* v, const double* Y, const GridDev& g, const MechDev* mech,
                                 unsigned long long* alpha_out, int* status, cudaStream_t st) {
  const int thr = 256;
  const unsigned blocks = (unsigned)((g.n + thr - 1) / thr);
  switch (ns) {
    case 1: k_set_primitive<1><<<blocks, thr, 0, st>>>(S, T, p, u, v, Y, g, mech, alpha_out, status); break;
    case 3: k_set_primitive<3><<<blocks, thr, 0, st>>>(S, T, p, u, v, Y, g, mech, alpha_out, status); break;
    case 9: k_set_primitive<9><<<blocks, thr, 0, st>>>(S, T, p, u, v, Y, g, mech, alpha_out, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_set_conserved(int ns, const StateView& S, const double* T0, const GridDev& g, const MechDev* mech,
                                 unsigned long long* alpha_out, int* status, cudaStream_t st) {
  const int thr = 256;
  const unsigned blocks = (unsigned)((g.n + thr - 1) / thr);
  switch (ns) {
    case 1: k_set_conserved<1><<<blocks, thr, 0, st>>>(S, T0, g, mech, alpha_out, status); break;
    case 3: k_set_conserved<3><<<blocks, thr, 0, st>>>(S, T0, g, mech, alpha_out, status); break;
    case 9: k_set_conserved<9><<<blocks, thr, 0, st>>>(S, T0, g, mech, alpha_out, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Halo pack of the x-slab exchange (Sec. 4.4, Fig. 3): the 3 columns of
// every plane of S nearest each x side, into the halo layout [planes][ny][3]
// (lo_dst: columns 0..2, hi_dst: columns nx-3..nx-1; either may be null).
// Thread per (side, plane, row, column); the destinations are contiguous.
__global__ void k_halo_pack(StateView S, int planes, int nx, int ny, long long n, double* __restrict__ lo_dst,
                            double* __restrict__ hi_dst) {
  const long long per = (long long)planes * ny * 3;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2 * per) return;
  const bool hi = q >= per;
  double* dst = hi ? hi_dst : lo_dst;
  if (!dst) return;
  const long long r = hi ? q - per : q;
  const int c = (int)(r % 3);
  const long long pj = r / 3;  // plane * ny + row
  const int k = (int)(pj / ny);
  const int j = (int)(pj % ny);
  const int i = hi ? nx - 3 + c : c;
  dst[r] = S.plane(k, n)[(long long)j * nx + i];
}

cudaError_t launch_halo_pack(int planes, const StateView& S, const GridDev& g, double* lo_dst, double* hi_dst,
                             cudaStream_t st) {
  if (!lo_dst && !hi_dst) return cudaSuccess;
  const long long tot = 2LL * planes * g.ny * 3;
  k_halo_pack<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(S, planes, g.nx, g.ny, g.n, lo_dst, hi_dst);
  return cudaGetLastError();
}

__global__ void k_rhs_L(int nv, const double* __restrict__ Fx, const double* __restrict__ Gy, double* __restrict__ L,
                        GridDev g) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)nv * g.n;
  if (q >= tot) return;
  const int k = (int)(q / g.n);
  const long long idx = q % g.n;
  const int j = (int)(idx / g.nx), i = (int)(idx % g.nx);
  const double dF = Fx[((long long)k * g.ny + j) * (g.nx + 1) + i + 1] - Fx[((long long)k * g.ny + j) * (g.nx + 1) + i];
  const double dG = Gy[((long long)k * (g.ny + 1) + j + 1) * g.nx + i] - Gy[((long long)k * (g.ny + 1) + j) * g.nx + i];
  L[q] = -fma(dF, g.rdx, dG * g.rdy);
}

cudaError_t launch_rhs_L(int nv, const double* Fx, const double* Gy, double* L, const GridDev& g, cudaStream_t st) {
  const long long tot = (long long)nv * g.n;
  k_rhs_L<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nv, Fx, Gy, L, g);
  return cudaGetLastError();
}

}  // namespace janc
