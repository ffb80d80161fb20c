// Block-structured adaptive mesh refinement of the reacting-flow step
// (arXiv 2504.13750, Sec. 3: the multi-layer blocks of Sec. 3.1, the main
// loop of Algorithm 2 and the solver of Algorithm 3).
//
// Layer 0 is an ordinary grid object (janc_step with a fixed dt). Layer i >= 1
// holds blocks of 16 x 16 cells at twice the resolution of layer i - 1, at
// fixed positions: block (bx, by) covers the layer-i cells
// [16 bx, 16 bx + 16) x [16 by, 16 by + 16), one quarter of layer-(i-1) block
// (bx / 2, by / 2). A layer's state is stored like a grid's, plane by plane
// (conserved, T, u, v, p), with the cells of block b at [256 b, 256 b + 256)
// (row-major inside the block), so the per-cell kernels (chemistry) treat a
// layer as a flat array of cells.
//
// Per layer solve (Algorithm 3), for each RK stage:
//   k_amr_flux    face fluxes of every block; the 3 ghost cells per side come
//                 from the same-layer neighbour (periodic partners included),
//                 from the physical boundary on the domain's walls and
//                 zero-gradient sides, and on external sides (no neighbour:
//                 the exterior is layer i - 1) from the block's own edge;
//   k_amr_update  stage combination and Newton T; the cells within 3 of an
//                 external side take the layer-(i-1) values instead
//                 (update_external_boundary, one-to-four copy), which are
//                 exactly the cells whose update read those ghosts;
// then the point-implicit chemistry over the layer's dt (launch_chem).
// Crossover advance (Fig. 2a): layer i + 1 takes two steps of dt / 2 before
// each step of layer i; after the base step the four-to-one mean runs from the
// deepest layer up (k_amr_f2c). Regridding (k_amr_mark, k_amr_flags, the
// block lists built on the device by k_amr_compact and k_amr_neighbours,
// k_amr_fill) happens every regrid_every base steps before the solve; a block
// present before and after keeps its data. With a CFL number the base dt is
// computed on the device from the base layer's LF speeds, and layer i's dt is
// that dt times 2^-i (exact), so a step needs no host round trip; a regrid
// reads back one block count per layer. Layer buffers grow and are never
// shrunk, so steady refinement allocates nothing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/janc.h"
#include "janc_device.cuh"
#include "janc_host.h"
#include "janc_internal.h"
#include "janc_weno.cuh"

namespace janc {

constexpr int AB = 16;            // block edge in cells
constexpr int AB2 = AB * AB;
constexpr int AH = AB / 2;        // parent cells per block edge
constexpr int NGH = 3;            // ghost cells per side = cells of the external band
constexpr int ALINES = 8;         // lines per flux tile
constexpr int AWIN = AB + 1 + 5;  // window of a line: 17 faces with the 5-point stencils
constexpr int NB_EXTERNAL = host::NB_EXTERNAL, NB_PHYSICAL = host::NB_PHYSICAL;
static_assert(host::BC_PERIODIC_CODE == BC_PERIODIC, "boundary codes of janc_host.h");

struct LayerDev {
  int nblk;
  long long n;        // nblk * 256: cell count and plane stride
  const int* pos;     // [nblk] bx | by << 16
  const int* nbr;     // [nblk][4] north, south, west, east: block, NB_EXTERNAL or NB_PHYSICAL
  double rdx, rdy, eps4, newton_tol;
  int newton_maxit;
  int bc[4];
};

// Where a cell of the parent layer lives.
struct ParentDev {
  StateView S;
  long long n;       // plane stride
  int base;          // 1: the base grid, row-major with width w
  int w;             // base: nx; layer: blocks per row of its index space
  const int* map;    // layer: block number per (by, bx), or -1
};

__device__ __forceinline__ long long parent_index(const ParentDev& P, int px, int py) {
  if (P.base) return (long long)py * P.w + px;
  const int b = P.map[(py / AB) * P.w + px / AB];
  return (long long)b * AB2 + (py % AB) * AB + (px % AB);
}

__device__ __forceinline__ bool in_band(const int* nb, int i, int j) {
  return (nb[0] == NB_EXTERNAL && j >= AB - NGH) || (nb[1] == NB_EXTERNAL && j < NGH) ||
         (nb[2] == NB_EXTERNAL && i < NGH) || (nb[3] == NB_EXTERNAL && i >= AB - NGH);
}

// ---- face fluxes of every block: 4 tiles per block (x rows 0-7, 8-15; y columns 0-7, 8-15) ----
template <int NV>
__global__ void __launch_bounds__(ALINES* NV) k_amr_flux(StateView S, const unsigned long long* __restrict__ alpha,
                                                         double* __restrict__ Fx, double* __restrict__ Gy,
                                                         LayerDev L) {
  extern __shared__ double smem[];
  double* sU = smem;                       // [NV][ALINES][AWIN]
  double* sLp = sU + NV * ALINES * AWIN;   // lambda+ = (u_n + alpha) / 2
  double* sLm = sLp + ALINES * AWIN;       // lambda- = (u_n - alpha) / 2
  double* sHp = sLm + ALINES * AWIN;       // p / 2
  double* sHpu = sHp + ALINES * AWIN;      // p u_n / 2
  const int blk = blockIdx.x >> 2;
  const int q = blockIdx.x & 3;
  const bool xdir = q < 2;
  const int l0 = (q & 1) * ALINES;
  const long long n = L.n;
  const int* nb = L.nbr + 4 * blk;
  const int lo = xdir ? nb[2] : nb[1];
  const int hi = xdir ? nb[3] : nb[0];
  const int bc_lo = xdir ? L.bc[0] : L.bc[2];
  const int bc_hi = xdir ? L.bc[1] : L.bc[3];
  const int nmom = xdir ? 1 : 2;
  const double ha = 0.5 * bitsd(alpha[xdir ? 0 : 1]);
  const double* uplane = S.plane(xdir ? NV + 1 : NV + 2, n);
  const double* pplane = S.plane(NV + 3, n);

  for (int t = threadIdx.x; t < ALINES * AWIN; t += blockDim.x) {
    int line, w;
    if (xdir) { line = t / AWIN; w = t % AWIN; } else { w = t / ALINES; line = t % ALINES; }
    const int c = w - NGH;  // -3 .. 18 along the line
    int b = blk, cc = c;
    bool flip = false;
    if (c < 0) {
      if (lo >= 0) { b = lo; cc = c + AB; }
      else if (lo == NB_PHYSICAL && bc_lo == BC_WALL) { cc = -1 - c; flip = true; }
      else cc = 0;  // zero-gradient side, or external side (its band is reset)
    } else if (c >= AB) {
      if (hi >= 0) { b = hi; cc = c - AB; }
      else if (hi == NB_PHYSICAL && bc_hi == BC_WALL) { cc = 2 * AB - 1 - c; flip = true; }
      else cc = AB - 1;
    }
    const int li = l0 + line;
    const long long idx = (long long)b * AB2 + (xdir ? li * AB + cc : cc * AB + li);
    double un = uplane[idx];
    if (flip) un = -un;
    const double hp = 0.5 * pplane[idx];
    const int o = line * AWIN + w;
    sLp[o] = fma(0.5, un, ha);
    sLm[o] = fma(0.5, un, -ha);
    sHp[o] = hp;
    sHpu[o] = hp * un;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double v = S.plane(k, n)[idx];
      if (flip && k == nmom) v = -v;
      sU[(k * ALINES + line) * AWIN + w] = v;
    }
  }
  __syncthreads();

  const int var = threadIdx.x / ALINES;
  const int line = threadIdx.x % ALINES;
  const int li = l0 + line;
  const double* Ul = sU + (var * ALINES + line) * AWIN;
  const double* pt = (var == nmom) ? sHp + line * AWIN : (var == 3 ? sHpu + line * AWIN : nullptr);
  double* out;
  long long stride;
  if (xdir) {
    out = Fx + (((long long)var * L.nblk + blk) * AB + li) * (AB + 1);
    stride = 1;
  } else {
    out = Gy + ((long long)var * L.nblk + blk) * (AB + 1) * AB + li;
    stride = AB;
  }
  slide_line2(Ul, sLp + line * AWIN, sLm + line * AWIN, pt, L.eps4, AB + 1, out, stride);
}

// ---- RK stage of every block; the external band takes the parent layer ----
template <int NS, int STAGE>
__global__ void __launch_bounds__(AB2) k_amr_update(StateView Sin, StateView S0, StateView Sout,
                                                    const double* __restrict__ Fx, const double* __restrict__ Gy,
                                                    LayerDev L, ParentDev P, const MechDev* __restrict__ mech,
                                                    StepCtl ctl, const unsigned long long* __restrict__ a_step,
                                                    unsigned long long* alpha_out, int* status) {
  constexpr int NV = NS + 3;
  const double dt = step_dt(ctl, a_step);  // the layer's dt: fixed, or from the base layer's LF speeds
  const int blk = blockIdx.x;
  const int i = threadIdx.x % AB, j = threadIdx.x / AB;
  const long long n = L.n;
  const long long idx = (long long)blk * AB2 + j * AB + i;
  double u[NV];
  double T, p, c, rrho;
  int st = 0;
  if (in_band(L.nbr + 4 * blk, i, j)) {
    const int pk = L.pos[blk];
    const long long pi = parent_index(P, ((pk & 0xffff) * AB + i) >> 1, ((pk >> 16) * AB + j) >> 1);
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = P.S.plane(k, P.n)[pi];
    T = P.S.plane(NV, P.n)[pi];
    p = P.S.plane(NV + 3, P.n)[pi];
    c = sound_speed<NS>(u, T, *mech);
    rrho = rcp(u[0]);
  } else {
    const double* fx = Fx + ((long long)blk * AB + j) * (AB + 1) + i;
    const double* gy = Gy + ((long long)blk * (AB + 1) + j) * AB + i;
    const long long sfx = (long long)L.nblk * AB * (AB + 1);
    const double cx = dt * L.rdx, cy = dt * L.rdy;  // as the grid's stage update
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double dF = fx[k * sfx + 1] - fx[k * sfx];
      const double dG = gy[k * sfx + AB] - gy[k * sfx];
      const double uin = Sin.plane(k, n)[idx];
      const double t = fma(-cx, dF, fma(-cy, dG, uin));
      if (STAGE == 1) {
        u[k] = t;
      } else {
        const double u0 = S0.plane(k, n)[idx];
        u[k] = (STAGE == 2) ? fma(0.75, u0, 0.25 * t) : fma(1.0 / 3.0, u0, (2.0 / 3.0) * t);
      }
    }
    st = newton_cell<NS>(u, Sin.plane(NV, n)[idx], *mech, L.newton_tol, L.newton_maxit, T, p, c, rrho);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) Sout.plane(k, n)[idx] = u[k];
  const double vx = u[1] * rrho, vy = u[2] * rrho;
  Sout.plane(NV, n)[idx] = T;
  Sout.plane(NV + 1, n)[idx] = vx;
  Sout.plane(NV + 2, n)[idx] = vy;
  Sout.plane(NV + 3, n)[idx] = p;
  block_reduce_alpha_status(dbits(dabs(vx) + c), dbits(dabs(vy) + c), st, alpha_out, status);
}

// ---- LF speeds of a stored state (cells [0, n)) ----
template <int NS>
__global__ void __launch_bounds__(256) k_amr_alpha(StateView S, long long n, const MechDev* __restrict__ mech,
                                                   unsigned long long* alpha_out, int* status) {
  constexpr int NV = NS + 3;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long sx = 0, sy = 0;
  if (q < n) {
    double u[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = S.plane(k, n)[q];
    const double c = sound_speed<NS>(u, S.plane(NV, n)[q], *mech);
    const double rr = rcp(u[0]);
    sx = dbits(dabs(u[1] * rr) + c);
    sy = dbits(dabs(u[2] * rr) + c);
  }
  block_reduce_alpha_status(sx, sy, 0, alpha_out, status);
}

// ---- four-to-one mean onto the parent, then Newton T and aux planes ----
// Parent cells with a child in the external band keep their own value: the
// band holds copies of the parent, not values the fine solver computed.
template <int NS>
__global__ void __launch_bounds__(AH* AH) k_amr_f2c(StateView Sf, LayerDev L, ParentDev P,
                                                    const MechDev* __restrict__ mech, double newton_tol,
                                                    int newton_maxit, int* status) {
  constexpr int NV = NS + 3;
  const int blk = blockIdx.x;
  const int a = threadIdx.x % AH, b = threadIdx.x / AH;
  const int* nb = L.nbr + 4 * blk;
  if (in_band(nb, 2 * a, 2 * b) || in_band(nb, 2 * a + 1, 2 * b) || in_band(nb, 2 * a, 2 * b + 1) ||
      in_band(nb, 2 * a + 1, 2 * b + 1))
    return;
  const int pk = L.pos[blk];
  const long long pi = parent_index(P, (pk & 0xffff) * AH + a, (pk >> 16) * AH + b);
  const long long f00 = (long long)blk * AB2 + (2 * b) * AB + 2 * a;
  const long long n = L.n;
  double u[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double* f = Sf.plane(k, n);
    u[k] = 0.25 * ((f[f00] + f[f00 + 1]) + (f[f00 + AB] + f[f00 + AB + 1]));
  }
  double T, p, c, rrho;
  const int st = newton_cell<NS>(u, P.S.plane(NV, P.n)[pi], *mech, newton_tol, newton_maxit, T, p, c, rrho);
#pragma unroll
  for (int k = 0; k < NV; ++k) P.S.plane(k, P.n)[pi] = u[k];
  P.S.plane(NV, P.n)[pi] = T;
  P.S.plane(NV + 1, P.n)[pi] = u[1] * rrho;
  P.S.plane(NV + 2, P.n)[pi] = u[2] * rrho;
  P.S.plane(NV + 3, P.n)[pi] = p;
  if (st) atomicOr(status, st);
}

// ---- refinement: |grad T| > threshold on a layer (get_refinement_grid_mask) ----
// Central differences over the layer, one-sided where the neighbouring cell is
// outside the domain or outside the layer's valid blocks; the squares and the
// sum are kept unfused so that the decision is taken in the rounding of a
// plain evaluation.
__device__ __forceinline__ bool grad_over(double tp_x, double tm_x, int dix, double tp_y, double tm_y, int djy,
                                          double dx, double dy, double thr) {
  const double gx = dix ? __ddiv_rn(tp_x - tm_x, (double)dix * dx) : 0.0;
  const double gy = djy ? __ddiv_rn(tp_y - tm_y, (double)djy * dy) : 0.0;
  return __dsqrt_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy))) > thr;
}

__global__ void k_amr_mark_base(const double* __restrict__ T, int nx, int ny, double dx, double dy, double thr,
                                unsigned char* mask) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)nx * ny) return;
  const int i = (int)(q % nx), j = (int)(q / nx);
  const int ip = min(i + 1, nx - 1), im = max(i - 1, 0);
  const int jp = min(j + 1, ny - 1), jm = max(j - 1, 0);
  const long long r = (long long)j * nx;
  mask[q] = grad_over(T[r + ip], T[r + im], ip - im, T[(long long)jp * nx + i], T[(long long)jm * nx + i], jp - jm, dx,
                      dy, thr)
                ? 1
                : 0;
}

// T of a layer cell (gx, gy) of its index space, or false when the cell is
// outside it or in no valid block.
__device__ __forceinline__ bool layer_T_at(const double* __restrict__ T, const int* __restrict__ map, int nbx, int nby,
                                           int gx, int gy, double& out) {
  if (gx < 0 || gy < 0 || gx >= nbx * AB || gy >= nby * AB) return false;
  const int b = map[(gy / AB) * nbx + gx / AB];
  if (b < 0) return false;
  out = T[(long long)b * AB2 + (gy % AB) * AB + gx % AB];
  return true;
}

__global__ void k_amr_mark_layer(const double* __restrict__ T, LayerDev L, const int* __restrict__ map, int nbx,
                                 int nby, double dx, double dy, double thr, unsigned char* mask) {
  const int blk = blockIdx.x;
  const int i = threadIdx.x % AB, j = threadIdx.x / AB;
  const int pk = L.pos[blk];
  const int gx = (pk & 0xffff) * AB + i, gy = (pk >> 16) * AB + j;
  const double tc = T[(long long)blk * AB2 + j * AB + i];
  double xp = tc, xm = tc, yp = tc, ym = tc;
  int dix = 0, djy = 0;
  if (layer_T_at(T, map, nbx, nby, gx + 1, gy, xp)) ++dix;
  if (layer_T_at(T, map, nbx, nby, gx - 1, gy, xm)) ++dix;
  if (layer_T_at(T, map, nbx, nby, gx, gy + 1, yp)) ++djy;
  if (layer_T_at(T, map, nbx, nby, gx, gy - 1, ym)) ++djy;
  mask[(long long)gy * (nbx * AB) + gx] = grad_over(xp, xm, dix, yp, ym, djy, dx, dy, thr) ? 1 : 0;
}

// A candidate block of layer i is refined when the parent-layer mask dilated
// by n_buffer (Chebyshev) meets its 8 x 8 parent region and its parent block
// is valid (get_refinement_block_mask).
__global__ void k_amr_flags(const unsigned char* __restrict__ mask, int width, int height, int nbx, int nby,
                            int nbuf, const int* __restrict__ parent_map, int parent_nbx, unsigned char* flags) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nbx * nby) return;
  const int bx = q % nbx, by = q / nbx;
  unsigned char f = 0;
  if (!parent_map || parent_map[(by / 2) * parent_nbx + bx / 2] >= 0) {
    const int x0 = max(bx * AH - nbuf, 0), x1 = min(bx * AH + AH - 1 + nbuf, width - 1);
    const int y0 = max(by * AH - nbuf, 0), y1 = min(by * AH + AH - 1 + nbuf, height - 1);
    for (int y = y0; y <= y1 && !f; ++y)
      for (int x = x0; x <= x1; ++x)
        if (mask[(long long)y * width + x]) { f = 1; break; }
  }
  flags[q] = f;
}

// New layer data: kept blocks copy their old cells, new blocks copy the parent
// one-to-four (all planes: conserved, T, u, v, p).
template <int NS>
__global__ void __launch_bounds__(AB2) k_amr_fill(StateView Snew, LayerDev L, const int* __restrict__ old_index,
                                                  StateView Sold, long long n_old, ParentDev P) {
  constexpr int NP = NS + 3 + 4;
  const int blk = blockIdx.x;
  const int i = threadIdx.x % AB, j = threadIdx.x / AB;
  const long long idx = (long long)blk * AB2 + j * AB + i;
  const int ob = old_index[blk];
  if (ob >= 0) {
    const long long oi = (long long)ob * AB2 + j * AB + i;
#pragma unroll
    for (int k = 0; k < NP; ++k) Snew.plane(k, L.n)[idx] = Sold.plane(k, n_old)[oi];
  } else {
    const int pk = L.pos[blk];
    const long long pi = parent_index(P, ((pk & 0xffff) * AB + i) >> 1, ((pk >> 16) * AB + j) >> 1);
#pragma unroll
    for (int k = 0; k < NP; ++k) Snew.plane(k, L.n)[idx] = P.S.plane(k, P.n)[pi];
  }
}

// Block list of a layer from its refinement flags, in (by, bx) order, on
// the device (one block of AMR_SCAN threads): map[cand] = the block number or
// -1, pos[b] = bx | by << 16, old_index[b] = the block's number before the
// regrid (old_map, or -1 for a new block), *count = the number of blocks.
constexpr int AMR_SCAN = 1024;
__global__ void __launch_bounds__(AMR_SCAN) k_amr_compact(const unsigned char* __restrict__ flags, int ncand, int nbx,
                                                         const int* __restrict__ old_map, int* __restrict__ map,
                                                         int* __restrict__ pos, int* __restrict__ old_index,
                                                         int* __restrict__ count) {
  __shared__ int part[AMR_SCAN];
  const int t = threadIdx.x;
  const int per = (ncand + AMR_SCAN - 1) / AMR_SCAN;
  const int c0 = min(t * per, ncand), c1 = min(c0 + per, ncand);
  int mine = 0;
  for (int c = c0; c < c1; ++c) mine += flags[c] ? 1 : 0;
  part[t] = mine;
  __syncthreads();
  // inclusive scan of the per-thread counts (Hillis-Steele)
  for (int o = 1; o < AMR_SCAN; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int b = part[t] - mine;  // this thread's first block number
  for (int c = c0; c < c1; ++c) {
    if (flags[c]) {
      map[c] = b;
      pos[b] = (c % nbx) | ((c / nbx) << 16);
      old_index[b] = old_map ? old_map[c] : -1;
      ++b;
    } else {
      map[c] = -1;
    }
  }
  if (t == AMR_SCAN - 1) *count = part[t];
}

// Neighbour table of a layer's blocks (north, south, west, east): the block
// across that side (its periodic partner on a periodic side), NB_PHYSICAL on
// a non-periodic domain side, NB_EXTERNAL where no block of the layer is
// there.
__global__ void k_amr_neighbours(const int* __restrict__ pos, const int* __restrict__ map, int nblk, int nbx, int nby,
                                 int bcl, int bcr, int bcb, int bct, int* __restrict__ nbr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 4 * nblk) return;
  const int b = q >> 2, s = q & 3;
  const int bx = pos[b] & 0xffff, by = pos[b] >> 16;
  const int dxs[4] = {0, 0, -1, 1}, dys[4] = {1, -1, 0, 0};
  const int side_bc[4] = {bct, bcb, bcl, bcr};
  int qx = bx + dxs[s], qy = by + dys[s];
  if (qx < 0 || qx >= nbx || qy < 0 || qy >= nby) {
    if (side_bc[s] != BC_PERIODIC) {
      nbr[q] = NB_PHYSICAL;
      return;
    }
    qx = (qx + nbx) % nbx;
    qy = (qy + nby) % nby;
  }
  const int m = map[qy * nbx + qx];
  nbr[q] = m >= 0 ? m : NB_EXTERNAL;
}

}  // namespace janc

using namespace janc;

// ----------------------------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------------------------
namespace {

thread_local std::string a_err;

int afail(int code, const std::string& msg) {
  a_err = msg;
  set_last_error(msg.c_str());
  return code;
}
int afail_cuda(cudaError_t e, const char* where) {
  return afail(JANC_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// One refined layer. The index buffers (positions, neighbours, old block
// numbers, two position maps used in turn by consecutive regrids) are sized
// for every candidate block of the layer's index space once, at creation.
// The state and face-flux buffers hold `cap` blocks and grow (never shrink)
// when a regrid needs more; a state is stored with plane stride nblk * 256
// inside them. `spare` receives the regridded state, then trades places
// with S[0].
struct AmrLayer {
  int nbx = 0, nby = 0;          // blocks of the layer's index space
  int nblk = 0;
  int cap = 0;                   // blocks the state and flux buffers hold
  int cur = 0;                   // d_mapv[cur] is the current position map
  int* d_pos = nullptr;          // [nbx nby] bx | by << 16, in (by, bx) order
  int* d_nbr = nullptr;          // [4 nbx nby]
  int* d_oldidx = nullptr;       // [nbx nby]
  int* d_mapv[2] = {nullptr, nullptr};  // [nby][nbx] block number or -1
  int* d_count = nullptr;
  int* d_map = nullptr;          // = d_mapv[cur]
  double* S[3] = {nullptr, nullptr, nullptr};
  double* spare = nullptr;
  double* Fx = nullptr;
  double* Gy = nullptr;
  unsigned long long* alpha = nullptr;  // 6 slots x 2
};

void free_state_bufs(AmrLayer& L) {
  for (double*& p : L.S) { if (p) cudaFree(p); p = nullptr; }
  if (L.spare) cudaFree(L.spare);
  if (L.Fx) cudaFree(L.Fx);
  if (L.Gy) cudaFree(L.Gy);
  L.spare = L.Fx = L.Gy = nullptr;
  L.cap = 0;
}

void free_layer_bufs(AmrLayer& L) {
  free_state_bufs(L);
  for (int* p : {L.d_pos, L.d_nbr, L.d_oldidx, L.d_mapv[0], L.d_mapv[1], L.d_count})
    if (p) cudaFree(p);
  L.d_pos = L.d_nbr = L.d_oldidx = L.d_mapv[0] = L.d_mapv[1] = L.d_count = L.d_map = nullptr;
}

}  // namespace

struct janc_amr_s {
  janc_grid_t g0 = nullptr;
  janc_grid_desc d;
  janc_amr_desc a;
  int ns = 0, nv = 0;
  cudaStream_t stream = nullptr;
  std::vector<AmrLayer> L;           // index 1..levels used
  unsigned char* d_mask = nullptr;   // largest parent index space
  unsigned char* d_flags = nullptr;  // largest candidate set
  int* d_status = nullptr;
  size_t mask_bytes = 0, flags_bytes = 0;
  long long nstep = 0;
  long long updates_last = 0;
  long long grow_events = 0;         // regrids that had to enlarge a layer's buffers
};

namespace {

LayerDev layer_dev(const janc_amr_s* A, int i) {
  const AmrLayer& L = A->L[i];
  const GridParts gp = grid_parts(A->g0);
  LayerDev D;
  D.nblk = L.nblk;
  D.n = (long long)L.nblk * AB2;
  D.pos = L.d_pos;
  D.nbr = L.d_nbr;
  const double s = std::ldexp(1.0, i);
  D.rdx = s / A->d.dx;
  D.rdy = s / A->d.dy;
  D.eps4 = gp.gd.eps4;
  D.newton_tol = gp.gd.newton_tol;
  D.newton_maxit = gp.gd.newton_maxit;
  for (int k = 0; k < 4; ++k) D.bc[k] = A->d.bc[k];
  return D;
}

ParentDev parent_dev(const janc_amr_s* A, int i) {  // the parent of layer i
  ParentDev P;
  if (i == 1) {
    const GridParts gp = grid_parts(A->g0);
    P.S = gp.S0;
    P.n = gp.gd.n;
    P.base = 1;
    P.w = gp.gd.nx;
    P.map = nullptr;
  } else {
    const AmrLayer& Q = A->L[i - 1];
    P.S = StateView{Q.S[0]};
    P.n = (long long)Q.nblk * AB2;
    P.base = 0;
    P.w = Q.nbx;
    P.map = Q.d_map;
  }
  return P;
}

GridDev layer_grid(const janc_amr_s* A, int i) {  // for the per-cell chemistry kernel
  GridDev g = grid_parts(A->g0).gd;
  const double s = std::ldexp(1.0, i);
  g.nx = AB;
  g.ny = AB * A->L[i].nblk;
  g.n = (long long)A->L[i].nblk * AB2;
  g.dx = A->d.dx / s;
  g.dy = A->d.dy / s;
  g.rdx = s / A->d.dx;
  g.rdy = s / A->d.dy;
  return g;
}

cudaError_t launch_alpha(int ns, const StateView& S, long long n, const MechDev* mech, unsigned long long* out,
                         int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  switch (ns) {
    case 1: k_amr_alpha<1><<<blocks, 256, 0, st>>>(S, n, mech, out, status); break;
    case 3: k_amr_alpha<3><<<blocks, 256, 0, st>>>(S, n, mech, out, status); break;
    case 9: k_amr_alpha<9><<<blocks, 256, 0, st>>>(S, n, mech, out, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// lc: the layer's step control, a fixed dt or the CFL number with the
// layer's scaled spacing, so that step_dt() of the base layer's LF speeds
// gives this layer's dt on the device.
template <int NS>
cudaError_t solve_layer_t(janc_amr_s* A, int i, const StepCtl& lc) {
  constexpr int NV = NS + 3;
  AmrLayer& L = A->L[i];
  const GridParts gp = grid_parts(A->g0);
  cudaStream_t st = A->stream;
  const LayerDev D = layer_dev(A, i);
  const ParentDev P = parent_dev(A, i);
  const StateView S0{L.S[0]}, S1{L.S[1]}, S2{L.S[2]};
  unsigned long long* a = L.alpha;
  cudaError_t e = cudaMemsetAsync(a, 0, 12 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_alpha(NS, S0, D.n, gp.mech, a, A->d_status, st);
  const size_t smem = sizeof(double) * (NV + 4) * ALINES * AWIN;
  const unsigned ftiles = 4u * (unsigned)L.nblk;
  const StateView ins[3] = {S0, S1, S2};
  const StateView outs[3] = {S1, S2, S0};
  for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
    k_amr_flux<NV><<<ftiles, ALINES * NV, smem, st>>>(ins[s], a + 2 * s, L.Fx, L.Gy, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    if (s == 0)
      k_amr_update<NS, 1><<<L.nblk, AB2, 0, st>>>(ins[s], S0, outs[s], L.Fx, L.Gy, D, P, gp.mech, lc, gp.alpha, a + 2,
                                                  A->d_status);
    else if (s == 1)
      k_amr_update<NS, 2><<<L.nblk, AB2, 0, st>>>(ins[s], S0, outs[s], L.Fx, L.Gy, D, P, gp.mech, lc, gp.alpha, a + 4,
                                                  A->d_status);
    else
      k_amr_update<NS, 3><<<L.nblk, AB2, 0, st>>>(ins[s], S0, outs[s], L.Fx, L.Gy, D, P, gp.mech, lc, gp.alpha, a + 6,
                                                  A->d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && A->d.chemistry == JANC_CHEM_LIE)
    e = launch_chem(NS, S0, layer_grid(A, i), gp.mech, lc, gp.alpha, a + 8, A->d_status, st);
  return e;
}

cudaError_t solve_layer(janc_amr_s* A, int i, const StepCtl& lc) {
  if (A->L[i].nblk == 0) return cudaSuccess;
  switch (A->ns) {
    case 1: return solve_layer_t<1>(A, i, lc);
    case 3: return solve_layer_t<3>(A, i, lc);
    case 9: return solve_layer_t<9>(A, i, lc);
    default: return cudaErrorInvalidValue;
  }
}

// Step control of a layer whose dt is 2^-k times the given one: a fixed dt
// halves, a CFL dt halves through the spacing (exact in floating point).
StepCtl halved(StepCtl c, int k) {
  if (c.dt_fixed > 0.0) c.dt_fixed = std::ldexp(c.dt_fixed, -k);
  else c.hmin = std::ldexp(c.hmin, -k);
  return c;
}

// Crossover advance of layer i and everything finer (Fig. 2a): two steps of
// the next layer per step of this one. The base layer (i = 0) steps through
// janc_step with the same dt (its CFL dt is computed the same way).
int advance(janc_amr_s* A, int i, const StepCtl& c) {
  if (i < A->a.levels && A->L[i + 1].nblk > 0) {
    const StepCtl f = halved(c, 1);
    int rc = advance(A, i + 1, f);
    if (rc == JANC_OK) rc = advance(A, i + 1, f);
    if (rc != JANC_OK) return rc;
  }
  if (i == 0) return janc_step(A->g0, 1, c.dt_fixed, c.dt_fixed > 0.0 ? 0.0 : c.cfl, nullptr, nullptr);
  cudaError_t e = solve_layer(A, i, c);
  return e == cudaSuccess ? JANC_OK : afail_cuda(e, "AMR layer solve");
}

template <int NS>
cudaError_t f2c_t(janc_amr_s* A, int i) {
  const GridParts gp = grid_parts(A->g0);
  k_amr_f2c<NS><<<A->L[i].nblk, AH * AH, 0, A->stream>>>(StateView{A->L[i].S[0]}, layer_dev(A, i), parent_dev(A, i),
                                                          gp.mech, gp.gd.newton_tol, gp.gd.newton_maxit,
                                                          A->d_status);
  return cudaGetLastError();
}

// Enlarges a layer's state and flux buffers to hold at least `need` blocks
// (about 1.25 x need, so that a slowly growing layer does not reallocate at
// every regrid). S[0] keeps its data; the other buffers hold nothing yet.
cudaError_t grow_layer(janc_amr_s* A, AmrLayer& L, int need) {
  const int cap = std::max(need, need + need / 4);
  const int np = A->nv + 4;
  const size_t cells = (size_t)cap * AB2;
  double* S0 = nullptr;
  cudaError_t e = cudaMalloc(&S0, sizeof(double) * np * cells);
  // S[0] holds the layer's current data: copy the nblk blocks into the new one
  if (e == cudaSuccess && L.nblk > 0)
    e = cudaMemcpyAsync(S0, L.S[0], sizeof(double) * np * (size_t)L.nblk * AB2, cudaMemcpyDeviceToDevice, A->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(A->stream);
  if (e != cudaSuccess) {
    if (S0) cudaFree(S0);
    return e;
  }
  free_state_bufs(L);
  L.S[0] = S0;
  for (int k = 1; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&L.S[k], sizeof(double) * np * cells);
  if (e == cudaSuccess) e = cudaMalloc(&L.spare, sizeof(double) * np * cells);
  if (e == cudaSuccess) e = cudaMalloc(&L.Fx, sizeof(double) * A->nv * (size_t)cap * AB * (AB + 1));
  if (e == cudaSuccess) e = cudaMalloc(&L.Gy, sizeof(double) * A->nv * (size_t)cap * AB * (AB + 1));
  if (e == cudaSuccess) L.cap = cap;
  ++A->grow_events;
  return e;
}

int regrid(janc_amr_s* A) {
  const GridParts gp = grid_parts(A->g0);
  cudaStream_t st = A->stream;
  for (int i = 1; i <= A->a.levels; ++i) {
    AmrLayer& O = A->L[i];
    // mask of layer i-1 in its index space
    const int width = A->d.nx << (i - 1), height = A->d.ny << (i - 1);
    const double s = std::ldexp(1.0, i - 1);
    const double dx = A->d.dx / s, dy = A->d.dy / s;
    cudaError_t e = cudaMemsetAsync(A->d_mask, 0, (size_t)width * height, st);
    if (e != cudaSuccess) return afail_cuda(e, "AMR mask clear");
    if (i == 1) {
      const long long nc = (long long)width * height;
      k_amr_mark_base<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(gp.S0.plane(A->nv, gp.gd.n), width, height, dx,
                                                                    dy, A->a.threshold, A->d_mask);
    } else if (A->L[i - 1].nblk > 0) {
      const LayerDev Dp = layer_dev(A, i - 1);
      k_amr_mark_layer<<<A->L[i - 1].nblk, AB2, 0, st>>>(StateView{A->L[i - 1].S[0]}.plane(A->nv, Dp.n), Dp,
                                                         A->L[i - 1].d_map, A->L[i - 1].nbx, A->L[i - 1].nby, dx,
                                                         dy, A->a.threshold, A->d_mask);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return afail_cuda(e, "AMR mask");
    const int ncand = O.nbx * O.nby;
    if (i >= 2 && A->L[i - 1].nblk == 0) {
      e = cudaMemsetAsync(A->d_flags, 0, (size_t)ncand, st);  // no parent blocks: nothing can refine
    } else {
      k_amr_flags<<<(ncand + 255) / 256, 256, 0, st>>>(A->d_mask, width, height, O.nbx, O.nby, A->a.n_buffer,
                                                       i >= 2 ? A->L[i - 1].d_map : nullptr, A->L[i - 1].nbx,
                                                       A->d_flags);
      e = cudaGetLastError();
    }
    // the new block list, from the flags, on the device; only the count comes back
    const int nxt = O.cur ^ 1;
    if (e == cudaSuccess)
      k_amr_compact<<<1, AMR_SCAN, 0, st>>>(A->d_flags, ncand, O.nbx, O.nblk > 0 ? O.d_map : nullptr, O.d_mapv[nxt],
                                           O.d_pos, O.d_oldidx, O.d_count);
    if (e == cudaSuccess) e = cudaGetLastError();
    int nblk = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nblk, O.d_count, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail_cuda(e, "AMR block list");
    if (nblk > 0) {
      if (nblk > O.cap) {
        e = grow_layer(A, O, nblk);
        if (e != cudaSuccess) return afail_cuda(e, "AMR layer buffers");
      }
      k_amr_neighbours<<<(4 * nblk + 255) / 256, 256, 0, st>>>(O.d_pos, O.d_mapv[nxt], nblk, O.nbx, O.nby, A->d.bc[0],
                                                              A->d.bc[1], A->d.bc[2], A->d.bc[3], O.d_nbr);
      e = cudaGetLastError();
      // kept blocks copy their old cells, new ones their parent (into the spare state)
      const int nblk_old = O.nblk;
      O.nblk = nblk;
      O.d_map = O.d_mapv[nxt];
      const LayerDev D = layer_dev(A, i);
      const ParentDev P = parent_dev(A, i);
      const StateView Sold{O.S[0]};
      const long long n_old = (long long)nblk_old * AB2;
      if (e == cudaSuccess) {
        if (A->ns == 9) k_amr_fill<9><<<nblk, AB2, 0, st>>>(StateView{O.spare}, D, O.d_oldidx, Sold, n_old, P);
        else if (A->ns == 3) k_amr_fill<3><<<nblk, AB2, 0, st>>>(StateView{O.spare}, D, O.d_oldidx, Sold, n_old, P);
        else k_amr_fill<1><<<nblk, AB2, 0, st>>>(StateView{O.spare}, D, O.d_oldidx, Sold, n_old, P);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) return afail_cuda(e, "AMR regrid");
      std::swap(O.S[0], O.spare);
    } else {
      O.nblk = 0;
      O.d_map = O.d_mapv[nxt];
    }
    O.cur = nxt;
  }
  return JANC_OK;
}

}  // namespace

extern "C" {

int janc_amr_create(const janc_grid_desc* base, const janc_mechanism* m, const janc_amr_desc* a, void* cuda_stream,
                    janc_amr_t* out) {
  if (!base || !m || !a || !out) return afail(JANC_E_INVALID, "janc_amr_create: null argument");
  if (a->block != AB) return afail(JANC_E_UNSUPPORTED, "janc_amr_create: block must be 16");
  if (a->levels < 0 || a->levels > 6) return afail(JANC_E_INVALID, "janc_amr_create: levels must be 0..6");
  if (a->n_buffer < 0 || a->regrid_every <= 0) return afail(JANC_E_INVALID, "janc_amr_create: bad buffer or period");
  if (base->nx % AH || base->ny % AH) return afail(JANC_E_INVALID, "janc_amr_create: nx, ny must be multiples of 8");
  if (base->chemistry == JANC_CHEM_STRANG || base->chemistry == JANC_CHEM_EXPLICIT)
    return afail(JANC_E_UNSUPPORTED, "janc_amr_create: Lie order only");
  if (((long long)base->nx << a->levels) > 65535 || ((long long)base->ny << a->levels) > 65535 * AB)
    return afail(JANC_E_INVALID, "janc_amr_create: finest index space too large");
  janc_amr_s* A = new janc_amr_s();
  A->d = *base;
  A->a = *a;
  int rc = janc_create_grid(base, m, nullptr, 0, cuda_stream, &A->g0);
  if (rc != JANC_OK) {
    delete A;
    return rc;
  }
  const GridParts gp = grid_parts(A->g0);
  A->ns = gp.ns;
  A->nv = gp.nv;
  A->stream = gp.stream;
  A->L.resize(a->levels + 1);
  cudaError_t e = cudaSuccess;
  for (int i = 1; i <= a->levels; ++i) {
    AmrLayer& L = A->L[i];
    L.nbx = (base->nx << i) / AB;
    L.nby = (base->ny << i) / AB;
    const size_t ncand = (size_t)L.nbx * L.nby;
    if (e == cudaSuccess) e = cudaMalloc(&L.alpha, 12 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&L.d_pos, sizeof(int) * ncand);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_nbr, sizeof(int) * 4 * ncand);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_oldidx, sizeof(int) * ncand);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaMalloc(&L.d_mapv[k], sizeof(int) * ncand);
      if (e == cudaSuccess) e = cudaMemsetAsync(L.d_mapv[k], 0xff, sizeof(int) * ncand, A->stream);  // -1
    }
    if (e == cudaSuccess) e = cudaMalloc(&L.d_count, sizeof(int));
    L.d_map = L.d_mapv[0];
    A->flags_bytes = std::max(A->flags_bytes, (size_t)A->L[i].nbx * A->L[i].nby);
    A->mask_bytes = std::max(A->mask_bytes, ((size_t)base->nx << (i - 1)) * ((size_t)base->ny << (i - 1)));
  }
  if (e == cudaSuccess && a->levels > 0) e = cudaMalloc(&A->d_mask, A->mask_bytes);
  if (e == cudaSuccess && a->levels > 0) e = cudaMalloc(&A->d_flags, A->flags_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&A->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(A->d_status, 0, sizeof(int), A->stream);
  if (e != cudaSuccess) {
    janc_amr_destroy(A);
    return afail_cuda(e, "janc_amr_create");
  }
  *out = A;
  return JANC_OK;
}

int janc_amr_set_state_primitive(janc_amr_t A, const double* T, const double* p, const double* u, const double* v,
                                 const double* Y, int where) {
  if (!A) return afail(JANC_E_INVALID, "null AMR object");
  const int rc = janc_set_state_primitive(A->g0, T, p, u, v, Y, where);
  if (rc != JANC_OK) return rc;
  for (int i = 1; i <= A->a.levels; ++i) A->L[i].nblk = 0;  // rebuilt at the next step (buffers kept)
  A->nstep = 0;
  return JANC_OK;
}

int janc_amr_step(janc_amr_t A, int n_steps, double dt, double cfl, double* t_out) {
  if (!A || n_steps < 0) return afail(JANC_E_INVALID, "janc_amr_step: bad argument");
  if ((dt > 0.0) == (cfl > 0.0)) return afail(JANC_E_INVALID, "give exactly one of dt > 0 or cfl > 0");
  const GridParts gp = grid_parts(A->g0);
  cudaStream_t st = A->stream;
  double t0 = 0.0;
  if (t_out) {  // the base grid's clock advances by every base step's dt
    janc_status_info si;
    const int rc = janc_status(A->g0, &si);
    if (rc != JANC_OK) return rc;
    t0 = si.t;
  }
  // the base step's control: a fixed dt, or the CFL of the base layer's LF
  // speeds at the step's start, computed on the device by every kernel
  StepCtl c;
  c.dt_fixed = dt > 0.0 ? dt : 0.0;
  c.cfl = dt > 0.0 ? 0.0 : cfl;
  c.hmin = A->d.dx < A->d.dy ? A->d.dx : A->d.dy;
  c.chem_frac = 1.0;
  c.source = 0;
  for (int s = 0; s < n_steps; ++s) {
    if (A->nstep % A->a.regrid_every == 0 && A->a.levels > 0) {
      const int rc = regrid(A);
      if (rc != JANC_OK) return rc;
    }
    int rc = JANC_OK;
    if (A->a.synchronous) {  // Fig. 2b: every layer takes this dt, deepest first
      // a fixed dt as given; the CFL dt of the base layer over 2^levels
      const StepCtl cs = c.dt_fixed > 0.0 ? c : halved(c, A->a.levels);
      for (int i = A->a.levels; i >= 1 && rc == JANC_OK; --i) {
        cudaError_t e = solve_layer(A, i, cs);
        if (e != cudaSuccess) rc = afail_cuda(e, "AMR layer solve");
      }
      if (rc == JANC_OK)
        rc = janc_step(A->g0, 1, cs.dt_fixed, cs.dt_fixed > 0.0 ? 0.0 : std::ldexp(cfl, -A->a.levels), nullptr,
                       nullptr);
    } else {
      rc = advance(A, 0, c);
    }
    if (rc != JANC_OK) return rc;
    cudaError_t e = cudaSuccess;
    for (int i = A->a.levels; i >= 1 && e == cudaSuccess; --i)
      if (A->L[i].nblk > 0) e = A->ns == 9 ? f2c_t<9>(A, i) : (A->ns == 3 ? f2c_t<3>(A, i) : f2c_t<1>(A, i));
    // the base state changed under the layers: its LF speeds for the next step
    if (e == cudaSuccess) e = cudaMemsetAsync(gp.alpha, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_alpha(A->ns, gp.S0, gp.gd.n, gp.mech, gp.alpha, A->d_status, st);
    if (e != cudaSuccess) return afail_cuda(e, "AMR fine-to-coarse");
    long long up = (long long)A->d.nx * A->d.ny;
    for (int i = 1; i <= A->a.levels; ++i) up += ((long long)A->L[i].nblk * AB2) << (A->a.synchronous ? 0 : i);
    A->updates_last = up;
    A->nstep += 1;
  }
  if (t_out) {
    janc_status_info si;
    const int rc = janc_status(A->g0, &si);
    if (rc != JANC_OK) return rc;
    *t_out = si.t - t0;
  }
  return JANC_OK;
}

int janc_amr_block_lists(const unsigned char* flags, int nbx, int nby, const int* bc, int* pos, int* map, int* nbr,
                         int* nblk) {
  if (!flags || !bc || !pos || !map || !nbr || !nblk || nbx < 1 || nby < 1 || nbx > 65535 || nby > 65535)
    return afail(JANC_E_INVALID, "janc_amr_block_lists: bad argument");
  const size_t nc = (size_t)nbx * nby;
  unsigned char* d_flags = nullptr;
  int *d_map = nullptr, *d_pos = nullptr, *d_old = nullptr, *d_nbr = nullptr, *d_count = nullptr;
  cudaError_t e = cudaMalloc(&d_flags, nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_map, sizeof(int) * nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_pos, sizeof(int) * nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_old, sizeof(int) * nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_nbr, sizeof(int) * 4 * nc);
  if (e == cudaSuccess) e = cudaMalloc(&d_count, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(d_flags, flags, nc, cudaMemcpyHostToDevice);
  int n = 0;
  if (e == cudaSuccess) {
    k_amr_compact<<<1, AMR_SCAN>>>(d_flags, (int)nc, nbx, nullptr, d_map, d_pos, d_old, d_count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&n, d_count, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && n > 0) {
    k_amr_neighbours<<<(4 * n + 255) / 256, 256>>>(d_pos, d_map, n, nbx, nby, bc[0], bc[1], bc[2], bc[3], d_nbr);
    e = cudaGetLastError();
  }
  std::vector<int> pk((size_t)n);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(pk.data(), d_pos, sizeof(int) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(map, d_map, sizeof(int) * nc, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(nbr, d_nbr, sizeof(int) * 4 * n, cudaMemcpyDeviceToHost);
  for (void* p : {(void*)d_flags, (void*)d_map, (void*)d_pos, (void*)d_old, (void*)d_nbr, (void*)d_count})
    if (p) cudaFree(p);
  if (e != cudaSuccess) return afail_cuda(e, "janc_amr_block_lists");
  for (int b = 0; b < n; ++b) {
    pos[2 * b] = pk[b] & 0xffff;
    pos[2 * b + 1] = pk[b] >> 16;
  }
  *nblk = n;
  return JANC_OK;
}

int janc_amr_layer_blocks(janc_amr_t A, int level, int* nblk) {
  if (!A || !nblk || level < 1 || level > A->a.levels) return afail(JANC_E_INVALID, "janc_amr_layer_blocks");
  *nblk = A->L[level].nblk;
  return JANC_OK;
}

int janc_amr_get_layer(janc_amr_t A, int level, int* pos, double* U, double* T) {
  if (!A || level < 1 || level > A->a.levels) return afail(JANC_E_INVALID, "janc_amr_get_layer");
  const AmrLayer& L = A->L[level];
  if (pos && L.nblk > 0) {
    std::vector<int> pk((size_t)L.nblk);
    cudaError_t e = cudaMemcpyAsync(pk.data(), L.d_pos, sizeof(int) * L.nblk, cudaMemcpyDeviceToHost, A->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(A->stream);
    if (e != cudaSuccess) return afail_cuda(e, "janc_amr_get_layer");
    for (int b = 0; b < L.nblk; ++b) {
      pos[2 * b] = pk[b] & 0xffff;
      pos[2 * b + 1] = pk[b] >> 16;
    }
  }
  if (L.nblk == 0 || (!U && !T)) return JANC_OK;
  const size_t cells = (size_t)L.nblk * AB2;
  std::vector<double> h((size_t)(A->nv + 1) * cells);
  cudaError_t e = cudaMemcpyAsync(h.data(), L.S[0], sizeof(double) * h.size(), cudaMemcpyDeviceToHost, A->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(A->stream);
  if (e != cudaSuccess) return afail_cuda(e, "janc_amr_get_layer");
  for (int b = 0; b < L.nblk; ++b)
    for (int q = 0; q < AB2; ++q) {
      if (U)
        for (int k = 0; k < A->nv; ++k) U[((size_t)b * A->nv + k) * AB2 + q] = h[(size_t)k * cells + (size_t)b * AB2 + q];
      if (T) T[(size_t)b * AB2 + q] = h[(size_t)A->nv * cells + (size_t)b * AB2 + q];
    }
  return JANC_OK;
}

int janc_amr_get_base(janc_amr_t A, double* U, double* T, int where) {
  if (!A) return afail(JANC_E_INVALID, "null AMR object");
  return janc_get_state(A->g0, U, T, where);
}

int janc_amr_status(janc_amr_t A, int* status) {
  if (!A || !status) return afail(JANC_E_INVALID, "janc_amr_status");
  int s = 0;
  cudaError_t e = cudaMemcpyAsync(&s, A->d_status, sizeof(int), cudaMemcpyDeviceToHost, A->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(A->stream);
  if (e != cudaSuccess) return afail_cuda(e, "janc_amr_status");
  janc_status_info gi;
  const int rc = janc_status(A->g0, &gi);
  if (rc != JANC_OK) return rc;
  *status = s | gi.status;
  return JANC_OK;
}

int janc_amr_cell_updates(janc_amr_t A, long long* per_step) {
  if (!A || !per_step) return afail(JANC_E_INVALID, "janc_amr_cell_updates");
  *per_step = A->updates_last;
  return JANC_OK;
}

void janc_amr_destroy(janc_amr_t A) {
  if (!A) return;
  if (A->stream) cudaStreamSynchronize(A->stream);
  for (size_t i = 1; i < A->L.size(); ++i) {
    free_layer_bufs(A->L[i]);
    if (A->L[i].alpha) cudaFree(A->L[i].alpha);
  }
  if (A->d_mask) cudaFree(A->d_mask);
  if (A->d_flags) cudaFree(A->d_flags);
  if (A->d_status) cudaFree(A->d_status);
  if (A->g0) janc_destroy_grid(A->g0);
  delete A;
}

}  // extern "C"
