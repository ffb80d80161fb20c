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
// deepest layer up (k_amr_f2c). Regridding (k_amr_mark, k_amr_flags, host
// block lists, k_amr_fill) happens every regrid_every base steps before the
// solve; a block present before and after keeps its data.
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
                                                    double dt, unsigned long long* alpha_out, int* status) {
  constexpr int NV = NS + 3;
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

struct AmrLayer {
  int nbx = 0, nby = 0;          // blocks of the layer's index space
  int nblk = 0;
  std::vector<int> pos;          // bx | by << 16, in (by, bx) order
  std::vector<int> map;          // [nby][nbx] block number or -1
  int* d_pos = nullptr;
  int* d_nbr = nullptr;
  int* d_map = nullptr;
  double* S[3] = {nullptr, nullptr, nullptr};
  double* Fx = nullptr;
  double* Gy = nullptr;
  unsigned long long* alpha = nullptr;  // 6 slots x 2
};

void free_layer_bufs(AmrLayer& L) {
  for (double*& p : L.S) { if (p) cudaFree(p); p = nullptr; }
  if (L.Fx) cudaFree(L.Fx);
  if (L.Gy) cudaFree(L.Gy);
  if (L.d_pos) cudaFree(L.d_pos);
  if (L.d_nbr) cudaFree(L.d_nbr);
  if (L.d_map) cudaFree(L.d_map);
  L.Fx = L.Gy = nullptr;
  L.d_pos = L.d_nbr = L.d_map = nullptr;
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
  int* d_oldidx = nullptr;
  size_t mask_bytes = 0, flags_bytes = 0, oldidx_count = 0;
  long long nstep = 0;
  double t = 0.0;
  long long updates_last = 0;
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

template <int NS>
cudaError_t solve_layer_t(janc_amr_s* A, int i, double dt) {
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
      k_amr_update<NS, 1><<<L.nblk, AB2, 0, st>>>(ins[s], S0, outs[s], L.Fx, L.Gy, D, P, gp.mech, dt, a + 2,
                                                  A->d_status);
    else if (s == 1)
      k_amr_update<NS, 2><<<L.nblk, AB2, 0, st>>>(ins[s], S0, outs[s], L.Fx, L.Gy, D, P, gp.mech, dt, a + 4,
                                                  A->d_status);
    else
      k_amr_update<NS, 3><<<L.nblk, AB2, 0, st>>>(ins[s], S0, outs[s], L.Fx, L.Gy, D, P, gp.mech, dt, a + 6,
                                                  A->d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && A->d.chemistry == JANC_CHEM_LIE) {
    StepCtl ctl;
    ctl.dt_fixed = dt;
    ctl.cfl = 0.0;
    ctl.hmin = 1.0;
    ctl.chem_frac = 1.0;
    ctl.source = 0;
    e = launch_chem(NS, S0, layer_grid(A, i), gp.mech, ctl, a, a + 8, A->d_status, st);
  }
  return e;
}

cudaError_t solve_layer(janc_amr_s* A, int i, double dt) {
  if (A->L[i].nblk == 0) return cudaSuccess;
  switch (A->ns) {
    case 1: return solve_layer_t<1>(A, i, dt);
    case 3: return solve_layer_t<3>(A, i, dt);
    case 9: return solve_layer_t<9>(A, i, dt);
    default: return cudaErrorInvalidValue;
  }
}

int advance(janc_amr_s* A, int i, double dt) {
  if (i < A->a.levels && A->L[i + 1].nblk > 0) {
    int rc = advance(A, i + 1, 0.5 * dt);
    if (rc == JANC_OK) rc = advance(A, i + 1, 0.5 * dt);
    if (rc != JANC_OK) return rc;
  }
  if (i == 0) return janc_step(A->g0, 1, dt, 0.0, nullptr, nullptr);
  cudaError_t e = solve_layer(A, i, dt);
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

// New block list of a layer from the flags; neighbours (periodic wrap,
// physical sides, external sides) and the position map (janc_host.h).
void build_lists(const janc_amr_s* A, const std::vector<unsigned char>& flags, AmrLayer& N, std::vector<int>& nbr) {
  janc::host::build_block_lists(flags.data(), N.nbx, N.nby, A->d.bc, N.pos, N.map, nbr);
  N.nblk = (int)N.pos.size();
}

int regrid(janc_amr_s* A) {
  const GridParts gp = grid_parts(A->g0);
  cudaStream_t st = A->stream;
  const int np = A->nv + 4;
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
    k_amr_flags<<<(ncand + 255) / 256, 256, 0, st>>>(A->d_mask, width, height, O.nbx, O.nby, A->a.n_buffer,
                                                     i >= 2 ? A->L[i - 1].d_map : nullptr, A->L[i - 1].nbx,
                                                     A->d_flags);
    e = cudaGetLastError();
    std::vector<unsigned char> flags((size_t)ncand);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags.data(), A->d_flags, (size_t)ncand, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail_cuda(e, "AMR flags");
    if (i >= 2 && A->L[i - 1].nblk == 0) std::fill(flags.begin(), flags.end(), (unsigned char)0);

    AmrLayer N;
    N.nbx = O.nbx;
    N.nby = O.nby;
    N.alpha = O.alpha;
    std::vector<int> nbr;
    build_lists(A, flags, N, nbr);
    std::vector<int> oldidx((size_t)N.nblk);
    for (int b = 0; b < N.nblk; ++b) {
      const int bx = N.pos[b] & 0xffff, by = N.pos[b] >> 16;
      oldidx[b] = O.nblk ? O.map[(size_t)by * O.nbx + bx] : -1;
    }
    const size_t cells = (size_t)N.nblk * AB2;
    e = cudaMalloc(&N.d_map, sizeof(int) * N.map.size());
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(N.d_map, N.map.data(), sizeof(int) * N.map.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && N.nblk > 0) {
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&N.S[k], sizeof(double) * np * cells);
      if (e == cudaSuccess) e = cudaMalloc(&N.Fx, sizeof(double) * A->nv * N.nblk * AB * (AB + 1));
      if (e == cudaSuccess) e = cudaMalloc(&N.Gy, sizeof(double) * A->nv * N.nblk * AB * (AB + 1));
      if (e == cudaSuccess) e = cudaMalloc(&N.d_pos, sizeof(int) * N.nblk);
      if (e == cudaSuccess) e = cudaMalloc(&N.d_nbr, sizeof(int) * 4 * N.nblk);
      if (e == cudaSuccess && (size_t)N.nblk > A->oldidx_count) {
        if (A->d_oldidx) cudaFree(A->d_oldidx);
        A->d_oldidx = nullptr;
        e = cudaMalloc(&A->d_oldidx, sizeof(int) * N.nblk);
        A->oldidx_count = e == cudaSuccess ? (size_t)N.nblk : 0;
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(N.d_pos, N.pos.data(), sizeof(int) * N.nblk, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(N.d_nbr, nbr.data(), sizeof(int) * 4 * N.nblk, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(A->d_oldidx, oldidx.data(), sizeof(int) * N.nblk, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) {
        AmrLayer keep = A->L[i];
        A->L[i] = N;  // layer_dev / parent_dev of the new list
        const LayerDev D = layer_dev(A, i);
        const ParentDev P = parent_dev(A, i);
        const StateView Sold{keep.S[0]};
        const long long n_old = (long long)keep.nblk * AB2;
        if (A->ns == 9) k_amr_fill<9><<<N.nblk, AB2, 0, st>>>(StateView{N.S[0]}, D, A->d_oldidx, Sold, n_old, P);
        else if (A->ns == 3) k_amr_fill<3><<<N.nblk, AB2, 0, st>>>(StateView{N.S[0]}, D, A->d_oldidx, Sold, n_old, P);
        else k_amr_fill<1><<<N.nblk, AB2, 0, st>>>(StateView{N.S[0]}, D, A->d_oldidx, Sold, n_old, P);
        e = cudaGetLastError();
        A->L[i] = keep;
      }
      // the old buffers are read by the fill: wait before freeing them
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    } else if (e == cudaSuccess) {
      e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
      free_layer_bufs(N);
      return afail_cuda(e, "AMR regrid");
    }
    free_layer_bufs(O);
    A->L[i] = N;
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
    A->L[i].nbx = (base->nx << i) / AB;
    A->L[i].nby = (base->ny << i) / AB;
    A->L[i].map.assign((size_t)A->L[i].nbx * A->L[i].nby, -1);
    if (e == cudaSuccess) e = cudaMalloc(&A->L[i].alpha, 12 * sizeof(unsigned long long));
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
  for (int i = 1; i <= A->a.levels; ++i) {  // layers are rebuilt at the next step
    free_layer_bufs(A->L[i]);
    A->L[i].nblk = 0;
    A->L[i].pos.clear();
    A->L[i].map.assign((size_t)A->L[i].nbx * A->L[i].nby, -1);
  }
  A->nstep = 0;
  A->t = 0.0;
  return JANC_OK;
}

int janc_amr_step(janc_amr_t A, int n_steps, double dt, double cfl, double* t_out) {
  if (!A || n_steps < 0) return afail(JANC_E_INVALID, "janc_amr_step: bad argument");
  if ((dt > 0.0) == (cfl > 0.0)) return afail(JANC_E_INVALID, "give exactly one of dt > 0 or cfl > 0");
  const GridParts gp = grid_parts(A->g0);
  cudaStream_t st = A->stream;
  const double t0 = A->t;
  for (int s = 0; s < n_steps; ++s) {
    if (A->nstep % A->a.regrid_every == 0 && A->a.levels > 0) {
      const int rc = regrid(A);
      if (rc != JANC_OK) return rc;
    }
    double h = dt;
    if (!(h > 0.0)) {  // CFL of the base layer at the step's start
      unsigned long long al[2];
      cudaError_t e = cudaMemcpyAsync(al, gp.alpha, sizeof(al), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return afail_cuda(e, "AMR alpha read");
      double ax, ay;
      std::memcpy(&ax, &al[0], 8);
      std::memcpy(&ay, &al[1], 8);
      const double hmin = A->d.dx < A->d.dy ? A->d.dx : A->d.dy;
      h = cfl * hmin / (ax > ay ? ax : ay);
    }
    int rc = JANC_OK;
    if (A->a.synchronous) {  // Fig. 2b: every layer takes this dt, deepest first
      if (!(dt > 0.0)) h = std::ldexp(h, -A->a.levels);
      for (int i = A->a.levels; i >= 1 && rc == JANC_OK; --i) {
        cudaError_t e = solve_layer(A, i, h);
        if (e != cudaSuccess) rc = afail_cuda(e, "AMR layer solve");
      }
      if (rc == JANC_OK) rc = janc_step(A->g0, 1, h, 0.0, nullptr, nullptr);
    } else {
      rc = advance(A, 0, h);
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
    A->t += h;
  }
  if (t_out) *t_out = A->t - t0;
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
  if (pos)
    for (int b = 0; b < L.nblk; ++b) {
      pos[2 * b] = L.pos[b] & 0xffff;
      pos[2 * b + 1] = L.pos[b] >> 16;
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
  if (A->d_oldidx) cudaFree(A->d_oldidx);
  if (A->g0) janc_destroy_grid(A->g0);
  delete A;
}

}  // extern "C"
