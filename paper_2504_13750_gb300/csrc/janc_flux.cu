// Face fluxes of the conservative finite-difference scheme (arXiv 2504.13750,
// Eq. 4.10): global Lax-Friedrichs flux-vector splitting (Eq. 4.11) and
// WENO5 reconstruction of F+ and F- at every cell face, with the 3 ghost
// layers of the text after Eq. 4.11 produced on the fly during the tile load.
//
// One launch covers both directions: blocks [0, nbx) take x-face tiles and the
// rest take y-face tiles. A tile is LINES grid lines (rows for x, columns for
// y) by 32 consecutive faces along them (16 or 8 on grids too small to fill
// the GPU with 32-face tiles; the batched launch always uses 32). Its cells,
// with the 5-cell stencil
// margin, are staged in shared memory once; every thread then owns one
// (line, variable) and slides two 5-point windows (F+ and F-) along its line,
// so the first and second differences and the 13/3 S^2 part of the
// smoothness indicators are computed once per point instead of once per
// face, and each thread carries two independent dependency chains.
//
// Per face and sign the reconstruction costs 27 FP64 instructions plus 5 per
// new point (Jiang-Shu weights in divide-free form, one reciprocal).
#include <atomic>

#include "janc_device.cuh"
#include "janc_internal.h"
#include "janc_weno.cuh"

namespace janc {

constexpr int LINES = 8;
constexpr int FACES = 32;  // faces per tile of the batched launch and of large grids

// One tile of the face-flux launch (FC faces per line); `blk` is the tile's
// index in the launch (x tiles first). Shared by the single-grid and the
// batched kernels. HALO: the grid is a slab of an x-slab decomposition and
// the ghost columns of its BC_HALO sides come from the halo buffers.
// LIN: also store the reconstructions' derivatives (slide_line2_lin) in
// `lin`: x faces [8][NV][nx + 1][ny], then y faces [8][NV][ny + 1][nx]
// (line index fastest, so a warp's stores are contiguous per variable).
template <int NV, int FC = FACES, bool HALO = false, bool LIN = false>
__device__ __forceinline__ void face_flux_tile(const StateView& S, const unsigned long long* __restrict__ alpha,
                                               double* __restrict__ Fx, double* __restrict__ Gy, const GridDev& g,
                                               int blk, int nbx, int ntx_x, int ntx_y, double* smem,
                                               double* __restrict__ lin = nullptr) {
  constexpr int WIN = FC + 5;
  double* sU = smem;                       // [NV][LINES][WIN]
  double* sLp = sU + NV * LINES * WIN;     // lambda+ = (u_n + alpha) / 2
  double* sLm = sLp + LINES * WIN;         // lambda- = (u_n - alpha) / 2
  double* sHp = sLm + LINES * WIN;         // p / 2
  double* sHpu = sHp + LINES * WIN;        // p u_n / 2

  const bool xdir = blk < nbx;
  const int tile = xdir ? blk : blk - nbx;
  const int ntl = xdir ? ntx_x : ntx_y;
  const int ta = tile % ntl;
  const int tb = tile / ntl;
  const long long n = g.n;
  const int nx = g.nx, ny = g.ny;
  // x tiles: faces along x (ta), rows (tb). y tiles: columns (ta), faces along y (tb).
  const int f0 = xdir ? ta * FC : tb * FC;
  const int l0 = xdir ? tb * LINES : ta * LINES;
  const int nlines = xdir ? ny : nx;          // number of lines in the domain
  const int nfaces = (xdir ? nx : ny) + 1;    // faces per line
  const int ncell = xdir ? nx : ny;           // cells along a line
  const int bc_lo = xdir ? g.bc[0] : g.bc[2];
  const int bc_hi = xdir ? g.bc[1] : g.bc[3];
  const int nmom = xdir ? 1 : 2;  // wall-normal momentum plane
  const double alph = bitsd(alpha[xdir ? 0 : 1]);
  const double ha = 0.5 * alph;
  const int uk = xdir ? NV + 1 : NV + 2;  // plane of the face-normal velocity

  // ---- stage the tile: LINES x WIN cells, ghosts mapped on the fly ----
  const int nthr = blockDim.x;
  for (int q = threadIdx.x; q < LINES * WIN; q += nthr) {
    int line, w;
    if (xdir) { line = q / WIN; w = q % WIN; } else { w = q / LINES; line = q % LINES; }
    int lg = l0 + line;
    if (lg >= nlines) lg = nlines - 1;  // inactive line: any valid cell
    int cg = f0 - 3 + w;
    if (cg > ncell + 2) cg = ncell + 2;   // beyond the last needed ghost: clamp
    bool flip;
    const double* base = S.base;  // planes of `base` are `ps` apart
    long long ps = n, idx;
    if (HALO && xdir && ((cg < 0 && bc_lo == BC_HALO) || (cg >= ncell && bc_hi == BC_HALO))) {
      // a ghost column of a side shared with the neighbouring slab
      const bool lo = cg < 0;
      base = lo ? g.halo_lo : g.halo_hi;
      ps = 3LL * nlines;
      idx = (long long)lg * 3 + (lo ? cg + 3 : cg - ncell);
      flip = false;
    } else {
      const int src = ghost_src(cg, ncell, bc_lo, bc_hi, flip);
      idx = xdir ? (long long)lg * nx + src : (long long)src * nx + lg;
    }
    double un = base[uk * ps + idx];
    if (flip) un = -un;
    const double hp = 0.5 * base[(NV + 3) * ps + idx];
    const int o = line * WIN + w;
    sLp[o] = fma(0.5, un, ha);
    sLm[o] = fma(0.5, un, -ha);
    sHp[o] = hp;
    sHpu[o] = hp * un;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double v = base[k * ps + idx];
      if (flip && k == nmom) v = -v;
      sU[(k * LINES + line) * WIN + w] = v;
    }
  }
  __syncthreads();

  // ---- reconstruct and store: thread = (variable, line), both signs ----
  const int nf = min(FC, nfaces - f0);
  const int var = threadIdx.x / LINES;
  const int line = threadIdx.x % LINES;
  const int lg = l0 + line;
  if (lg < nlines) {
    const double* Ul = sU + (var * LINES + line) * WIN;
    const double* pt = (var == nmom) ? sHp + line * WIN : (var == 3 ? sHpu + line * WIN : nullptr);
    double* out;
    long long stride;
    if (xdir) { out = Fx + ((long long)var * ny + lg) * (nx + 1) + f0; stride = 1; }
    else { out = Gy + ((long long)var * (ny + 1) + f0) * nx + lg; stride = nx; }
    if (LIN) {
      const long long nfx = nx + 1, nfy = ny + 1;
      double* lb;
      long long cstride;
      if (xdir) { lb = lin + ((long long)var * nfx + f0) * ny + lg; cstride = (long long)NV * nfx * ny; }
      else { lb = lin + 8LL * NV * nfx * ny + ((long long)var * nfy + f0) * nx + lg; cstride = (long long)NV * nfy * nx; }
      slide_line2_lin(Ul, sLp + line * WIN, sLm + line * WIN, pt, g.eps4, nf, out, stride, lb, nlines, cstride);
    } else {
      slide_line2(Ul, sLp + line * WIN, sLm + line * WIN, pt, g.eps4, nf, out, stride);
    }
  }
}

template <int NV, int FC, bool HALO>
__global__ void __launch_bounds__(LINES * NV) k_face_flux(StateView S, const unsigned long long* __restrict__ alpha,
                                                          double* __restrict__ Fx, double* __restrict__ Gy,
                                                          GridDev g, int nbx, int ntx_x, int ntx_y) {
  extern __shared__ double smem[];
  face_flux_tile<NV, FC, HALO>(S, alpha, Fx, Gy, g, blockIdx.x, nbx, ntx_x, ntx_y, smem);
}

// The same face fluxes, bit for bit, plus the derivatives of every
// reconstruction with respect to its window differences in `lin` (the
// discrete adjoint's face-derivative store).
template <int NV, int FC>
__global__ void __launch_bounds__(LINES * NV) k_face_flux_lin(StateView S, const unsigned long long* __restrict__ alpha,
                                                              double* __restrict__ Fx, double* __restrict__ Gy,
                                                              double* __restrict__ lin, GridDev g, int nbx, int ntx_x,
                                                              int ntx_y) {
  extern __shared__ double smem[];
  face_flux_tile<NV, FC, false, true>(S, alpha, Fx, Gy, g, blockIdx.x, nbx, ntx_x, ntx_y, smem, lin);
}

// Batched form: a persistent grid walks the flattened (request, tile) list;
// request r owns entries [first[r], first[r+1]).
template <int NV>
__global__ void __launch_bounds__(LINES * NV) k_face_flux_batch(const BatchReq* __restrict__ reqs,
                                                                const int* __restrict__ first, int nreq, int state) {
  extern __shared__ double smem[];
  const int total = first[nreq];
  for (int e = blockIdx.x; e < total; e += gridDim.x) {
    const int r = batch_owner(first, nreq, e);
    const BatchReq& q = reqs[r];
    face_flux_tile<NV>(q.S[state], q.alpha + 2 * state, q.Fx, q.Gy, q.g, e - first[r], q.nbx, q.ntx_x, q.ntx_y,
                       smem);
    __syncthreads();
  }
}

template <int NV, int FC = FACES>
static size_t flux_smem_bytes() {
  return sizeof(double) * (size_t)(NV + 4) * LINES * (FC + 5);
}

int sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = s > 0 ? s : 1;
  }
  return cache[dev];
}

// Sets kernel attribute `attr` to `value` once per device: function
// attributes belong to the context of the device current at the call, so a
// process that drives several devices (or slabs on several devices) needs one
// flag per device. The flags are atomics, so concurrent first calls from
// several host threads set the attribute twice at worst, which is harmless.
cudaError_t set_attr_once(const void* func, cudaFuncAttribute attr, int value, std::atomic<unsigned long long>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done->load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(func, attr, value);
  if (e == cudaSuccess) done->fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Tiles of FC faces: x tiles first, then y tiles.
static void tiles_of(const GridDev& g, int fc, int* nbx, int* ntx_x, int* ntx_y, int* total) {
  *ntx_x = (g.nx + 1 + fc - 1) / fc;
  const int nty_x = (g.ny + LINES - 1) / LINES;
  *ntx_y = (g.nx + LINES - 1) / LINES;
  const int nty_y = (g.ny + 1 + fc - 1) / fc;
  *nbx = *ntx_x * nty_x;
  *total = *nbx + *ntx_y * nty_y;
}

template <int NV, int FC, bool HALO>
static cudaError_t launch_face_flux_fc(const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                       const GridDev& g, cudaStream_t st) {
  int nbx, ntx_x, ntx_y, total;
  tiles_of(g, FC, &nbx, &ntx_x, &ntx_y, &total);
  const size_t smem = flux_smem_bytes<NV, FC>();
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = set_attr_once((const void*)k_face_flux<NV, FC, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem, &attr_done);
  if (e != cudaSuccess) return e;
  k_face_flux<NV, FC, HALO><<<total, LINES * NV, smem, st>>>(S, alpha, Fx, Gy, g, nbx, ntx_x, ntx_y);
  return cudaGetLastError();
}

// Tile length by grid size: 32 faces while that gives at least 8 blocks per
// SM, 16 while that gives at least 2, else 8. Shorter tiles mean more blocks
// and a larger share of stencil margin; on small grids, whose launches are a
// fraction of a wave and latency-bound, the blocks win (measured on one
// GB300: 256 x 32 runs best at 8, 512 x 64 at 16, 4096 x 512 at 32).
static int flux_tile_faces(const GridDev& g) {
  const int sms = sm_count();
  int nbx, ntx_x, ntx_y, total;
  tiles_of(g, 32, &nbx, &ntx_x, &ntx_y, &total);
  if (total >= 8 * sms) return 32;
  tiles_of(g, 16, &nbx, &ntx_x, &ntx_y, &total);
  return total >= 2 * sms ? 16 : 8;
}

template <int NV, bool HALO>
static cudaError_t launch_face_flux_h(const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                      const GridDev& g, cudaStream_t st) {
  switch (flux_tile_faces(g)) {
    case 32: return launch_face_flux_fc<NV, 32, HALO>(S, alpha, Fx, Gy, g, st);
    case 16: return launch_face_flux_fc<NV, 16, HALO>(S, alpha, Fx, Gy, g, st);
    default: return launch_face_flux_fc<NV, 8, HALO>(S, alpha, Fx, Gy, g, st);
  }
}

template <int NV>
static cudaError_t launch_face_flux_t(const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                      const GridDev& g, cudaStream_t st) {
  if (g.bc[0] == BC_HALO || g.bc[1] == BC_HALO) return launch_face_flux_h<NV, true>(S, alpha, Fx, Gy, g, st);
  return launch_face_flux_h<NV, false>(S, alpha, Fx, Gy, g, st);
}

template <int NV, int FC>
static cudaError_t launch_face_flux_lin_fc(const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                           double* lin, const GridDev& g, cudaStream_t st) {
  int nbx, ntx_x, ntx_y, total;
  tiles_of(g, FC, &nbx, &ntx_x, &ntx_y, &total);
  const size_t smem = flux_smem_bytes<NV, FC>();
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = set_attr_once((const void*)k_face_flux_lin<NV, FC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem, &attr_done);
  if (e != cudaSuccess) return e;
  k_face_flux_lin<NV, FC><<<total, LINES * NV, smem, st>>>(S, alpha, Fx, Gy, lin, g, nbx, ntx_x, ntx_y);
  return cudaGetLastError();
}

template <int NV>
static cudaError_t launch_face_flux_lin_t(const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                          double* lin, const GridDev& g, cudaStream_t st) {
  switch (flux_tile_faces(g)) {
    case 32: return launch_face_flux_lin_fc<NV, 32>(S, alpha, Fx, Gy, lin, g, st);
    case 16: return launch_face_flux_lin_fc<NV, 16>(S, alpha, Fx, Gy, lin, g, st);
    default: return launch_face_flux_lin_fc<NV, 8>(S, alpha, Fx, Gy, lin, g, st);
  }
}

size_t face_lin_doubles(int nv, const GridDev& g) {
  return 8 * (size_t)nv * ((size_t)(g.nx + 1) * g.ny + (size_t)(g.ny + 1) * g.nx);
}

cudaError_t launch_face_flux_lin(int nv, const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                 double* lin, const GridDev& g, cudaStream_t st) {
  if (g.bc[0] == BC_HALO || g.bc[1] == BC_HALO) return cudaErrorInvalidValue;  // whole grids only
  switch (nv) {
    case 4: return launch_face_flux_lin_t<4>(S, alpha, Fx, Gy, lin, g, st);
    case 6: return launch_face_flux_lin_t<6>(S, alpha, Fx, Gy, lin, g, st);
    case 12: return launch_face_flux_lin_t<12>(S, alpha, Fx, Gy, lin, g, st);
    default: return cudaErrorInvalidValue;
  }
}

void face_flux_tiles(const GridDev& g, int* nbx, int* ntx_x, int* ntx_y, int* total) {
  tiles_of(g, FACES, nbx, ntx_x, ntx_y, total);
}

template <int NV>
static cudaError_t launch_face_flux_batch_t(const BatchReq* reqs, const int* first, int nreq, int total, int state,
                                            cudaStream_t st) {
  const size_t smem = flux_smem_bytes<NV>();
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = set_attr_once((const void*)k_face_flux_batch<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem, &attr_done);
  if (e != cudaSuccess) return e;
  const int sms = sm_count();
  const int grid = total < sms * 8 ? total : sms * 8;
  if (grid > 0) k_face_flux_batch<NV><<<grid, LINES * NV, smem, st>>>(reqs, first, nreq, state);
  return cudaGetLastError();
}

cudaError_t launch_face_flux_batch(int nv, const BatchReq* reqs, const int* first, int nreq, int total, int state,
                                   cudaStream_t st) {
  switch (nv) {
    case 4: return launch_face_flux_batch_t<4>(reqs, first, nreq, total, state, st);
    case 6: return launch_face_flux_batch_t<6>(reqs, first, nreq, total, state, st);
    case 12: return launch_face_flux_batch_t<12>(reqs, first, nreq, total, state, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_face_flux(int nv, const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                             const GridDev& g, cudaStream_t st) {
  switch (nv) {
    case 4: return launch_face_flux_t<4>(S, alpha, Fx, Gy, g, st);
    case 6: return launch_face_flux_t<6>(S, alpha, Fx, Gy, g, st);
    case 12: return launch_face_flux_t<12>(S, alpha, Fx, Gy, g, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace janc
