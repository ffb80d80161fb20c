// Face fluxes of the conservative finite-difference scheme (arXiv 2504.13750,
// Eq. 4.10): global Lax-Friedrichs flux-vector splitting (Eq. 4.11) and
// WENO5 reconstruction of F+ and F- at every cell face, with the 3 ghost
// layers of the text after Eq. 4.11 produced on the fly during the tile load.
//
// One launch covers both directions: blocks [0, nbx) take x-face tiles and the
// rest take y-face tiles. A tile is LINES grid lines (rows for x, columns for
// y) by FACES consecutive faces along them. Its cells, with the 5-cell stencil
// margin, are staged in shared memory once; every thread then owns one
// (line, variable) and slides two 5-point windows (F+ and F-) along its line,
// so the first and second differences and the 13/3 S^2 part of the
// smoothness indicators are computed once per point instead of once per
// face, and each thread carries two independent dependency chains.
//
// Per face and sign the reconstruction costs 27 FP64 instructions plus 5 per
// new point (Jiang-Shu weights in divide-free form, one reciprocal).
#include "janc_device.cuh"
#include "janc_internal.h"

namespace janc {

constexpr int LINES = 8;
constexpr int FACES = 32;
constexpr int WIN = FACES + 5;

// WENO5-JS at one face from the sliding-window state. The window holds the
// split flux at 5 consecutive cells F_0..F_4 through
//   D_j = F_j - F_{j-1} (j = 1..4), S_j = D_{j+1} - D_j (j = 1..3),
//   T_j = 13/3 S_j^2 + 4 eps,
// and centre F_2. MINUS = false reconstructs F+ at the right face of cell 2;
// MINUS = true reconstructs F- at the left face of cell 2 (mirrored stencil).
// With smoothness indicators scaled by 4 (4 beta = 13/3 S^2 + e^2) the
// candidate weights d_k / (eps + beta_k)^2 keep their ratios. Writing
// s_k = (4 (eps + beta_k))^2, the weighted value is
//   F_2 + [Q0/6 s1 s2 + s0 (Q1 s2 + Q2/2 s1)] / [s1 s2 + s0 (6 s2 + 3 s1)]
// with the candidate offsets Q_k from the linear weights (1, 6, 3)/10.
template <bool MINUS>
__device__ __forceinline__ double weno_face(double F2, double D1, double D2, double D3, double D4, double S1,
                                            double S3, double T1, double T2, double T3) {
  const double X = fma(2.0, D2, S1);
  const double Z = D2 + D3;
  const double Y = fma(-2.0, D3, S3);
  const double bA = fma(X, X, T1);  // left 3-point substencil
  const double bB = fma(Z, Z, T2);  // centred
  const double bC = fma(Y, Y, T3);  // right
  const double sA = bA * bA, sB = bB * bB, sC = bC * bC;
  double s0, s1, s2, q0s, q1, q2h;
  if (!MINUS) {
    s0 = sA; s1 = sB; s2 = sC;
    q0s = fma(5.0 / 6.0, D2, (-1.0 / 3.0) * D1);
    q1 = fma(2.0, D3, D2);
    q2h = fma(-0.5, D4, 2.0 * D3);
  } else {
    s0 = sC; s1 = sB; s2 = sA;
    q0s = fma(1.0 / 3.0, D4, (-5.0 / 6.0) * D3);
    q1 = fma(-2.0, D2, -D3);
    q2h = fma(0.5, D1, -2.0 * D2);
  }
  const double P12 = s1 * s2;
  const double uu = fma(6.0, s2, 3.0 * s1);
  const double den = fma(s0, uu, P12);
  const double vv = fma(q1, s2, q2h * s1);
  const double num = fma(s0, vv, q0s * P12);
  return fma(num, rcp(den), F2);
}

// Sliding-window state of one sign along a line: the 5 split-flux values
// F_0..F_4 of the current face held as centre F2, differences D1..D4,
// second differences S1, S2, S3 and the shared indicator parts T1..T3.
struct Win {
  double F2, F3, F4, D1, D2, D3, D4, S1, S2, S3, T1, T2, T3;
  __device__ __forceinline__ void init(double F0, double F1, double f2, double f3, double f4, double eps4) {
    constexpr double c13 = 13.0 / 3.0;
    F2 = f2; F3 = f3; F4 = f4;
    D1 = F1 - F0; D2 = F2 - F1; D3 = F3 - F2; D4 = F4 - F3;
    S1 = D2 - D1; S2 = D3 - D2; S3 = D4 - D3;
    T1 = fma(c13 * S1, S1, eps4); T2 = fma(c13 * S2, S2, eps4); T3 = fma(c13 * S3, S3, eps4);
  }
  __device__ __forceinline__ void push(double Fn, double eps4) {
    constexpr double c13 = 13.0 / 3.0;
    const double Dn = Fn - F4;
    F2 = F3; F3 = F4; F4 = Fn;
    D1 = D2; D2 = D3; D3 = D4; D4 = Dn;
    S1 = S2; S2 = S3; S3 = D4 - D3;
    T1 = T2; T2 = T3; T3 = fma(c13 * S3, S3, eps4);
  }
};

// One (variable, line): reconstructs F+ (window starting at cell w = 0) and
// F- (window starting at w = 1) at every face of the line, two independent
// dependency chains per thread, and stores F^ = F+^ + F-^ at out[t * stride].
__device__ __forceinline__ void slide_line2(const double* __restrict__ Ul, const double* __restrict__ lp,
                                            const double* __restrict__ lm, const double* __restrict__ pt,
                                            double eps4, int nf, double* __restrict__ out, long long stride) {
  auto Fp = [&](int w) -> double { return pt ? fma(lp[w], Ul[w], pt[w]) : lp[w] * Ul[w]; };
  auto Fm = [&](int w) -> double { return pt ? fma(lm[w], Ul[w], pt[w]) : lm[w] * Ul[w]; };
  Win P, M;
  P.init(Fp(0), Fp(1), Fp(2), Fp(3), Fp(4), eps4);
  M.init(Fm(1), Fm(2), Fm(3), Fm(4), Fm(5), eps4);
  for (int t = 0; t < nf; ++t) {
    const double rp = weno_face<false>(P.F2, P.D1, P.D2, P.D3, P.D4, P.S1, P.S3, P.T1, P.T2, P.T3);
    const double rm = weno_face<true>(M.F2, M.D1, M.D2, M.D3, M.D4, M.S1, M.S3, M.T1, M.T2, M.T3);
    out[(long long)t * stride] = rp + rm;
    if (t + 1 < nf) {
      P.push(Fp(t + 5), eps4);
      M.push(Fm(t + 6), eps4);
    }
  }
}

// One tile of the face-flux launch; `blk` is the tile's index in the
// launch (x tiles first). Shared by the single-grid and the batched kernels.
template <int NV>
__device__ __forceinline__ void face_flux_tile(const StateView& S, const unsigned long long* __restrict__ alpha,
                                               double* __restrict__ Fx, double* __restrict__ Gy, const GridDev& g,
                                               int blk, int nbx, int ntx_x, int ntx_y, double* smem) {
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
  const int f0 = xdir ? ta * FACES : tb * FACES;
  const int l0 = xdir ? tb * LINES : ta * LINES;
  const int nlines = xdir ? ny : nx;          // number of lines in the domain
  const int nfaces = (xdir ? nx : ny) + 1;    // faces per line
  const int ncell = xdir ? nx : ny;           // cells along a line
  const int bc_lo = xdir ? g.bc[0] : g.bc[2];
  const int bc_hi = xdir ? g.bc[1] : g.bc[3];
  const int nmom = xdir ? 1 : 2;  // wall-normal momentum plane
  const double alph = bitsd(alpha[xdir ? 0 : 1]);
  const double ha = 0.5 * alph;
  const double* uplane = S.plane(xdir ? NV + 1 : NV + 2, n);
  const double* pplane = S.plane(NV + 3, n);

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
    const int src = ghost_src(cg, ncell, bc_lo, bc_hi, flip);
    const long long idx = xdir ? (long long)lg * nx + src : (long long)src * nx + lg;
    double un = uplane[idx];
    if (flip) un = -un;
    const double hp = 0.5 * pplane[idx];
    const int o = line * WIN + w;
    sLp[o] = fma(0.5, un, ha);
    sLm[o] = fma(0.5, un, -ha);
    sHp[o] = hp;
    sHpu[o] = hp * un;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double v = S.plane(k, n)[idx];
      if (flip && k == nmom) v = -v;
      sU[(k * LINES + line) * WIN + w] = v;
    }
  }
  __syncthreads();

  // ---- reconstruct and store: thread = (variable, line), both signs ----
  const int nf = min(FACES, nfaces - f0);
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
    slide_line2(Ul, sLp + line * WIN, sLm + line * WIN, pt, g.eps4, nf, out, stride);
  }
}

template <int NV>
__global__ void __launch_bounds__(LINES * NV) k_face_flux(StateView S, const unsigned long long* __restrict__ alpha,
                                                          double* __restrict__ Fx, double* __restrict__ Gy,
                                                          GridDev g, int nbx, int ntx_x, int ntx_y) {
  extern __shared__ double smem[];
  face_flux_tile<NV>(S, alpha, Fx, Gy, g, blockIdx.x, nbx, ntx_x, ntx_y, smem);
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

template <int NV>
static size_t flux_smem_bytes() {
  return sizeof(double) * (size_t)(NV + 4) * LINES * WIN;
}

template <int NV>
static cudaError_t launch_face_flux_t(const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                      const GridDev& g, cudaStream_t st) {
  const int ntx_x = (g.nx + 1 + FACES - 1) / FACES;
  const int nty_x = (g.ny + LINES - 1) / LINES;
  const int ntx_y = (g.nx + LINES - 1) / LINES;
  const int nty_y = (g.ny + 1 + FACES - 1) / FACES;
  const int nbx = ntx_x * nty_x;
  const int nby = ntx_y * nty_y;
  const size_t smem = flux_smem_bytes<NV>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_face_flux<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_face_flux<NV><<<nbx + nby, LINES * NV, smem, st>>>(S, alpha, Fx, Gy, g, nbx, ntx_x, ntx_y);
  return cudaGetLastError();
}

void face_flux_tiles(const GridDev& g, int* nbx, int* ntx_x, int* ntx_y, int* total) {
  *ntx_x = (g.nx + 1 + FACES - 1) / FACES;
  const int nty_x = (g.ny + LINES - 1) / LINES;
  *ntx_y = (g.nx + LINES - 1) / LINES;
  const int nty_y = (g.ny + 1 + FACES - 1) / FACES;
  *nbx = *ntx_x * nty_x;
  *total = *nbx + *ntx_y * nty_y;
}

template <int NV>
static cudaError_t launch_face_flux_batch_t(const BatchReq* reqs, const int* first, int nreq, int total, int state,
                                            cudaStream_t st) {
  const size_t smem = flux_smem_bytes<NV>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_face_flux_batch<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
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
