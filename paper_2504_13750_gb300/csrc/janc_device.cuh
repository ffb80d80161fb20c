// Device-side data layout and helpers shared by the kernels of the reacting-
// flow step (arXiv 2504.13750, Sec. 4). All arithmetic is FP64.
//
// GB300 notes that shape this code: the FP64 pipe issues about 2 DFMA per
// clock per SM (roughly 1/64 of the FP32 rate), while integer, FP32, load and
// shuffle instructions issue at full rate. So every operation that can be
// done exactly outside the FP64 pipe is done there: maxima of non-negative
// doubles compare their bit patterns as integers, absolute values clear the
// sign bit, pivot searches and row swaps are integer compares and selects,
// and the reciprocal starts from the MUFU approximation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace janc {

constexpr double RU = 8.314472;     // universal gas constant (text after Eq. 4.5)
constexpr double P_REF = 101325.0;  // reference pressure of Eq. 4.9
constexpr int MAX_NS = 9;
constexpr int MAX_NR = 32;
constexpr int MAX_SIDE = 3;  // distinct species per reaction side

enum : int { ST_NONFINITE = 1, ST_NONPOSITIVE = 2, ST_NEWTON_FAIL = 4, ST_SINGULAR = 8 };
// BC_HALO marks an x side shared with the neighbouring slab of an x-slab
// decomposition (Sec. 4.4): its 3 ghost columns are read from a halo buffer
// that the exchange fills, not derived from the slab's own cells.
enum : int { BC_WALL = 0, BC_ZEROGRAD = 1, BC_PERIODIC = 2, BC_HALO = 3 };

// Mechanism in the form the kernels consume (built on the host from the
// user's table, copied once to device memory).
struct MechDev {
  int ns, nr;
  double M[MAX_NS];
  double invM[MAX_NS];
  // Enthalpy polynomial h_k/(Ru/M_k) = sum_{m<5} hc[k][m] T^{m+1} + hc[k][5]
  // with hc[k][m] = a_m/(m+1) (Eq. 4.4).
  double hc[MAX_NS][6];
  // Dimensionless Gibbs term of Eq. 4.9, G_k = s_k/R - h_k/(RT) (Eq. 4.4-4.5):
  // G = gc0 ln T + gc6 + T (gc1 + T (gc2 + T (gc3 + T gc4))) + gc5 / T with
  // gc0 = a0, gc1 = a1/2, gc2 = a2/6, gc3 = a3/12, gc4 = a4/20, gc5 = -a5,
  // gc6 = a6 - a0.
  double gc[MAX_NS][7];
  // Reactions (Eq. 4.6-4.8): ln k_f = lnA + b ln T - EaR / T.
  double lnA[MAX_NR], b[MAX_NR], EaR[MAX_NR];
  int nre[MAX_NR], rsp[MAX_NR][MAX_SIDE], rnu[MAX_NR][MAX_SIDE];
  int npr[MAX_NR], psp[MAX_NR][MAX_SIDE], pnu[MAX_NR][MAX_SIDE];
  int dnu[MAX_NR];  // sum of (nu_b - nu_f)
  int tb[MAX_NR];
  double rnud[MAX_NR][MAX_SIDE], pnud[MAX_NR][MAX_SIDE];  // the coefficients as doubles
  // Third-body factor as sum_j X_j + sum over the few species whose
  // coefficient differs from one: neff entries of (species, eff - 1).
  int neff[MAX_NR], effsp[MAX_NR][MAX_NS];
  double effv[MAX_NR][MAX_NS];
  double effm1[MAX_NR][MAX_NS];  // third-body coefficient minus one
  // Column factor for the Jacobian in carried variables (text after Eq. 4.13):
  // eff_il - (M_l / M_ns) eff_i,ns for l < ns - 1.
  double ceff[MAX_NR][MAX_NS];
  double mratio[MAX_NS];  // M_l / M_ns
  // Mixture sums in the carried variables: since rho Y_ns = rho - sum_{k<ns-1}
  // rho Y_k, sum_k (rho Y_k / M_k) c_k = rho cN + sum_{k<ns-1} rho Y_k cd_k
  // with cN = c_ns / M_ns and cd_k = c_k / M_k - cN. For the enthalpy
  // coefficients (hcN, hcd) and for c = 1 (WN, Wd: W = sum_k z_k).
  double hcN[6];
  double hcd[MAX_NS][6];
  double WN;
  double Wd[MAX_NS];
};

// Grid constants passed by value to every kernel.
struct GridDev {
  int nx, ny;
  long long n;  // nx * ny
  double dx, dy, rdx, rdy;
  int bc[4];  // left, right, bottom, top
  double eps4;  // 4 * WENO epsilon (smoothness indicators are carried scaled by 4)
  double newton_tol;
  int newton_maxit;
  // Halo buffers of the x sides whose bc is BC_HALO: [nv + 4][ny][3] each,
  // the 3 columns nearest the side, plane by plane like the state (column c
  // of the low halo is ghost cell c - 3, of the high halo cell nx + c).
  const double* halo_lo;
  const double* halo_hi;
  // 1: the mechanism has the reaction structure compiled into the fixed
  // chemistry kernels (the same operations, every index a constant)
  int chem_fixed;
};

// One state buffer: planes 0..nv-1 conserved, nv: T, nv+1: u, nv+2: v, nv+3: p.
struct StateView {
  double* base;
  __host__ __device__ double* plane(int k, long long n) const { return base + (long long)k * n; }
};

// Per-step control: fixed dt (> 0) or CFL; alpha slots hold max(|u|+c),
// max(|v|+c) as the bit patterns of non-negative doubles.
struct StepCtl {
  double dt_fixed;
  double cfl;
  double hmin;       // min(dx, dy)
  double chem_frac;  // share of the step's dt taken by one chemistry launch: 1, or 1/2 in the Strang order
  int source;        // 1: the production rates are an explicit source of every RK stage
};

// One request of a batched (serving) launch: its grid constants and buffers.
// Alpha slots (2 x u64 each): 0 = U^n, 1 = U^1, 2 = U^2, 3 = U^*, 4 = U^{n+1}.
struct BatchReq {
  GridDev g;
  StateView S[3];
  double* Fx;
  double* Gy;
  unsigned long long* alpha;
  double* clock2;
  int* status;
  const MechDev* mech;
  StepCtl ctl;
  int nbx, ntx_x, ntx_y;  // face-flux tiling
  int ubx, uby;           // update-kernel blocks in x and y
  int fresh;              // 1 until the first batched step after admission
};

// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }
// |x| by clearing the sign bit (integer pipe).
__device__ __forceinline__ double dabs(double x) { return bitsd(dbits(x) & 0x7fffffffffffffffull); }
__device__ __forceinline__ bool finite_bits(double x) {
  return ((dbits(x) >> 52) & 0x7ff) != 0x7ff;
}

// Reciprocal of a normal double: the MUFU approximation (relative error
// below 2^-20) refined by one third-order step of the iteration for 1/d,
// x' = x (1 + e + e^2) with e = 1 - d x, which cubes the relative error
// (2^-60, below double rounding) in three FMAs.
__device__ __forceinline__ double rcp(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  const double e = fma(-d, r, 1.0);
  const double e2 = fma(e, e, e);
  return fma(r, e2, r);
}

// 2^(j/64), j = 0..63, rounded to double (computed to 200 bits).
static __device__ const double kExp2Tab[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0};

// FP64 exponential by P. T. P. Tang's table-driven method (ACM TOMS 15(2),
// 1989): x = (64 m + j) ln2/64 + r with |r| <= ln2/128, the reduction split
// Cody-Waite style (L1 carries 32 significant bits, so n L1 is exact),
// exp(r) - 1 from its Taylor series through r^5/120 (truncation below
// 4e-17), then 2^(j/64) from the table and 2^m added to the exponent field
// with integer instructions. 10 FP64 instructions; about 1 ulp. Results that
// would overflow give +inf, underflow gives 0, NaN stays NaN.
__device__ __forceinline__ double exp_t(double x) {
  constexpr double kInv = 0x1.71547652b82fep+6;  // 64 / ln 2
  constexpr double kL1 = 0x1.62e42fee00000p-7;   // ln 2 / 64, leading part
  constexpr double kL2 = 0x1.a39ef35793c76p-39;  // ln 2 / 64 - kL1
  constexpr double kMagic = 0x1.8p52;            // rounds to an integer in the low mantissa bits
  const double t = fma(x, kInv, kMagic);
  const int n = __double2loint(t);
  const double nd = t - kMagic;
  double r = fma(nd, -kL1, x);
  r = fma(nd, -kL2, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const double T = __ldg(&kExp2Tab[n & 63]);
  const double y = fma(T, p, T);
  const int m = n >> 6;
  double out = bitsd(dbits(y) + ((unsigned long long)(long long)m << 52));
  const unsigned xe = (unsigned)(dbits(x) >> 52) & 0x7ffu;
  if (m > 1023) out = bitsd(0x7ff0000000000000ull);
  if (m < -1021) out = 0.0;
  if (xe == 0x7ffu) out = (dbits(x) & 0xfffffffffffffull) ? x : ((long long)dbits(x) < 0 ? 0.0 : x);
  return out;
}

// dt of the step from the alpha slot of its starting state (cfl() of Sec. 4.3).
__device__ __forceinline__ double step_dt(const StepCtl& c, const unsigned long long* a0) {
  if (c.dt_fixed > 0.0) return c.dt_fixed;
  unsigned long long ax = a0[0], ay = a0[1];
  double amax = bitsd(ax > ay ? ax : ay);
  return c.cfl * c.hmin / amax;
}

// W = sum_k z_k and the first NH mixture enthalpy coefficients
// h[q] = sum_k z_k hc_k[q] (z_k = rho Y_k / M_k) from the carried variables,
// through the folded tables of MechDev: 1 + (ns - 1) FP64 operations each.
template <int NS, int NH>
__device__ __forceinline__ void mixture_sums(const double* u, const MechDev& m, double& W, double* h) {
  const double rho = u[0];
  W = rho * m.WN;
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) W = fma(u[4 + k], m.Wd[k], W);
#pragma unroll
  for (int q = 0; q < NH; ++q) {
    double s = rho * m.hcN[q];
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) s = fma(u[4 + k], m.hcd[k][q], s);
    h[q] = s;
  }
}

// Sound speed exactly as newton_cell finishes it, from the stored T.
template <int NS>
__device__ __forceinline__ double sound_speed(const double* u, double t, const MechDev& m) {
  const double rrho = rcp(u[0]);
  double W, h[5];
  mixture_sums<NS, 5>(u, m, W, h);
  const double c1 = 2.0 * h[1], c2 = 3.0 * h[2], c3 = 4.0 * h[3], c4 = 5.0 * h[4];
  const double K1 = h[0] - W;
  const double Cv = fma(t, fma(t, fma(t, fma(t, c4, c3), c2), c1), K1);
  const double Cp = Cv + W;
  const double p = RU * W * t;
  return sqrt(Cp * p * rrho * rcp(Cv));
}

// Molar production rates (Eq. 4.7-4.9) of the carried species k < ns - 1 at
// (T, X(u)), for the explicit source-term form of the step.
template <int NS>
// keep (the discrete adjoint's store): k_f and k_b of reaction i go to
// keep[2i n + idx] and keep[(2i+1) n + idx].
__device__ __forceinline__ void carried_rates(const double* u, double T, const MechDev& m, double* wd,
                                              double* __restrict__ keep = nullptr, long long n = 0,
                                              long long idx = 0) {
  constexpr int NSP = NS - 1;
  double X[NS];
  double rest = u[0];
#pragma unroll
  for (int k = 0; k < NSP; ++k) {
    X[k] = u[4 + k] * m.invM[k];
    rest -= u[4 + k];
    wd[k] = 0.0;
  }
  X[NSP] = rest * m.invM[NSP];
  double Ctot = X[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) Ctot += X[k];
  const double lnT = log(T);
  const double rT = rcp(T);
  double eG[NS], reG[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* c = m.gc[k];
    eG[k] = exp_t(fma(c[0], lnT, fma(c[5], rT, fma(T, fma(T, fma(T, fma(T, c[4], c[3]), c[2]), c[1]), c[6]))));
    reG[k] = rcp(eG[k]);
  }
  const double cref = (P_REF / RU) * rT;
  const double rcref = (RU / P_REF) * T;
  for (int i = 0; i < m.nr; ++i) {
    const int nre = m.nre[i], npr = m.npr[i];
    const double kf = exp_t(fma(m.b[i], lnT, fma(-m.EaR[i], rT, m.lnA[i])));
    double kb = kf;
    for (int r = 0; r < nre; ++r)
      for (int q = 0; q < m.rnu[i][r]; ++q) kb *= eG[m.rsp[i][r]];
    for (int r = 0; r < npr; ++r)
      for (int q = 0; q < m.pnu[i][r]; ++q) kb *= reG[m.psp[i][r]];
    for (int q = 0; q < m.dnu[i]; ++q) kb *= rcref;
    for (int q = 0; q < -m.dnu[i]; ++q) kb *= cref;
    if (keep) {
      keep[(2LL * i) * n + idx] = kf;
      keep[(2LL * i + 1) * n + idx] = kb;
    }
    double fwd = kf, bwd = kb;
    for (int r = 0; r < nre; ++r)
      for (int q = 0; q < m.rnu[i][r]; ++q) fwd *= X[m.rsp[i][r]];
    for (int r = 0; r < npr; ++r)
      for (int q = 0; q < m.pnu[i][r]; ++q) bwd *= X[m.psp[i][r]];
    double Mi = 1.0;
    if (m.tb[i]) {
      Mi = Ctot;
      for (int e = 0; e < m.neff[i]; ++e) Mi = fma(m.effv[i][e], X[m.effsp[i][e]], Mi);
    }
    const double q = Mi * (fwd - bwd);
    for (int r = 0; r < nre; ++r)
      if (m.rsp[i][r] < NSP) wd[m.rsp[i][r]] = fma(-m.rnud[i][r], q, wd[m.rsp[i][r]]);
    for (int r = 0; r < npr; ++r)
      if (m.psp[i][r] < NSP) wd[m.psp[i][r]] = fma(m.pnud[i][r], q, wd[m.psp[i][r]]);
  }
}

// Ghost-cell source index along one axis (3 layers, text after Eq. 4.11).
__device__ __forceinline__ int ghost_src(int i, int n, int bc_lo, int bc_hi, bool& flip) {
  flip = false;
  if (i < 0) {
    if (bc_lo == BC_WALL) { flip = true; return -1 - i; }
    if (bc_lo == BC_ZEROGRAD) return 0;
    return i + n;
  }
  if (i >= n) {
    if (bc_hi == BC_WALL) { flip = true; return 2 * n - 1 - i; }
    if (bc_hi == BC_ZEROGRAD) return n - 1;
    return i - n;
  }
  return i;
}

// Request that owns entry e of a flattened list with per-request starts
// first[0..nreq] (first[0] = 0): the last r with first[r] <= e.
__device__ __forceinline__ int batch_owner(const int* __restrict__ first, int nreq, int e) {
  int lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Block-wide max of two non-negative doubles (as bits) and OR of a status
// word, then one atomic per block. blockDim.x * blockDim.y <= 1024.
__device__ __forceinline__ void block_reduce_alpha_status(unsigned long long sx, unsigned long long sy, int st,
                                                          unsigned long long* alpha_out, int* status) {
  __shared__ unsigned long long red_x[32], red_y[32];
  __shared__ int red_s[32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ox = __shfl_xor_sync(0xffffffffu, sx, o);
    unsigned long long oy = __shfl_xor_sync(0xffffffffu, sy, o);
    int os = __shfl_xor_sync(0xffffffffu, st, o);
    sx = ox > sx ? ox : sx;
    sy = oy > sy ? oy : sy;
    st |= os;
  }
  const int w = tid >> 5, lane = tid & 31;
  if (lane == 0) { red_x[w] = sx; red_y[w] = sy; red_s[w] = st; }
  __syncthreads();
  if (w == 0) {
    const int nw = (nthr + 31) >> 5;
    sx = lane < nw ? red_x[lane] : 0ull;
    sy = lane < nw ? red_y[lane] : 0ull;
    st = lane < nw ? red_s[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ox = __shfl_xor_sync(0xffffffffu, sx, o);
      unsigned long long oy = __shfl_xor_sync(0xffffffffu, sy, o);
      int os = __shfl_xor_sync(0xffffffffu, st, o);
      sx = ox > sx ? ox : sx;
      sy = oy > sy ? oy : sy;
      st |= os;
    }
    if (lane == 0) {
      if (alpha_out) {
        atomicMax(alpha_out, sx);
        atomicMax(alpha_out + 1, sy);
      }
      if (st) atomicOr(status, st);
    }
  }
}

// Newton-Raphson T recovery (end of Sec. 4.2) from the energy, warm-started
// at Tw, followed by p (Eq. 4.2) and the frozen sound speed. The mixture is
// reduced to polynomial coefficients once per cell (mixture_sums):
//   H(T) = sum_k z_k h_k(T)/Ru with z_k = rho Y_k / M_k,
//   F(T) = H(T) - W T - rho e / Ru  (W = sum_k z_k, rho e = E - |rho u|^2 / (2 rho)),
//   F'(T) = sum_k z_k cv_k / Ru.
// Stops when |dT| <= tol * T after the update. Returns status bits.
template <int NS>
__device__ __forceinline__ int newton_cell(const double* u, double Tw, const MechDev& m, double tol, int maxit,
                                           double& T, double& p, double& c, double& rrho) {
  const double rho = u[0];
  rrho = rcp(rho);
  double W, h[6];
  mixture_sums<NS, 6>(u, m, W, h);
  const double c1 = 2.0 * h[1], c2 = 3.0 * h[2], c3 = 4.0 * h[3], c4 = 5.0 * h[4];
  const double ke = fma(u[1], u[1], u[2] * u[2]);
  const double rhoe_R = fma(-0.5 * rrho, ke, u[3]) * (1.0 / RU);
  const double K0 = h[5] - rhoe_R;
  const double K1 = h[0] - W;
  double t = Tw;
  int st = 0;
  int it = 0;
  for (; it < maxit; ++it) {
    double F = fma(t, fma(t, fma(t, fma(t, fma(t, h[4], h[3]), h[2]), h[1]), K1), K0);
    double Fp = fma(t, fma(t, fma(t, fma(t, c4, c3), c2), c1), K1);
    double dT = -F * rcp(Fp);
    t += dT;
    if (!(dabs(dT) > tol * dabs(t))) break;
  }
  if (it == maxit) st |= ST_NEWTON_FAIL;
  T = t;
  const double Cv = fma(t, fma(t, fma(t, fma(t, c4, c3), c2), c1), K1);
  const double Cp = Cv + W;
  p = RU * W * t;
  c = sqrt(Cp * p * rrho * rcp(Cv));
  if (!(rho > 0.0) || !(t > 0.0) || !(p > 0.0)) st |= ST_NONPOSITIVE;
  if (!finite_bits(t) || !finite_bits(p) || !finite_bits(c) || !finite_bits(u[3])) st |= ST_NONFINITE;
  return st;
}

}  // namespace janc
