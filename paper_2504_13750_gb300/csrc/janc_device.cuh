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
enum : int { BC_WALL = 0, BC_ZEROGRAD = 1, BC_PERIODIC = 2 };

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
  double effm1[MAX_NR][MAX_NS];  // third-body coefficient minus one
  // Column factor for the Jacobian in carried variables (text after Eq. 4.13):
  // eff_il - (M_l / M_ns) eff_i,ns for l < ns - 1.
  double ceff[MAX_NR][MAX_NS];
  double mratio[MAX_NS];  // M_l / M_ns
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
  double hmin;  // min(dx, dy)
};

// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }
// |x| by clearing the sign bit (integer pipe).
__device__ __forceinline__ double dabs(double x) { return bitsd(dbits(x) & 0x7fffffffffffffffull); }
__device__ __forceinline__ bool finite_bits(double x) {
  return ((dbits(x) >> 52) & 0x7ff) != 0x7ff;
}

// Reciprocal of a normal double: MUFU approximation refined by two
// Newton-Raphson steps for 1/x (x_{k+1} = x_k (2 - d x_k), written as two
// FMAs per step), which square the relative error each time.
__device__ __forceinline__ double rcp(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  return r;
}

// dt of the step from the alpha slot of its starting state (cfl() of Sec. 4.3).
__device__ __forceinline__ double step_dt(const StepCtl& c, const unsigned long long* a0) {
  if (c.dt_fixed > 0.0) return c.dt_fixed;
  unsigned long long ax = a0[0], ay = a0[1];
  double amax = bitsd(ax > ay ? ax : ay);
  return c.cfl * c.hmin / amax;
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
// reduced to polynomial coefficients once per cell:
//   H(T) = sum_k z_k h_k(T)/Ru with z_k = rho Y_k / M_k,
//   F(T) = H(T) - W T - rho e / Ru  (W = sum_k z_k, rho e = E - |rho u|^2 / (2 rho)),
//   F'(T) = sum_k z_k cv_k / Ru.
// Stops when |dT| <= tol * T after the update. Returns status bits.
template <int NS>
__device__ __forceinline__ int newton_cell(const double* u, double Tw, const MechDev& m, double tol, int maxit,
                                           double& T, double& p, double& c, double& rrho) {
  const double rho = u[0];
  rrho = rcp(rho);
  double z[NS];
  double rest = rho;
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    z[k] = u[4 + k] * m.invM[k];
    rest -= u[4 + k];
  }
  z[NS - 1] = rest * m.invM[NS - 1];
  double W = z[0];
#pragma unroll
  for (int k = 1; k < NS; ++k) W += z[k];
  double h[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double s = z[0] * m.hc[0][q];
#pragma unroll
    for (int k = 1; k < NS; ++k) s = fma(z[k], m.hc[k][q], s);
    h[q] = s;
  }
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
