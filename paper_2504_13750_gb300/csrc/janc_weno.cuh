// Divide-free WENO5-JS reconstruction along a line of split fluxes, shared
// by the single-grid and the block (AMR) face-flux kernels.
#pragma once

#include "janc_device.cuh"

namespace janc {

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

}  // namespace janc
