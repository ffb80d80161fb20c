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
// cS_j = 13/3 S_j is kept for the derivative (weno_face_dD).
struct Win {
  double F2, F3, F4, D1, D2, D3, D4, S1, S2, S3, cS1, cS2, cS3, T1, T2, T3;
  __device__ __forceinline__ void init(double F0, double F1, double f2, double f3, double f4, double eps4) {
    constexpr double c13 = 13.0 / 3.0;
    F2 = f2; F3 = f3; F4 = f4;
    D1 = F1 - F0; D2 = F2 - F1; D3 = F3 - F2; D4 = F4 - F3;
    S1 = D2 - D1; S2 = D3 - D2; S3 = D4 - D3;
    cS1 = c13 * S1; cS2 = c13 * S2; cS3 = c13 * S3;
    T1 = fma(cS1, S1, eps4); T2 = fma(cS2, S2, eps4); T3 = fma(cS3, S3, eps4);
  }
  __device__ __forceinline__ void push(double Fn, double eps4) {
    constexpr double c13 = 13.0 / 3.0;
    const double Dn = Fn - F4;
    F2 = F3; F3 = F4; F4 = Fn;
    D1 = D2; D2 = D3; D3 = D4; D4 = Dn;
    S1 = S2; S2 = S3; S3 = D4 - D3;
    cS1 = cS2; cS2 = cS3; cS3 = c13 * S3;
    T1 = T2; T2 = T3; T3 = fma(cS3, S3, eps4);
  }
};

// The derivative of one reconstruction with respect to the differences of
// its window: for W = weno_face<MINUS>(window), the partials of W - F2 with
// respect to D1..D4 (the window's five values enter W only through D1..D4
// and, with weight one, F2). With s_k the squared scaled indicators,
// r = W - F2 = num/den and e_k the candidate offsets less r (scaled by the
// linear weights), reverse mode through num/den, s_k = b_k^2,
// b_k = (its first difference)^2 + T_k and the candidate offsets gives
//   dr/ds_0 = [s2 e1 + s1 e2] / den, dr/ds_1 = [s0 e2 + s2 e0] / den,
//   dr/ds_2 = [s0 e1 + s1 e0] / den,
// and db_k/dD_m in closed form (X = 3 D2 - D1, Z = D2 + D3, Y = D4 - 3 D3 and
// the 13/3 S^2 terms). The forward part repeats weno_face's operations in
// its order, so *F_hat equals weno_face's result bit for bit. scale4 is four
// times the factor the partials are multiplied by. ACC: the scaled partials
// are added to g1..g4; else they are written there.
template <bool MINUS, bool ACC>
__device__ __forceinline__ void weno_face_dD(const Win& w, double scale4, double* F_hat, double& g1, double& g2,
                                             double& g3, double& g4) {
  const double D1 = w.D1, D2 = w.D2, D3 = w.D3, D4 = w.D4;
  const double X = fma(2.0, D2, w.S1);
  const double Z = D2 + D3;
  const double Y = fma(-2.0, D3, w.S3);
  const double bA = fma(X, X, w.T1);
  const double bB = fma(Z, Z, w.T2);
  const double bC = fma(Y, Y, w.T3);
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
  const double R = rcp(den);
  if (F_hat) *F_hat = fma(num, R, w.F2);
  const double r = num * R;
  // reverse, everything times 4 scale (powers of two fold exactly)
  const double a4 = scale4 * R;
  const double e0 = q0s - r;
  const double e1 = fma(-6.0, r, q1);
  const double e2 = fma(-3.0, r, q2h);
  const double A0 = a4 * s0, A1 = a4 * s1, A2 = a4 * s2;
  const double gs0 = fma(A2, e1, A1 * e2);
  const double gs1 = fma(A0, e2, A2 * e0);
  const double gs2 = fma(A0, e1, A1 * e0);
  const double gq0 = A1 * s2, gq1 = A0 * s2, gq2 = A0 * s1;
  double hA, hC;
  const double hB = bB * gs1;
  if (!MINUS) { hA = bA * gs0; hC = bC * gs2; } else { hA = bA * gs2; hC = bC * gs0; }
  const double t1 = X + w.cS1, t2 = fma(3.0, X, w.cS1);
  const double t3 = Z - w.cS2, t4 = Z + w.cS2;
  const double t5 = fma(3.0, Y, w.cS3), t6 = Y + w.cS3;
  double c1, c2, c3, c4;  // the candidate-offset parts of the four partials
  if (!MINUS) {
    c1 = (-1.0 / 12.0) * gq0;
    c2 = fma(5.0 / 24.0, gq0, 0.25 * gq1);
    c3 = 0.5 * (gq1 + gq2);
    c4 = -0.125 * gq2;
  } else {
    c1 = 0.125 * gq2;
    c2 = -0.5 * (gq1 + gq2);
    c3 = fma(-5.0 / 24.0, gq0, -0.25 * gq1);
    c4 = (1.0 / 12.0) * gq0;
  }
  if (ACC) {
    g1 = fma(-hA, t1, g1 + c1);
    g2 = fma(hA, t2, fma(hB, t3, g2 + c2));
    g3 = fma(hB, t4, fma(-hC, t5, g3 + c3));
    g4 = fma(hC, t6, g4 + c4);
  } else {
    g1 = fma(-hA, t1, c1);
    g2 = fma(hA, t2, fma(hB, t3, c2));
    g3 = fma(hB, t4, fma(-hC, t5, c3));
    g4 = fma(hC, t6, c4);
  }
}

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

// slide_line2 that also stores, per face, the derivatives of both
// reconstructions with respect to their window differences (weno_face_dD),
// a quarter of each: component c (0..3: F+ window D1..D4, 4..7: F- window)
// of face t at lin[c * cstride + t * fstride]. The face values are
// slide_line2's bit for bit.
__device__ __forceinline__ void slide_line2_lin(const double* __restrict__ Ul, const double* __restrict__ lp,
                                                const double* __restrict__ lm, const double* __restrict__ pt,
                                                double eps4, int nf, double* __restrict__ out, long long stride,
                                                double* __restrict__ lin, long long fstride, long long cstride) {
  auto Fp = [&](int w) -> double { return pt ? fma(lp[w], Ul[w], pt[w]) : lp[w] * Ul[w]; };
  auto Fm = [&](int w) -> double { return pt ? fma(lm[w], Ul[w], pt[w]) : lm[w] * Ul[w]; };
  Win P, M;
  P.init(Fp(0), Fp(1), Fp(2), Fp(3), Fp(4), eps4);
  M.init(Fm(1), Fm(2), Fm(3), Fm(4), Fm(5), eps4);
  for (int t = 0; t < nf; ++t) {
    double rp, rm, g[8];
    weno_face_dD<false, false>(P, 1.0, &rp, g[0], g[1], g[2], g[3]);
    weno_face_dD<true, false>(M, 1.0, &rm, g[4], g[5], g[6], g[7]);
    out[(long long)t * stride] = rp + rm;
    double* l = lin + (long long)t * fstride;
#pragma unroll
    for (int c = 0; c < 8; ++c) l[c * cstride] = g[c];
    if (t + 1 < nf) {
      P.push(Fp(t + 5), eps4);
      M.push(Fm(t + 6), eps4);
    }
  }
}

}  // namespace janc
