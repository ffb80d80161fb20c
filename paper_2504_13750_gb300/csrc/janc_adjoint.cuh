// Reverse-mode pieces of the discrete adjoint (transposes of the operators
// of janc_flux.cu / janc_update.cu / janc_chem.cu), shared by the adjoint
// kernels.
#pragma once

#include "janc_device.cuh"

namespace janc {

// Reverse of weno_face<MINUS> (janc_weno.cuh) on the sliding-window state of
// the 5-point stencil F_0..F_4 (differences D1..D4, second differences
// S1..S3, indicator parts T1..T3, as the Win struct carries them): given the
// cotangent gW of the reconstructed value, returns the cotangents g[0..4] of
// the five split-flux inputs. Same algebra as the forward formula, reversed
// operation by operation.
template <bool MINUS>
__device__ __forceinline__ void weno_face_vjp(double D1, double D2, double D3, double D4, double S1, double S2,
                                              double S3, double T1, double T2, double T3, double gW, double* g) {
  constexpr double c13 = 13.0 / 3.0;
  const double X = fma(2.0, D2, S1), Z = D2 + D3, Y = fma(-2.0, D3, S3);
  const double bA = fma(X, X, T1), bB = fma(Z, Z, T2), bC = fma(Y, Y, T3);
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
  // ---- reverse ----
  const double R = rcp(den);
  const double gnum = gW * R;
  const double gden = -gW * num * R * R;
  double gs0 = gnum * vv + gden * uu;
  const double gvv = gnum * s0;
  const double gq0 = gnum * P12;
  const double gP12 = gnum * q0s + gden;
  const double guu = gden * s0;
  const double gq1 = gvv * s2, gq2 = gvv * s1;
  double gs2 = gvv * q1 + 6.0 * guu + gP12 * s1;
  double gs1 = gvv * q2h + 3.0 * guu + gP12 * s2;
  double gsA, gsB, gsC;
  double gD1 = 0.0, gD2 = 0.0, gD3 = 0.0, gD4 = 0.0;
  if (!MINUS) {
    gsA = gs0; gsB = gs1; gsC = gs2;
    gD2 += (5.0 / 6.0) * gq0; gD1 += (-1.0 / 3.0) * gq0;
    gD3 += 2.0 * gq1; gD2 += gq1;
    gD4 += -0.5 * gq2; gD3 += 2.0 * gq2;
  } else {
    gsC = gs0; gsB = gs1; gsA = gs2;
    gD4 += (1.0 / 3.0) * gq0; gD3 += (-5.0 / 6.0) * gq0;
    gD2 += -2.0 * gq1; gD3 += -gq1;
    gD1 += 0.5 * gq2; gD2 += -2.0 * gq2;
  }
  const double gbA = 2.0 * bA * gsA, gbB = 2.0 * bB * gsB, gbC = 2.0 * bC * gsC;
  const double gX = 2.0 * X * gbA, gZ = 2.0 * Z * gbB, gY = 2.0 * Y * gbC;
  double gS1 = 2.0 * c13 * S1 * gbA + gX;
  double gS2 = 2.0 * c13 * S2 * gbB;
  double gS3 = 2.0 * c13 * S3 * gbC + gY;
  gD2 += 2.0 * gX + gZ;
  gD3 += gZ - 2.0 * gY;
  // S_j = D_{j+1} - D_j
  gD2 += gS1; gD1 -= gS1;
  gD3 += gS2; gD2 -= gS2;
  gD4 += gS3; gD3 -= gS3;
  // D_j = F_j - F_{j-1}
  g[0] = -gD1;
  g[1] = gD1 - gD2;
  g[2] = gD2 - gD3 + gW;
  g[3] = gD3 - gD4;
  g[4] = gD4;
}

// Mixture quantities of one cell at a given T (the converged Newton T):
// W = sum z_k, hR_k(T) = h_k/(Ru/M_k), Cv = sum z_k cv_k / Ru and dCv/dT.
template <int NS>
struct CellThermo {
  double z[NS], hR[NS], cvR[NS];
  double W, Cv, dCv;
};

template <int NS>
__device__ __forceinline__ void cell_thermo(const double* u, double T, const MechDev& m, CellThermo<NS>& c) {
  double rest = u[0];
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    c.z[k] = u[4 + k] * m.invM[k];
    rest -= u[4 + k];
  }
  c.z[NS - 1] = rest * m.invM[NS - 1];
  c.W = 0.0;
  c.Cv = 0.0;
  c.dCv = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* h = m.hc[k];
    c.hR[k] = fma(T, fma(T, fma(T, fma(T, fma(T, h[4], h[3]), h[2]), h[1]), h[0]), h[5]);
    // cp/R = a0 + a1 T + ... with a_m = (m+1) hc_m
    const double cp = fma(T, fma(T, fma(T, fma(T, 5.0 * h[4], 4.0 * h[3]), 3.0 * h[2]), 2.0 * h[1]), h[0]);
    c.cvR[k] = cp - 1.0;
    const double dcp = fma(T, fma(T, fma(T, 20.0 * h[4], 12.0 * h[3]), 6.0 * h[2]), 2.0 * h[1]);
    c.W += c.z[k];
    c.Cv = fma(c.z[k], c.cvR[k], c.Cv);
    c.dCv = fma(c.z[k], dcp, c.dCv);
  }
}

// dT/dU (implicit derivative of the Newton T recovery) and dp/dU for one
// cell, NV = NS + 3 entries each. With F(T; U) = H(T; z) - W T - rho e / Ru:
// dT/dU = -(dF/dU) / Cv and p = Ru W T.
template <int NS>
__device__ __forceinline__ void dT_dp_dU(const double* u, double T, const MechDev& m, const CellThermo<NS>& c,
                                         double* dT, double* dp) {
  constexpr int NV = NS + 3;
  const double rrho = 1.0 / u[0];
  const double vx = u[1] * rrho, vy = u[2] * rrho;
  double dF[NV], dW[NV];
  const double fN = (c.hR[NS - 1] - T) * m.invM[NS - 1];
  dF[0] = fN - 0.5 * (vx * vx + vy * vy) * (1.0 / RU);
  dF[1] = vx * (1.0 / RU);
  dF[2] = vy * (1.0 / RU);
  dF[3] = -1.0 / RU;
  dW[0] = m.invM[NS - 1];
  dW[1] = dW[2] = dW[3] = 0.0;
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    dF[4 + k] = (c.hR[k] - T) * m.invM[k] - fN;
    dW[4 + k] = m.invM[k] - m.invM[NS - 1];
  }
  const double rCv = 1.0 / c.Cv;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    dT[q] = -dF[q] * rCv;
    dp[q] = RU * (T * dW[q] + c.W * dT[q]);
  }
}

}  // namespace janc
