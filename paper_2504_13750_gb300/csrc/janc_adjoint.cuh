// Reverse-mode pieces of the discrete adjoint (transposes of the operators
// of janc_flux.cu / janc_update.cu / janc_chem.cu), shared by the adjoint
// kernels.
#pragma once

#include "janc_device.cuh"

namespace janc {

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
  const double rrho = rcp(u[0]);
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
  const double rCv = rcp(c.Cv);
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    dT[q] = -dF[q] * rCv;
    dp[q] = RU * (T * dW[q] + c.W * dT[q]);
  }
}

}  // namespace janc
