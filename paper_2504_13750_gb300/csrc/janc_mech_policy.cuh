// Structure policies of the per-cell chemistry code (janc_chem.cu) and its
// reverse (janc_adjoint.cu): how a loop over the reactions of a mechanism
// sees each reaction's species, stoichiometric coefficients (Eq. 4.6) and
// third-body data (Eq. 4.7). DynRx reads them from the run-time table,
// FixRx<I> returns the compiled constants of the shipped H2-air mechanism
// (janc_mech_fixed.cuh). A loop written once over for_reactions<FIXED> runs
// the same operations in the same order either way; with FIXED every index
// it derives is a compile-time constant.
#pragma once

#include <utility>

#include "janc_device.cuh"
#include "janc_mech_fixed.cuh"

namespace janc {

// Reaction i of the run-time mechanism table.
struct DynRx {
  const MechDev& m;
  int i;
  __device__ __forceinline__ int idx() const { return i; }
  __device__ __forceinline__ int nre() const { return m.nre[i]; }
  __device__ __forceinline__ int npr() const { return m.npr[i]; }
  __device__ __forceinline__ int dnu() const { return m.dnu[i]; }
  __device__ __forceinline__ int tb() const { return m.tb[i]; }
  __device__ __forceinline__ int neff() const { return m.neff[i]; }
  __device__ __forceinline__ int rsp(int r) const { return m.rsp[i][r]; }
  __device__ __forceinline__ int rnu(int r) const { return m.rnu[i][r]; }
  __device__ __forceinline__ double rnud(int r) const { return m.rnud[i][r]; }
  __device__ __forceinline__ int psp(int r) const { return m.psp[i][r]; }
  __device__ __forceinline__ int pnu(int r) const { return m.pnu[i][r]; }
  __device__ __forceinline__ double pnud(int r) const { return m.pnud[i][r]; }
  __device__ __forceinline__ int effsp(int e) const { return m.effsp[i][e]; }
};

// Reaction I of the compiled H2-air structure (numbers still come from the table).
template <int I>
struct FixRx {
  using S = fixed_h2air::Rx<I>;
  __device__ __forceinline__ static constexpr int idx() { return I; }
  __device__ __forceinline__ static constexpr int nre() { return S::nre; }
  __device__ __forceinline__ static constexpr int npr() { return S::npr; }
  __device__ __forceinline__ static constexpr int dnu() { return S::dnu; }
  __device__ __forceinline__ static constexpr int tb() { return S::tb; }
  __device__ __forceinline__ static constexpr int neff() { return S::neff; }
  __device__ __forceinline__ static constexpr int rsp(int r) { return S::rsp(r); }
  __device__ __forceinline__ static constexpr int rnu(int r) { return S::rnu(r); }
  __device__ __forceinline__ static constexpr double rnud(int r) { return (double)S::rnu(r); }
  __device__ __forceinline__ static constexpr int psp(int r) { return S::psp(r); }
  __device__ __forceinline__ static constexpr int pnu(int r) { return S::pnu(r); }
  __device__ __forceinline__ static constexpr double pnud(int r) { return (double)S::pnu(r); }
  __device__ __forceinline__ static constexpr int effsp(int e) { return S::effsp(e); }
};

template <int... I, class F>
__device__ __forceinline__ void fixed_reactions(std::integer_sequence<int, I...>, F&& f) {
  (f(FixRx<I>{}), ...);
}

// f(reaction) for every reaction, in order.
template <bool FIXED, class F>
__device__ __forceinline__ void for_reactions(const MechDev& m, F&& f) {
  if constexpr (FIXED) {
    fixed_reactions(std::make_integer_sequence<int, fixed_h2air::NR>{}, f);
  } else {
    for (int i = 0; i < m.nr; ++i) f(DynRx{m, i});
  }
}

}  // namespace janc
