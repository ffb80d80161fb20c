// Generated by paper_2504_13750_gb300/mech_codegen.py from mechanisms/h2air_synth.json;
// regenerate instead of editing. The reaction structure (Eq. 4.6-4.7) of the shipped
// H2-air mechanism as compile-time constants: species 0 H2, 1 O2, 2 H, 3 O, 4 OH, 5 HO2, 6 H2O2, 7 H2O, 8 N2.
#pragma once

namespace janc {
namespace fixed_h2air {

constexpr int NS = 9;
constexpr int NR = 19;

// Reaction I: reactant / product species and coefficients in species order,
// the sum of product minus reactant coefficients, the third-body flag and the
// species whose third-body coefficient differs from one (in species order).
template <int I>
struct Rx;
template <>
struct Rx<0> {
  static constexpr int i = 0, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 1 : (r == 1 ? 2 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 3 : (r == 1 ? 4 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<1> {
  static constexpr int i = 1, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 0 : (r == 1 ? 3 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 2 : (r == 1 ? 4 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<2> {
  static constexpr int i = 2, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 0 : (r == 1 ? 4 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 2 : (r == 1 ? 7 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<3> {
  static constexpr int i = 3, nre = 1, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 4 : (-1); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 2 : (0); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 3 : (r == 1 ? 7 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<4> {
  static constexpr int i = 4, nre = 1, npr = 1, dnu = -1, tb = 1, neff = 2;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (-1); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 2 : (0); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 0 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return r == 0 ? 0 : (r == 1 ? 7 : (-1)); }
};
template <>
struct Rx<5> {
  static constexpr int i = 5, nre = 2, npr = 1, dnu = -1, tb = 1, neff = 2;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (r == 1 ? 4 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 7 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return r == 0 ? 0 : (r == 1 ? 7 : (-1)); }
};
template <>
struct Rx<6> {
  static constexpr int i = 6, nre = 2, npr = 1, dnu = -1, tb = 1, neff = 2;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (r == 1 ? 3 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 4 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return r == 0 ? 0 : (r == 1 ? 7 : (-1)); }
};
template <>
struct Rx<7> {
  static constexpr int i = 7, nre = 1, npr = 1, dnu = -1, tb = 1, neff = 2;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 3 : (-1); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 2 : (0); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 1 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return r == 0 ? 0 : (r == 1 ? 7 : (-1)); }
};
template <>
struct Rx<8> {
  static constexpr int i = 8, nre = 2, npr = 1, dnu = -1, tb = 1, neff = 2;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 1 : (r == 1 ? 2 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 5 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return r == 0 ? 0 : (r == 1 ? 7 : (-1)); }
};
template <>
struct Rx<9> {
  static constexpr int i = 9, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (r == 1 ? 5 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 0 : (r == 1 ? 1 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<10> {
  static constexpr int i = 10, nre = 2, npr = 1, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (r == 1 ? 5 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 4 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 2 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<11> {
  static constexpr int i = 11, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 3 : (r == 1 ? 5 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 1 : (r == 1 ? 4 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<12> {
  static constexpr int i = 12, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 4 : (r == 1 ? 5 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 1 : (r == 1 ? 7 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<13> {
  static constexpr int i = 13, nre = 1, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 5 : (-1); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 2 : (0); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 1 : (r == 1 ? 6 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<14> {
  static constexpr int i = 14, nre = 1, npr = 1, dnu = 1, tb = 1, neff = 2;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 6 : (-1); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (0); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 4 : (-1); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 2 : (0); }
  __host__ __device__ static constexpr int effsp(int r) { return r == 0 ? 0 : (r == 1 ? 7 : (-1)); }
};
template <>
struct Rx<15> {
  static constexpr int i = 15, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (r == 1 ? 6 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 4 : (r == 1 ? 7 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<16> {
  static constexpr int i = 16, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 2 : (r == 1 ? 6 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 0 : (r == 1 ? 5 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<17> {
  static constexpr int i = 17, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 3 : (r == 1 ? 6 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 4 : (r == 1 ? 5 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};
template <>
struct Rx<18> {
  static constexpr int i = 18, nre = 2, npr = 2, dnu = 0, tb = 0, neff = 0;
  __host__ __device__ static constexpr int rsp(int r) { return r == 0 ? 4 : (r == 1 ? 6 : (-1)); }
  __host__ __device__ static constexpr int rnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int psp(int r) { return r == 0 ? 5 : (r == 1 ? 7 : (-1)); }
  __host__ __device__ static constexpr int pnu(int r) { return r == 0 ? 1 : (r == 1 ? 1 : (0)); }
  __host__ __device__ static constexpr int effsp(int r) { return -1; }
};

// The same structure as plain tables, for the host-side match of a run-time
// mechanism: nuf / nub [NR][NS], tb [NR], eff_ne1 [NR][NS] (1 where the
// third-body coefficient of a third-body reaction is not one).
constexpr int kNuf[NR * NS] = {
    0, 1, 1, 0, 0, 0, 0, 0, 0,
    1, 0, 0, 1, 0, 0, 0, 0, 0,
    1, 0, 0, 0, 1, 0, 0, 0, 0,
    0, 0, 0, 0, 2, 0, 0, 0, 0,
    0, 0, 2, 0, 0, 0, 0, 0, 0,
    0, 0, 1, 0, 1, 0, 0, 0, 0,
    0, 0, 1, 1, 0, 0, 0, 0, 0,
    0, 0, 0, 2, 0, 0, 0, 0, 0,
    0, 1, 1, 0, 0, 0, 0, 0, 0,
    0, 0, 1, 0, 0, 1, 0, 0, 0,
    0, 0, 1, 0, 0, 1, 0, 0, 0,
    0, 0, 0, 1, 0, 1, 0, 0, 0,
    0, 0, 0, 0, 1, 1, 0, 0, 0,
    0, 0, 0, 0, 0, 2, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 1, 0, 0,
    0, 0, 1, 0, 0, 0, 1, 0, 0,
    0, 0, 1, 0, 0, 0, 1, 0, 0,
    0, 0, 0, 1, 0, 0, 1, 0, 0,
    0, 0, 0, 0, 1, 0, 1, 0, 0,
};
constexpr int kNub[NR * NS] = {
    0, 0, 0, 1, 1, 0, 0, 0, 0,
    0, 0, 1, 0, 1, 0, 0, 0, 0,
    0, 0, 1, 0, 0, 0, 0, 1, 0,
    0, 0, 0, 1, 0, 0, 0, 1, 0,
    1, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 1, 0,
    0, 0, 0, 0, 1, 0, 0, 0, 0,
    0, 1, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 1, 0, 0, 0,
    1, 1, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 2, 0, 0, 0, 0,
    0, 1, 0, 0, 1, 0, 0, 0, 0,
    0, 1, 0, 0, 0, 0, 0, 1, 0,
    0, 1, 0, 0, 0, 0, 1, 0, 0,
    0, 0, 0, 0, 2, 0, 0, 0, 0,
    0, 0, 0, 0, 1, 0, 0, 1, 0,
    1, 0, 0, 0, 0, 1, 0, 0, 0,
    0, 0, 0, 0, 1, 1, 0, 0, 0,
    0, 0, 0, 0, 0, 1, 0, 1, 0,
};
constexpr int kTb[NR] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0};
constexpr int kEffNe1[NR * NS] = {
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    1, 0, 0, 0, 0, 0, 0, 1, 0,
    1, 0, 0, 0, 0, 0, 0, 1, 0,
    1, 0, 0, 0, 0, 0, 0, 1, 0,
    1, 0, 0, 0, 0, 0, 0, 1, 0,
    1, 0, 0, 0, 0, 0, 0, 1, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    1, 0, 0, 0, 0, 0, 0, 1, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0,
};

}  // namespace fixed_h2air
}  // namespace janc
