// Host-side launchers shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "../../include/janc.h"
#include "janc_device.cuh"

namespace janc {

// Kernel-form mechanism table from the C-ABI description (janc_capi.cu).
int build_mech_table(const janc_mechanism* m, MechDev* h);
// Sets the text janc_last_error() returns on this thread (janc_capi.cu).
void set_last_error(const char* msg);

// The device pieces of a grid object that other subsystems drive directly
// (janc_capi.cu): its current state U^n, constants, mechanism table, alpha
// slot 0 (the state's LF speeds), status word and stream.
struct GridParts {
  StateView S0;
  GridDev gd;
  const MechDev* mech;
  unsigned long long* alpha;
  int* status;
  cudaStream_t stream;
  int ns, nv, chemistry;
};
GridParts grid_parts(janc_grid_t g);

// LF-split WENO5 face fluxes of state S (janc_flux.cu).
cudaError_t launch_face_flux(int nv, const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                             const GridDev& g, cudaStream_t st);

// The same face fluxes plus the derivatives of every WENO5 reconstruction
// with respect to its window differences, face_lin_doubles(nv, g) doubles
// at `lin` (janc_flux.cu; whole grids only).
cudaError_t launch_face_flux_lin(int nv, const StateView& S, const unsigned long long* alpha, double* Fx, double* Gy,
                                 double* lin, const GridDev& g, cudaStream_t st);
size_t face_lin_doubles(int nv, const GridDev& g);

// RK3 stage `stage` (1..3): Sout = combination of S0 and Sin + dt L(Sin), then
// Newton T warm-started from Sin's T, aux planes, and the alpha max of Sout
// into alpha_out (janc_update.cu). alpha_step holds the step's starting alpha.
// src_keep (explicit source only, may be null): k_f and k_b of every reaction
// at the stage input, 2 nr doubles per cell entry-major (carried_rates).
cudaError_t launch_rk_update(int ns, int stage, const StateView& Sin, const StateView& S0, const StateView& Sout,
                             const double* Fx, const double* Gy, const GridDev& g, const MechDev* mech,
                             const StepCtl& ctl, const unsigned long long* alpha_step, unsigned long long* alpha_out,
                             int* status, double* clock2, cudaStream_t st, double* src_keep = nullptr);

// Point-implicit chemistry in place on S (janc_chem.cu).
cudaError_t launch_chem(int ns, const StateView& S, const GridDev& g, const MechDev* mech, const StepCtl& ctl,
                        const unsigned long long* alpha_step, unsigned long long* alpha_out, int* status,
                        cudaStream_t st);

// Point-implicit chemistry that also keeps the factors the chemistry VJP
// reuses: chem_lin_entries(ns, nr) doubles per cell at clin, entry-major
// (janc_chem.cu).
cudaError_t launch_chem_lin(int ns, const StateView& S, const GridDev& g, const MechDev* mech, const StepCtl& ctl,
                            const unsigned long long* alpha_step, unsigned long long* alpha_out, int* status,
                            double* clin, cudaStream_t st);
size_t chem_lin_entries(int ns, int nr);

// State set-up kernels (janc_update.cu).
cudaError_t launch_set_primitive(int ns, const StateView& S, const double* T, const double* p, const double* u,
                                 const double* v, const double* Y, const GridDev& g, const MechDev* mech,
                                 unsigned long long* alpha_out, int* status, cudaStream_t st);
cudaError_t launch_set_conserved(int ns, const StateView& S, const double* T0, const GridDev& g, const MechDev* mech,
                                 unsigned long long* alpha_out, int* status, cudaStream_t st);
// Batched launches over a flattened (request, block) list; first[0..nreq]
// holds each request's first entry, first[nreq] the total (device memory).
void face_flux_tiles(const GridDev& g, int* nbx, int* ntx_x, int* ntx_y, int* total);
void update_blocks(const GridDev& g, int* ubx, int* uby);
int chem_blocks(const GridDev& g);
cudaError_t launch_batch_prep(BatchReq* reqs, int nreq, cudaStream_t st);
cudaError_t launch_face_flux_batch(int nv, const BatchReq* reqs, const int* first, int nreq, int total, int state,
                                   cudaStream_t st);
cudaError_t launch_rk_update_batch(int ns, int stage, const BatchReq* reqs, const int* first, int nreq, int total,
                                   int chem, cudaStream_t st);
cudaError_t launch_chem_batch(int ns, const BatchReq* reqs, const int* first, int nreq, int total, bool fixed,
                              cudaStream_t st);
// Whether a mechanism has the reaction structure compiled into the fixed
// chemistry kernels (janc_mech_fixed.cuh; janc_chem.cu).
bool fixed_structure(const janc_mechanism* m);

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

// Adjoint pieces (janc_adjoint.cu).
// Scratch of one launch_rhs_vjp: the two alpha cotangents and the per-block
// arg-max partials of the LF speeds (256-byte aligned start).
size_t rhs_vjp_scratch_bytes(const GridDev& g);
// Input and outputs of one RHS vector-Jacobian product nu = (dL/dU)^T mu
// with mu = mu_scale lam, fused with the linear combinations of an RK stage
// of the reverse sweep ([nv][ny][nx] arrays):
//   a = (acc_a ? a : 0) + ca xa + nu        (xa may be null)
//   b = (acc_b ? b : 0) + cb xb             (b may be null)
struct VjpIO {
  const double* lam;
  double mu_scale;
  double* a;
  const double* xa;
  double ca;
  int acc_a;
  double* b;
  const double* xb;
  double cb;
  int acc_b;
};
// lin: the state's face-derivative store (launch_face_flux_lin), or null to
// recompute the reconstructions. fresh: zero the per-position sums and the
// alpha cotangents first; otherwise they must be zero on entry (every call
// leaves them zero). src (explicit source-term form): add the VJP of the
// source S(U) at the state, (dS/dU)^T mu, to io.a; src_keep: the stage's rate
// constants kept by launch_rk_update, or null to form them again.
cudaError_t launch_rhs_vjp(int ns, const StateView& S, const double* alpha2_dev, const VjpIO& io, double* CFx,
                           double* CFy, double* scratch, const GridDev& g, const MechDev* mech, const double* lin,
                           bool fresh, bool src, const double* src_keep, cudaStream_t st);
// clin: the factors the segment recompute kept (launch_chem_lin), or null to
// form them again.
cudaError_t launch_chem_vjp(int ns, const StateView& Sstar, const GridDev& g, const MechDev* mech, double dt,
                            const double* lam, double* out, const double* clin, cudaStream_t st);
cudaError_t launch_lincomb(long long count, double* out, double a, const double* x, double b, const double* y,
                           bool accumulate, cudaStream_t st);
cudaError_t launch_loss_endwall(int ns, const StateView& S, const GridDev& g, double w, double* loss,
                                cudaStream_t st);
cudaError_t launch_seed_endwall(int ns, const StateView& S, const GridDev& g, const MechDev* mech, double w,
                                double* lam, cudaStream_t st);
cudaError_t launch_dot(long long count, const double* a, const double* b, double* out, cudaStream_t st);
cudaError_t launch_prim_T_vjp(int ns, const double* T, const double* p, const double* u, const double* v,
                              const double* Y, const double* dLdU, double* out, const GridDev& g,
                              const MechDev* mech, cudaStream_t st);

// Halo pack of the x-slab exchange: the 3 columns of each of `planes` planes
// of S nearest each x side into [planes][ny][3] buffers (janc_update.cu).
cudaError_t launch_halo_pack(int planes, const StateView& S, const GridDev& g, double* lo_dst, double* hi_dst,
                             cudaStream_t st);

// Sets a kernel attribute once per device (janc_flux.cu).
cudaError_t set_attr_once(const void* func, cudaFuncAttribute attr, int value, std::atomic<unsigned long long>* done);

// L = -(dF/dx + dG/dy) from the face fluxes.
cudaError_t launch_rhs_L(int nv, const double* Fx, const double* Gy, double* L, const GridDev& g, cudaStream_t st);

}  // namespace janc
