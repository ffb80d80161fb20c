// C ABI of the reacting-flow step (see include/janc.h for the contract).
//
// Device memory of one grid (one workspace, 256-byte aligned pieces):
//   3 state buffers of nv + 4 planes [ny][nx] each (conserved, T, u, v, p):
//     S0 = U^n (and U^{n+1} after the step), S1 = stage 1 / scratch,
//     S2 = stage 2;
//   Fx[nv][ny][nx+1], Gy[nv][ny+1][nx] face fluxes;
//   alpha slots: 2 x u64 per state of a chunk of steps (bit patterns of the
//     non-negative LF speeds, reduced with atomicMax);
//   clock2 (t, dt_last), status word, mechanism table.
// The step sequence per time step (advance_one_step, Sec. 4.3) is
//   flux(S0) -> update1 -> S1, flux(S1) -> update2 -> S2,
//   flux(S2) -> update3 -> S0 (in place), [chem on S0 in place],
// with dt computed on the device from the alpha slot of the step's start.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/janc.h"
#include "janc_device.cuh"
#include "janc_grid.h"
#include "janc_internal.h"

using namespace janc;

namespace {

thread_local std::string g_err;

int fail(int code, const char* msg) {
  g_err = msg;
  return code;
}
int fail_cuda(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return JANC_E_CUDA;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

namespace janc {

Layout layout_of(int nx, int ny, int nv, bool halos) {
  Layout L;
  const size_t n = (size_t)nx * ny;
  L.state = align256(sizeof(double) * (size_t)(nv + 4) * n);
  L.fx = align256(sizeof(double) * (size_t)nv * ny * (nx + 1));
  L.gy = align256(sizeof(double) * (size_t)nv * (ny + 1) * nx);
  L.alpha = align256(sizeof(unsigned long long) * 2 * (SLOTS_PER_STEP * CHUNK + 1));
  L.clock = align256(sizeof(double) * 2);
  L.status = align256(sizeof(int));
  L.mech = align256(sizeof(MechDev));
  L.halo = halos ? align256(sizeof(double) * (size_t)(nv + 4) * ny * 3) : 0;
  L.total = 3 * L.state + L.fx + L.gy + L.alpha + L.clock + L.status + L.mech + 2 * L.halo;
  return L;
}

int fail_cuda_at(cudaError_t e, const char* where) { return fail_cuda(e, where); }
int fail_msg(int code, const char* msg) { return fail(code, msg); }

}  // namespace janc

namespace {

int check_desc(const janc_grid_desc* d, const janc_mechanism* m) {
  if (!d || !m) return fail(JANC_E_INVALID, "null descriptor");
  if (d->nx < 1 || d->ny < 1) return fail(JANC_E_INVALID, "nx, ny must be >= 1");
  if (!(d->dx > 0.0) || !(d->dy > 0.0)) return fail(JANC_E_INVALID, "dx, dy must be > 0");
  for (int s = 0; s < 4; ++s)
    if (d->bc[s] < 0 || d->bc[s] > 2) return fail(JANC_E_INVALID, "unknown boundary kind");
  if ((d->bc[0] == JANC_BC_PERIODIC) != (d->bc[1] == JANC_BC_PERIODIC) ||
      (d->bc[2] == JANC_BC_PERIODIC) != (d->bc[3] == JANC_BC_PERIODIC))
    return fail(JANC_E_INVALID, "periodic boundaries must be set on both sides of an axis");
  if ((d->bc[0] != JANC_BC_ZEROGRAD || d->bc[1] != JANC_BC_ZEROGRAD) && d->nx < 3)
    return fail(JANC_E_INVALID, "wall or periodic boundaries in x need nx >= 3");
  if ((d->bc[2] != JANC_BC_ZEROGRAD || d->bc[3] != JANC_BC_ZEROGRAD) && d->ny < 3)
    return fail(JANC_E_INVALID, "wall or periodic boundaries in y need ny >= 3");
  if (!(m->ns == 1 || m->ns == 3 || m->ns == 9)) return fail(JANC_E_UNSUPPORTED, "species count must be 1, 3 or 9");
  if (m->nr < 0 || m->nr > MAX_NR) return fail(JANC_E_UNSUPPORTED, "at most 32 reactions");
  if (!m->M || !m->nasa) return fail(JANC_E_INVALID, "null molar masses or NASA-7 table");
  if (m->nr > 0 && (!m->A || !m->b || !m->Ea || !m->nuf || !m->nub || !m->tb || !m->eff))
    return fail(JANC_E_INVALID, "null reaction table");
  if (d->chemistry < JANC_CHEM_OFF || d->chemistry > JANC_CHEM_EXPLICIT)
    return fail(JANC_E_INVALID, "chemistry must be one of the JANC_CHEM_* modes");
  if (d->chemistry && (m->nr == 0 || m->ns < 3)) return fail(JANC_E_INVALID, "chemistry needs reactions and ns >= 3");
  return JANC_OK;
}

int build_mech(const janc_mechanism* m, MechDev* h) {
  std::memset(h, 0, sizeof(MechDev));
  const int ns = m->ns;
  h->ns = ns;
  h->nr = m->nr;
  for (int k = 0; k < ns; ++k) {
    if (!(m->M[k] > 0.0)) return fail(JANC_E_INVALID, "molar masses must be > 0");
    h->M[k] = m->M[k];
    h->invM[k] = 1.0 / m->M[k];
    const double* a = m->nasa + 7 * k;
    for (int q = 0; q < 5; ++q) h->hc[k][q] = a[q] / (q + 1);
    h->hc[k][5] = a[5];
    h->gc[k][0] = a[0];
    h->gc[k][1] = a[1] / 2.0;
    h->gc[k][2] = a[2] / 6.0;
    h->gc[k][3] = a[3] / 12.0;
    h->gc[k][4] = a[4] / 20.0;
    h->gc[k][5] = -a[5];
    h->gc[k][6] = a[6] - a[0];
    h->mratio[k] = m->M[k] / m->M[ns - 1];
  }
  h->WN = h->invM[ns - 1];
  for (int q = 0; q < 6; ++q) h->hcN[q] = h->hc[ns - 1][q] * h->invM[ns - 1];
  for (int k = 0; k < ns - 1; ++k) {
    h->Wd[k] = h->invM[k] - h->WN;
    for (int q = 0; q < 6; ++q) h->hcd[k][q] = h->hc[k][q] * h->invM[k] - h->hcN[q];
  }
  for (int i = 0; i < m->nr; ++i) {
    if (!(m->A[i] > 0.0)) return fail(JANC_E_INVALID, "Arrhenius A must be > 0");
    h->lnA[i] = std::log(m->A[i]);
    h->b[i] = m->b[i];
    h->EaR[i] = m->Ea[i] / RU;
    int nre = 0, npr = 0, dn = 0;
    for (int j = 0; j < ns; ++j) {
      const int f = m->nuf[i * ns + j], bb = m->nub[i * ns + j];
      if (f < 0 || f > 3 || bb < 0 || bb > 3) return fail(JANC_E_UNSUPPORTED, "stoichiometric coefficients 0..3");
      if (f) {
        if (nre == MAX_SIDE) return fail(JANC_E_UNSUPPORTED, "more than 3 reactant species");
        h->rsp[i][nre] = j;
        h->rnu[i][nre++] = f;
      }
      if (bb) {
        if (npr == MAX_SIDE) return fail(JANC_E_UNSUPPORTED, "more than 3 product species");
        h->psp[i][npr] = j;
        h->pnu[i][npr++] = bb;
      }
      dn += bb - f;
    }
    h->nre[i] = nre;
    h->npr[i] = npr;
    h->dnu[i] = dn;
    h->tb[i] = m->tb[i] ? 1 : 0;
    for (int r = 0; r < nre; ++r) h->rnud[i][r] = (double)h->rnu[i][r];
    for (int r = 0; r < npr; ++r) h->pnud[i][r] = (double)h->pnu[i][r];
    h->neff[i] = 0;
    for (int j = 0; j < ns; ++j) {
      const double e = m->tb[i] ? m->eff[i * ns + j] : 0.0;
      h->effm1[i][j] = e - 1.0;
      if (m->tb[i] && e != 1.0) {
        h->effsp[i][h->neff[i]] = j;
        h->effv[i][h->neff[i]++] = e - 1.0;
      }
    }
    for (int l = 0; l < ns - 1; ++l) {
      const double el = m->tb[i] ? m->eff[i * ns + l] : 0.0;
      const double eN = m->tb[i] ? m->eff[i * ns + ns - 1] : 0.0;
      h->ceff[i][l] = el - h->mratio[l] * eN;
    }
  }
  return JANC_OK;
}

}  // namespace

namespace janc {
int build_mech_table(const janc_mechanism* m, MechDev* h) { return build_mech(m, h); }
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace janc


namespace {

cudaEvent_t take_event(janc_grid_s* g) {
  if (!g->pool.empty()) {
    cudaEvent_t e = g->pool.back();
    g->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launches `f` (a callable returning cudaError_t) and, while profiling is on,
// brackets it with events on the grid's stream.
template <class F>
cudaError_t timed(janc_grid_s* g, int cls, F&& f) {
  if (!g->prof_on) return f();
  janc_grid_s::Mark m{take_event(g), take_event(g), cls};
  cudaEventRecord(m.a, g->stream);
  cudaError_t e = f();
  cudaEventRecord(m.b, g->stream);
  g->marks.push_back(m);
  return e;
}

}  // namespace

static StateView sv(const janc_grid_s* g, int k) { return StateView{g->S[k]}; }

namespace janc {
GridParts grid_parts(janc_grid_t g) {
  GridParts p;
  p.S0 = StateView{g->S[0]};
  p.gd = g->gd;
  p.mech = g->mech;
  p.alpha = g->alpha;
  p.status = g->status;
  p.stream = g->stream;
  p.ns = g->ns;
  p.nv = g->nv;
  p.chemistry = g->d.chemistry;
  return p;
}
}  // namespace janc

int janc::create_grid(const janc_grid_desc* d, const janc_mechanism* m, void* workspace, size_t workspace_bytes,
                      void* cuda_stream, const SlabOpts* so, janc_grid_s** out) {
  int rc = check_desc(d, m);
  if (rc) return rc;
  if (!out) return fail(JANC_E_INVALID, "null output handle");
  if (so && (so->halo_lo || so->halo_hi) && d->nx < 3)
    return fail(JANC_E_INVALID, "a slab needs nx >= 3 (its halo is 3 columns of its neighbour)");
  MechDev hm;
  rc = build_mech(m, &hm);
  if (rc) return rc;
  janc_grid_s* g = new janc_grid_s();
  g->d = *d;
  if (!(g->d.weno_eps > 0.0)) g->d.weno_eps = 1e-6;
  if (!(g->d.newton_tol > 0.0)) g->d.newton_tol = 1e-12;
  if (g->d.newton_maxit <= 0) g->d.newton_maxit = 50;
  g->ns = m->ns;
  g->nv = m->ns + 3;
  g->nr = m->nr;
  g->n = (long long)d->nx * d->ny;
  const bool own_halos = so && ((so->halo_lo && !so->halo_ext[0]) || (so->halo_hi && !so->halo_ext[1]));
  g->L = layout_of(d->nx, d->ny, g->nv, own_halos);
  g->stream = (cudaStream_t)cuda_stream;
  GridDev& gd = g->gd;
  gd.nx = d->nx;
  gd.ny = d->ny;
  gd.n = g->n;
  gd.dx = d->dx;
  gd.dy = d->dy;
  gd.rdx = 1.0 / d->dx;
  gd.rdy = 1.0 / d->dy;
  for (int s = 0; s < 4; ++s) gd.bc[s] = d->bc[s];
  gd.eps4 = 4.0 * g->d.weno_eps;
  gd.newton_tol = g->d.newton_tol;
  gd.newton_maxit = g->d.newton_maxit;
  gd.halo_lo = gd.halo_hi = nullptr;
  gd.chem_fixed = fixed_structure(m) ? 1 : 0;
  if (workspace) {
    if (workspace_bytes < g->L.total || ((uintptr_t)workspace & 255u)) {
      delete g;
      return fail(JANC_E_NOMEM, "workspace too small or not 256-byte aligned");
    }
    g->ws = (char*)workspace;
    g->owns_ws = false;
  } else {
    cudaError_t e = cudaMalloc(&g->ws, g->L.total);
    if (e != cudaSuccess) {
      delete g;
      return fail(JANC_E_NOMEM, "cudaMalloc of the grid workspace failed");
    }
    g->owns_ws = true;
  }
  char* p = g->ws;
  for (int k = 0; k < 3; ++k) { g->S[k] = (double*)p; p += g->L.state; }
  g->Fx = (double*)p; p += g->L.fx;
  g->Gy = (double*)p; p += g->L.gy;
  g->alpha = (unsigned long long*)p; p += g->L.alpha;
  g->clock2 = (double*)p; p += g->L.clock;
  g->status = (int*)p; p += g->L.status;
  g->mech = (MechDev*)p; p += g->L.mech;
  if (so) {
    // a slab: shared x sides read their ghosts from halo buffers
    const bool side[2] = {so->halo_lo, so->halo_hi};
    for (int k = 0; k < 2; ++k) {
      if (!side[k]) continue;
      g->halo_side[k] = true;
      if (so->halo_ext[k]) {
        g->halo[k] = so->halo_ext[k];
      } else {
        g->halo[k] = (double*)p;
        p += g->L.halo;
      }
      gd.bc[k] = BC_HALO;
    }
    gd.halo_lo = g->halo[0];
    gd.halo_hi = g->halo[1];
    if (so->alpha) {
      g->alpha = so->alpha;
      g->alpha_shared = true;
    }
  }
  cudaError_t e = cudaMemcpyAsync(g->mech, &hm, sizeof(MechDev), cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->clock2, 0, 2 * sizeof(double), g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->status, 0, sizeof(int), g->stream);
  if (e == cudaSuccess && !g->alpha_shared) e = cudaMemsetAsync(g->alpha, 0, g->L.alpha, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    if (g->owns_ws) cudaFree(g->ws);
    delete g;
    return fail_cuda(e, "janc_create_grid");
  }
  g->steps_done = 0;
  *out = g;
  return JANC_OK;
}

// The step loop of janc_step (advance_one_step of Sec. 4.3, n times) over
// ng grids advanced in lockstep. Per step, with the alpha slots a0 = U^n
// (dt source), aH = after the first half chemistry (Strang order only), a1,
// a2 = stages, a3 = U^*, a4 = U^{n+1} (the next step's a0):
//   [Strang: chem(dt/2) -> aH, exchange]
//   flux(S0) -> update1 -> S1, a1, exchange
//   flux(S1) -> update2 -> S2, a2, exchange
//   flux(S2) -> update3 -> S0 (a3 with chemistry, else a4) [no chemistry: exchange]
//   [chemistry: chem -> S0, a4, exchange]
// Each phase is launched for every grid before the exchange; the exchange
// runs only between phases, so every face-flux launch of a slab reads halos
// and alpha values that all slabs finished. A stage-3 output that chemistry
// consumes next needs no exchange: chemistry is per cell and reads a0 only.
int janc::step_grids(janc_grid_s* const* gs, int ng, Exchanger* ex, int n_steps, double dt, double cfl,
                     double* t_out, double* dt_last_out) {
  if (!gs || ng < 1 || !gs[0]) return fail(JANC_E_INVALID, "null grid");
  if (n_steps < 0) return fail(JANC_E_INVALID, "n_steps < 0");
  if ((dt > 0.0) == (cfl > 0.0)) return fail(JANC_E_INVALID, "give exactly one of dt > 0 or cfl > 0");
  janc_grid_s* g = gs[0];  // alpha slots, stream and clock of the lockstep set
  StepCtl ctl;
  ctl.dt_fixed = dt > 0.0 ? dt : 0.0;
  ctl.cfl = cfl > 0.0 ? cfl : 0.0;
  ctl.hmin = g->gd.dx < g->gd.dy ? g->gd.dx : g->gd.dy;
  const bool strang = g->d.chemistry == JANC_CHEM_STRANG;
  ctl.chem_frac = strang ? 0.5 : 1.0;
  ctl.source = g->d.chemistry == JANC_CHEM_EXPLICIT ? 1 : 0;
  double t_before = 0.0;
  if (t_out) {
    cudaError_t e = cudaMemcpyAsync(&t_before, g->clock2, sizeof(double), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail_cuda(e, "janc_step clock read");
  }
  const bool chem = g->d.chemistry == JANC_CHEM_LIE || g->d.chemistry == JANC_CHEM_STRANG;
  cudaStream_t st = g->stream;
  // one phase: `launch(grid)` for every grid, then (xk >= 0) the exchange of
  // state buffer xk with alpha slot xa
  auto phase = [&](int cls, auto&& launch, int xk, unsigned long long* xa) -> int {
    for (int q = 0; q < ng; ++q) {
      janc_grid_s* h = gs[q];
      const cudaError_t e = timed(h, cls, [&] { return launch(h); });
      if (e != cudaSuccess) return fail_cuda(e, "step launch");
    }
    if (ex && xk >= 0) return ex->after(xk, xa);
    return JANC_OK;
  };
  int done = 0;
  while (done < n_steps) {
    const int nc = (n_steps - done) < CHUNK ? (n_steps - done) : CHUNK;
    cudaError_t e = cudaMemsetAsync(g->alpha + 2, 0, sizeof(unsigned long long) * 2 * SLOTS_PER_STEP * nc, st);
    if (e != cudaSuccess) return fail_cuda(e, "alpha reset");
    for (int s = 0; s < nc; ++s) {
      unsigned long long* a0 = g->alpha + 2 * (SLOTS_PER_STEP * s);
      unsigned long long* aH = a0 + 2;
      unsigned long long* a1 = a0 + 4;
      unsigned long long* a2 = a0 + 6;
      unsigned long long* a3 = a0 + 8;
      unsigned long long* a4 = a0 + 10;
      unsigned long long* aF = a0;  // alpha of the flux stage-1 input
      int rc = JANC_OK;
      if (strang) {
        rc = phase(2, [&](janc_grid_s* h) { return launch_chem(h->ns, sv(h, 0), h->gd, h->mech, ctl, a0, aH, h->status, h->stream); },
                   0, aH);
        if (rc) return rc;
        aF = aH;
      }
      rc = phase(0, [&](janc_grid_s* h) { return launch_face_flux(h->nv, sv(h, 0), aF, h->Fx, h->Gy, h->gd, h->stream); },
                 -1, nullptr);
      if (!rc)
        rc = phase(1, [&](janc_grid_s* h) {
          return launch_rk_update(h->ns, 1, sv(h, 0), sv(h, 0), sv(h, 1), h->Fx, h->Gy, h->gd, h->mech, ctl, a0, a1,
                                  h->status, h->clock2, h->stream);
        }, 1, a1);
      if (!rc)
        rc = phase(0, [&](janc_grid_s* h) { return launch_face_flux(h->nv, sv(h, 1), a1, h->Fx, h->Gy, h->gd, h->stream); },
                   -1, nullptr);
      if (!rc)
        rc = phase(1, [&](janc_grid_s* h) {
          return launch_rk_update(h->ns, 2, sv(h, 1), sv(h, 0), sv(h, 2), h->Fx, h->Gy, h->gd, h->mech, ctl, a0, a2,
                                  h->status, nullptr, h->stream);
        }, 2, a2);
      if (!rc)
        rc = phase(0, [&](janc_grid_s* h) { return launch_face_flux(h->nv, sv(h, 2), a2, h->Fx, h->Gy, h->gd, h->stream); },
                   -1, nullptr);
      if (!rc)
        rc = phase(1, [&](janc_grid_s* h) {
          return launch_rk_update(h->ns, 3, sv(h, 2), sv(h, 0), sv(h, 0), h->Fx, h->Gy, h->gd, h->mech, ctl, a0,
                                  chem ? a3 : a4, h->status, nullptr, h->stream);
        }, chem ? -1 : 0, a4);
      if (!rc && chem)
        rc = phase(2, [&](janc_grid_s* h) { return launch_chem(h->ns, sv(h, 0), h->gd, h->mech, ctl, a0, a4, h->status, h->stream); },
                   0, a4);
      if (rc) return rc;
    }
    // the last state's alpha becomes slot 0
    e = cudaMemcpyAsync(g->alpha, g->alpha + 2 * (SLOTS_PER_STEP * nc), 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail_cuda(e, "alpha carry");
    done += nc;
  }
  for (int q = 0; q < ng; ++q) gs[q]->steps_done += n_steps;
  if (t_out || dt_last_out) {
    double c2[2];
    cudaError_t e = cudaMemcpyAsync(c2, g->clock2, sizeof(c2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "janc_step clock read");
    if (t_out) *t_out = c2[0] - t_before;
    if (dt_last_out) *dt_last_out = c2[1];
  }
  return JANC_OK;
}

extern "C" {

const char* janc_last_error(void) { return g_err.c_str(); }

int janc_workspace_bytes(const janc_grid_desc* d, const janc_mechanism* m, size_t* bytes) {
  int rc = check_desc(d, m);
  if (rc) return rc;
  if (!bytes) return fail(JANC_E_INVALID, "null output");
  *bytes = layout_of(d->nx, d->ny, m->ns + 3, false).total;
  return JANC_OK;
}

int janc_create_grid(const janc_grid_desc* d, const janc_mechanism* m, void* workspace, size_t workspace_bytes,
                     void* cuda_stream, janc_grid_t* out) {
  return janc::create_grid(d, m, workspace, workspace_bytes, cuda_stream, nullptr, out);
}

void janc_destroy_grid(janc_grid_t g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  for (auto& m : g->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : g->pool) cudaEventDestroy(e);
  if (g->owns_ws) cudaFree(g->ws);
  if (g->adj.own && g->adj.ws) cudaFree(g->adj.ws);  // a forward never reversed
  delete g->ex;
  delete g;
}

static int copy_in(janc_grid_t g, double* dst, const double* src, size_t count, int where) {
  cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(double),
                                  where == JANC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream);
  if (e == cudaSuccess && where == JANC_HOST) e = cudaStreamSynchronize(g->stream);
  return e == cudaSuccess ? JANC_OK : fail_cuda(e, "copy in");
}

static int copy_out(janc_grid_t g, double* dst, const double* src, size_t count, int where) {
  cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(double),
                                  where == JANC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream);
  if (e == cudaSuccess && where == JANC_HOST) e = cudaStreamSynchronize(g->stream);
  return e == cudaSuccess ? JANC_OK : fail_cuda(e, "copy out");
}

int janc_set_state(janc_grid_t g, const double* U, const double* T0, int where) {
  if (!g || !U) return fail(JANC_E_INVALID, "null argument");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  int rc = copy_in(g, g->S[0], U, (size_t)g->nv * g->n, where);
  if (rc) return rc;
  const double* t0 = nullptr;
  if (T0) {
    // stage the warm start in S1's T plane
    double* tp = g->S[1] + (size_t)g->nv * g->n;
    rc = copy_in(g, tp, T0, (size_t)g->n, where);
    if (rc) return rc;
    t0 = tp;
  }
  cudaError_t e = cudaMemsetAsync(g->status, 0, sizeof(int), g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->alpha, 0, 2 * sizeof(unsigned long long), g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "janc_set_state");
  e = launch_set_conserved(g->ns, sv(g, 0), t0, g->gd, g->mech, g->alpha, g->status, g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "set_conserved launch");
  if (g->ex) return g->ex->after(0, g->alpha);  // a stand-alone slab: halos and alpha of the loaded state
  return JANC_OK;
}

int janc_set_state_primitive(janc_grid_t g, const double* T, const double* p, const double* u, const double* v,
                             const double* Y, int where) {
  if (!g || !T || !p || !u || !v || !Y) return fail(JANC_E_INVALID, "null argument");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  const size_t n = (size_t)g->n;
  const double *dT = T, *dp = p, *du = u, *dv = v, *dY = Y;
  if (where == JANC_HOST) {
    // stage through S1 (4 + ns planes fit in nv + 4 = ns + 7 planes)
    double* base = g->S[1];
    int rc = copy_in(g, base, T, n, where);
    if (!rc) rc = copy_in(g, base + n, p, n, where);
    if (!rc) rc = copy_in(g, base + 2 * n, u, n, where);
    if (!rc) rc = copy_in(g, base + 3 * n, v, n, where);
    if (!rc) rc = copy_in(g, base + 4 * n, Y, (size_t)g->ns * n, where);
    if (rc) return rc;
    dT = base; dp = base + n; du = base + 2 * n; dv = base + 3 * n; dY = base + 4 * n;
  }
  cudaError_t e = cudaMemsetAsync(g->status, 0, sizeof(int), g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->alpha, 0, 2 * sizeof(unsigned long long), g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "janc_set_state_primitive");
  e = launch_set_primitive(g->ns, sv(g, 0), dT, dp, du, dv, dY, g->gd, g->mech, g->alpha, g->status, g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "set_primitive launch");
  if (g->ex) {
    const int rc = g->ex->after(0, g->alpha);
    if (rc) return rc;
  }
  if (where == JANC_HOST) {
    e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail_cuda(e, "set_primitive");
  }
  return JANC_OK;
}

int janc_step(janc_grid_t g, int n_steps, double dt, double cfl, double* t_out, double* dt_last_out) {
  if (!g) return fail(JANC_E_INVALID, "null grid");
  janc_grid_s* gs[1] = {g};
  return janc::step_grids(gs, 1, g->ex, n_steps, dt, cfl, t_out, dt_last_out);
}

int janc_source_step(janc_grid_t g, int n_steps, double dt) {
  if (!g || n_steps < 0 || !(dt > 0.0)) return fail(JANC_E_INVALID, "janc_source_step: bad argument");
  if (g->d.chemistry == JANC_CHEM_OFF) return fail(JANC_E_INVALID, "janc_source_step: the grid has no chemistry");
  if (g->halo_side[0] || g->halo_side[1]) return fail(JANC_E_UNSUPPORTED, "janc_source_step: not on an x-slab");
  StepCtl ctl;
  ctl.dt_fixed = dt;
  ctl.cfl = 0.0;
  ctl.hmin = g->gd.dx < g->gd.dy ? g->gd.dx : g->gd.dy;
  ctl.chem_frac = 1.0;
  ctl.source = 0;
  const StateView S0 = sv(g, 0);
  unsigned long long* a1 = g->alpha + 2;  // the new state's LF speeds, then slot 0
  for (int s = 0; s < n_steps; ++s) {
    cudaError_t e = cudaMemsetAsync(a1, 0, 2 * sizeof(unsigned long long), g->stream);
    if (e == cudaSuccess)
      e = timed(g, 2, [&] { return launch_chem(g->ns, S0, g->gd, g->mech, ctl, g->alpha, a1, g->status, g->stream); });
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->alpha, a1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, g->stream);
    if (e != cudaSuccess) return fail_cuda(e, "janc_source_step");
  }
  return JANC_OK;
}

int janc_get_state(janc_grid_t g, double* U, double* T, int where) {
  if (!g) return fail(JANC_E_INVALID, "null grid");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  int rc = JANC_OK;
  if (U) rc = copy_out(g, U, g->S[0], (size_t)g->nv * g->n, where);
  if (!rc && T) rc = copy_out(g, T, g->S[0] + (size_t)g->nv * g->n, (size_t)g->n, where);
  if (rc) return rc;
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, g->status, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "status read");
  if (st) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "device status word 0x%x", st);
    return fail(JANC_E_DEVICE, buf);
  }
  return JANC_OK;
}

int janc_rhs(janc_grid_t g, double* Fx, double* Gy, double* L, double* alpha, int where) {
  if (!g) return fail(JANC_E_INVALID, "null grid");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  cudaError_t e = launch_face_flux(g->nv, sv(g, 0), g->alpha, g->Fx, g->Gy, g->gd, g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "rhs flux launch");
  const int nv = g->nv, nx = g->gd.nx, ny = g->gd.ny;
  int rc = JANC_OK;
  if (Fx) rc = copy_out(g, Fx, g->Fx, (size_t)nv * ny * (nx + 1), where);
  if (!rc && Gy) rc = copy_out(g, Gy, g->Gy, (size_t)nv * (ny + 1) * nx, where);
  if (!rc && L) {
    double* tmp = g->S[1];  // nv planes of scratch
    e = launch_rhs_L(nv, g->Fx, g->Gy, tmp, g->gd, g->stream);
    if (e != cudaSuccess) return fail_cuda(e, "rhs L launch");
    rc = copy_out(g, L, tmp, (size_t)nv * g->n, where);
  }
  if (!rc && alpha) {
    unsigned long long a[2];
    e = cudaMemcpyAsync(a, g->alpha, sizeof(a), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail_cuda(e, "alpha read");
    double ad[2];
    std::memcpy(ad, a, sizeof(ad));
    if (where == JANC_HOST) {
      alpha[0] = ad[0];
      alpha[1] = ad[1];
    } else {
      e = cudaMemcpyAsync(alpha, ad, sizeof(ad), cudaMemcpyHostToDevice, g->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
      if (e != cudaSuccess) return fail_cuda(e, "alpha write");
    }
  }
  return rc;
}

int janc_profile(janc_grid_t g, int enable) {
  if (!g) return fail(JANC_E_INVALID, "null grid");
  g->prof_on = enable != 0;
  return JANC_OK;
}

int janc_profile_read(janc_grid_t g, double* ms, long long* launches) {
  if (!g || !ms || !launches) return fail(JANC_E_INVALID, "null argument");
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "janc_profile_read");
  for (int c = 0; c < 3; ++c) { ms[c] = 0.0; launches[c] = 0; }
  for (auto& m : g->marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess && m.cls >= 0 && m.cls < 3) {
      ms[m.cls] += t;
      launches[m.cls] += 1;
    }
    g->pool.push_back(m.a);
    g->pool.push_back(m.b);
  }
  g->marks.clear();
  return JANC_OK;
}

int janc_status(janc_grid_t g, janc_status_info* s) {
  if (!g || !s) return fail(JANC_E_INVALID, "null argument");
  int st = 0;
  double c2[2];
  unsigned long long a[2];
  cudaError_t e = cudaMemcpyAsync(&st, g->status, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c2, g->clock2, sizeof(c2), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a, g->alpha, sizeof(a), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return fail_cuda(e, "janc_status");
  s->status = st;
  s->steps_done = g->steps_done;
  s->t = c2[0];
  s->dt_last = c2[1];
  std::memcpy(s->alpha, a, sizeof(s->alpha));
  return JANC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Discrete adjoint (see janc_adjoint.cu for the operator transposes).
// ---------------------------------------------------------------------------
namespace {

struct AdjLayout {
  size_t state, ckpt, seg, alog, lin, lin_stage, clin, clin_step, lam, cfx, cfy, small, total;
  int ncp, seglen;
  int nstore;  // segment stores: 2 when segments are recomputed (the next one while the current is reversed)
};

// mode: JANC_ADJ_STORE_FACES adds to each segment store the face derivatives
// of its 3 ckpt_every stage states (lin_stage doubles each) and, per step
// (clin_step doubles), the chemistry factors of point-implicit chemistry or
// the rate constants of the explicit source at its three stage inputs.
AdjLayout adj_layout(const janc_grid_s* g, int n_steps, int ckpt_every, int mode) {
  AdjLayout L;
  const size_t n = (size_t)g->n;
  const int nv = g->nv;
  L.seglen = ckpt_every;
  L.ncp = n_steps > 0 ? (n_steps + ckpt_every - 1) / ckpt_every : 1;
  L.state = align256(sizeof(double) * (size_t)(nv + 4) * n);
  L.ckpt = (size_t)L.ncp * (L.state + 256);              // state + its alpha pair
  L.nstore = L.ncp > 1 ? 2 : 1;
  L.seg = (size_t)(4 * ckpt_every + 1) * L.state;        // S0[0..len], S1, S2, S* per step (one store)
  L.alog = align256(sizeof(unsigned long long) * 10 * ckpt_every);
  L.lin_stage = mode == JANC_ADJ_STORE_FACES ? face_lin_doubles(nv, g->gd) : 0;
  L.lin = align256(sizeof(double) * L.lin_stage * 3 * (size_t)ckpt_every);
  L.clin_step = 0;
  if (mode == JANC_ADJ_STORE_FACES && g->d.chemistry == JANC_CHEM_LIE) L.clin_step = chem_lin_entries(g->ns, g->nr) * n;
  if (mode == JANC_ADJ_STORE_FACES && g->d.chemistry == JANC_CHEM_EXPLICIT && g->ns > 1)
    L.clin_step = 3 * 2 * (size_t)g->nr * n;
  L.clin = align256(sizeof(double) * L.clin_step * (size_t)ckpt_every);
  L.lam = 7 * align256(sizeof(double) * (size_t)nv * n);
  L.cfx = align256(sizeof(double) * (size_t)nv * g->gd.ny * (g->gd.nx + 1) * 10);
  L.cfy = align256(sizeof(double) * (size_t)nv * (g->gd.ny + 1) * g->gd.nx * 10);
  L.small = 256 + rhs_vjp_scratch_bytes(g->gd);  // [0] loss, then the RHS-VJP scratch at +256
  L.total = L.ckpt + L.nstore * (L.seg + L.alog + L.lin + L.clin) + L.lam + L.cfx + L.cfy + L.small;
  return L;
}

}  // namespace

extern "C" {

int janc_adjoint_workspace_bytes(janc_grid_t g, int n_steps, int ckpt_every, size_t* bytes) {
  if (!g || !bytes || n_steps < 0 || ckpt_every <= 0) return fail(JANC_E_INVALID, "bad argument");
  *bytes = adj_layout(g, n_steps, ckpt_every, g->adj_mode).total;
  return JANC_OK;
}

int janc_set_adjoint_mode(janc_grid_t g, int mode) {
  if (!g) return fail(JANC_E_INVALID, "null grid");
  if (mode != JANC_ADJ_RECOMPUTE && mode != JANC_ADJ_STORE_FACES) return fail(JANC_E_INVALID, "adjoint mode");
  g->adj_mode = mode;
  return JANC_OK;
}

int janc_rhs_vjp(janc_grid_t g, const double* mu, double* nu, void* workspace, size_t workspace_bytes, int where) {
  if (!g || !mu || !nu) return fail(JANC_E_INVALID, "null argument");
  if (g->halo_side[0] || g->halo_side[1]) return fail(JANC_E_UNSUPPORTED, "janc_rhs_vjp runs on whole grids, not x-slabs");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  const size_t nvn = (size_t)g->nv * g->n;
  const size_t bx = align256(sizeof(double) * (size_t)g->nv * g->gd.ny * (g->gd.nx + 1) * 10);
  const size_t by = align256(sizeof(double) * (size_t)g->nv * (g->gd.ny + 1) * g->gd.nx * 10);
  const size_t need = 2 * align256(sizeof(double) * nvn) + bx + by + rhs_vjp_scratch_bytes(g->gd);
  char* ws = (char*)workspace;
  bool own = false;
  if (!ws) {
    if (cudaMalloc(&ws, need) != cudaSuccess) return fail(JANC_E_NOMEM, "janc_rhs_vjp: cudaMalloc failed");
    own = true;
  } else if (workspace_bytes < need) {
    return fail(JANC_E_NOMEM, "janc_rhs_vjp: workspace too small");
  }
  double* dmu = (double*)ws;
  double* dnu = (double*)(ws + align256(sizeof(double) * nvn));
  double* cfx = (double*)(ws + 2 * align256(sizeof(double) * nvn));
  double* cfy = (double*)((char*)cfx + bx);
  double* scratch = (double*)((char*)cfy + by);
  int rc = JANC_OK;
  cudaError_t e = cudaMemcpyAsync(dmu, mu, sizeof(double) * nvn,
                                  where == JANC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream);
  if (e == cudaSuccess)
    e = launch_rhs_vjp(g->ns, sv(g, 0), (const double*)g->alpha,
                       VjpIO{dmu, 1.0, dnu, nullptr, 0.0, 0, nullptr, nullptr, 0.0, 0}, cfx, cfy, scratch, g->gd,
                       g->mech, nullptr, true, false, nullptr, g->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nu, dnu, sizeof(double) * nvn,
                        where == JANC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) rc = fail_cuda(e, "janc_rhs_vjp");
  if (own) cudaFree(ws);
  return rc;
}

}  // extern "C"

namespace {

// One segment store: the states of a segment, their alpha log and (mode
// JANC_ADJ_STORE_FACES) the face derivatives of every stage state.
struct SegStore {
  char* seg;
  unsigned long long* alog;
  double* lin;   // null in mode JANC_ADJ_RECOMPUTE
  double* clin;  // chemistry factors; null in mode JANC_ADJ_RECOMPUTE or without point-implicit chemistry
};

// Pointers into an adjoint workspace (see adj_layout).
struct AdjPtrs {
  char* ckpt;
  SegStore store[2];  // store[c % nstore] holds segment c
  double* lam[7];
  double* cfx;
  double* cfy;
  double* small;  // [0] loss; from +256 bytes the RHS-VJP scratch
};

AdjPtrs adj_ptrs(const janc_grid_s* g, const AdjLayout& L, char* ws) {
  AdjPtrs q;
  const size_t lamb = align256(sizeof(double) * (size_t)g->nv * (size_t)g->n);
  char* p = ws;
  q.ckpt = p; p += L.ckpt;
  for (int k = 0; k < L.nstore; ++k) {
    q.store[k].seg = p; p += L.seg;
    q.store[k].alog = (unsigned long long*)p; p += L.alog;
    q.store[k].lin = L.lin_stage ? (double*)p : nullptr; p += L.lin;
    q.store[k].clin = L.clin_step ? (double*)p : nullptr; p += L.clin;
  }
  if (L.nstore == 1) q.store[1] = q.store[0];
  for (int k = 0; k < 7; ++k) { q.lam[k] = (double*)p; p += lamb; }
  q.cfx = (double*)p; p += L.cfx;
  q.cfy = (double*)p; p += L.cfy;
  q.small = (double*)p;
  return q;
}

StepCtl adj_ctl(const janc_grid_s* g, double dt) {
  StepCtl ctl;
  ctl.dt_fixed = dt;
  ctl.cfl = 0.0;
  ctl.hmin = g->gd.dx < g->gd.dy ? g->gd.dx : g->gd.dy;
  ctl.chem_frac = 1.0;
  ctl.source = g->d.chemistry == JANC_CHEM_EXPLICIT ? 1 : 0;
  return ctl;
}

void adj_release(janc_grid_s* g) {
  if (g->adj.own && g->adj.ws) cudaFree(g->adj.ws);
  g->adj = janc_grid_s::AdjPending();
}

// Segment store: slots 0..len hold U^{m0+m} (with T and the aux planes),
// then S1, S2, S* of every step of the segment.
StateView seg_S0(const SegStore& q, const AdjLayout& L, int m) {
  return StateView{(double*)(q.seg + (size_t)m * L.state)};
}
StateView seg_S(const SegStore& q, const AdjLayout& L, int m, int which) {  // which: 1 = S1, 2 = S2, 3 = S*
  return StateView{(double*)(q.seg + (size_t)(L.seglen + 1 + 3 * m + which - 1) * L.state)};
}
// Face derivatives of RK stage s (0: U^n, 1: U1, 2: U2) of step m, or null.
const double* seg_lin(const SegStore& q, const AdjLayout& L, int m, int s) {
  return q.lin ? q.lin + (size_t)(3 * m + s) * L.lin_stage : nullptr;
}
// Chemistry factors of step m, or null.
double* seg_clin(const SegStore& q, const AdjLayout& L, int m) {
  return q.clin ? q.clin + (size_t)m * L.clin_step : nullptr;
}
// Explicit source: the rate constants at the input of RK stage s (0..2) of step m, or null.
double* seg_src(const SegStore& q, const AdjLayout& L, int m, int s) {
  return q.clin ? q.clin + (size_t)m * L.clin_step + (size_t)s * (L.clin_step / 3) : nullptr;
}

// `len` fixed-dt steps of the Lie (or explicit-source) order from segment
// slot 0, whose alpha pair is in alog[0..1], keeping every stage state in
// the segment store and every alpha in alog (10 slots per step: U^n, U1, U2,
// U*, U^{n+1}). The kernels and their order are those of janc_step, so the
// stored trajectory is the forward's, bit for bit. With `clock` the simulated
// time advances as in janc_step; with `loss` the end-wall loss of every new
// state accumulates into loss[0]. Runs on stream st; it uses the grid's face
// flux arrays, so two segments never run at once.
cudaError_t adj_segment(janc_grid_s* g, const AdjLayout& L, const SegStore& q, int len, const StepCtl& ctl,
                        double* clock, double* loss, double w_loss, cudaStream_t st) {
  const int nv = g->nv;
  const bool chem = g->d.chemistry == JANC_CHEM_LIE;
  const bool src = g->d.chemistry == JANC_CHEM_EXPLICIT;
  unsigned long long* alog = q.alog;
  // the explicit source's rate constants at stage s's input, when the store keeps them
  auto keep = [&](int m, int s) { return src ? seg_src(q, L, m, s) : nullptr; };
  // the face fluxes of stage s of step m, with its derivatives when the store keeps them
  auto flux = [&](const StateView& Sin, const unsigned long long* a, int m, int s) {
    if (!q.lin) return launch_face_flux(nv, Sin, a, g->Fx, g->Gy, g->gd, st);
    return launch_face_flux_lin(nv, Sin, a, g->Fx, g->Gy, q.lin + (size_t)(3 * m + s) * L.lin_stage, g->gd, st);
  };
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < len && e == cudaSuccess; ++m) {
    unsigned long long* a = alog + 10 * m;
    if (m > 0) e = cudaMemcpyAsync(a, alog + 10 * (m - 1) + 8, 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = flux(seg_S0(q, L, m), a, m, 0);
    if (e == cudaSuccess)
      e = launch_rk_update(g->ns, 1, seg_S0(q, L, m), seg_S0(q, L, m), seg_S(q, L, m, 1), g->Fx, g->Gy, g->gd,
                           g->mech, ctl, a, a + 2, g->status, clock, st, keep(m, 0));
    if (e == cudaSuccess) e = flux(seg_S(q, L, m, 1), a + 2, m, 1);
    if (e == cudaSuccess)
      e = launch_rk_update(g->ns, 2, seg_S(q, L, m, 1), seg_S0(q, L, m), seg_S(q, L, m, 2), g->Fx, g->Gy, g->gd,
                           g->mech, ctl, a, a + 4, g->status, nullptr, st, keep(m, 1));
    if (e == cudaSuccess) e = flux(seg_S(q, L, m, 2), a + 4, m, 2);
    if (e == cudaSuccess)
      e = launch_rk_update(g->ns, 3, seg_S(q, L, m, 2), seg_S0(q, L, m), seg_S(q, L, m, 3), g->Fx, g->Gy, g->gd,
                           g->mech, ctl, a, chem ? a + 6 : a + 8, g->status, nullptr, st, keep(m, 2));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(seg_S0(q, L, m + 1).base, seg_S(q, L, m, 3).base, L.state, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && chem) {
      if (q.clin)
        e = launch_chem_lin(g->ns, seg_S0(q, L, m + 1), g->gd, g->mech, ctl, a, a + 8, g->status, seg_clin(q, L, m),
                            st);
      else
        e = launch_chem(g->ns, seg_S0(q, L, m + 1), g->gd, g->mech, ctl, a, a + 8, g->status, st);
    }
    if (e == cudaSuccess && loss) e = launch_loss_endwall(g->ns, seg_S0(q, L, m + 1), g->gd, w_loss, loss, st);
  }
  return e;
}

}  // namespace

extern "C" {

int janc_adjoint_forward(janc_grid_t g, int n_steps, double dt, int ckpt_every, int loss_kind, double* loss_out,
                         void* workspace, size_t workspace_bytes) {
  if (!g || n_steps < 0 || !(dt > 0.0) || ckpt_every <= 0) return fail(JANC_E_INVALID, "bad argument");
  if (loss_kind != JANC_LOSS_ENDWALL_P && loss_kind != JANC_LOSS_SEEDED) return fail(JANC_E_INVALID, "loss kind");
  if (g->d.chemistry == JANC_CHEM_STRANG) return fail(JANC_E_UNSUPPORTED, "the adjoint reverses the Lie order only");
  if (g->halo_side[0] || g->halo_side[1]) return fail(JANC_E_UNSUPPORTED, "the adjoint runs on whole grids, not x-slabs");
  adj_release(g);
  const int mode = g->adj_mode;
  const AdjLayout L = adj_layout(g, n_steps, ckpt_every, mode);
  char* ws = (char*)workspace;
  bool own = false;
  if (!ws) {
    if (cudaMalloc(&ws, L.total) != cudaSuccess) return fail(JANC_E_NOMEM, "janc_adjoint_forward: cudaMalloc failed");
    own = true;
  } else if (workspace_bytes < L.total || ((uintptr_t)ws & 255u)) {
    return fail(JANC_E_NOMEM, "janc_adjoint_forward: workspace too small or misaligned");
  }
  cudaStream_t st = g->stream;
  const AdjPtrs q = adj_ptrs(g, L, ws);
  auto ckpt_state = [&](int c) { return StateView{(double*)(q.ckpt + (size_t)c * (L.state + 256))}; };
  auto ckpt_alpha = [&](int c) { return (unsigned long long*)(q.ckpt + (size_t)c * (L.state + 256) + L.state); };
  const double w_loss = dt / g->gd.ny;
  // The steps of the last nstore segments (one per segment store) run
  // straight into the stores, so that the reverse sweep starts on them
  // without recomputing anything; with ckpt_every >= n_steps nothing is
  // recomputed at all.
  const int m_first = (L.ncp - L.nstore) * ckpt_every;
  int rc = JANC_OK;
  cudaError_t e = cudaMemsetAsync(q.small, 0, 256, st);
  for (int s = 0; s < n_steps && e == cudaSuccess;) {
    if (s % ckpt_every == 0) {
      const int c = s / ckpt_every;
      e = cudaMemcpyAsync(ckpt_state(c).base, g->S[0], L.state, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ckpt_alpha(c), g->alpha, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) break;
    if (s >= m_first) {  // s is the first step of segment s / ckpt_every
      const int len = (n_steps - s) < ckpt_every ? (n_steps - s) : ckpt_every;
      const SegStore& sq = q.store[(s / ckpt_every) % L.nstore];
      e = cudaMemcpyAsync(seg_S0(sq, L, 0).base, g->S[0], L.state, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(sq.alog, 0, L.alog, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(sq.alog, g->alpha, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = adj_segment(g, L, sq, len, adj_ctl(g, dt), g->clock2,
                        loss_kind == JANC_LOSS_ENDWALL_P ? q.small : nullptr, w_loss, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->S[0], seg_S0(sq, L, len).base, L.state, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->alpha, sq.alog + 10 * (len - 1) + 8, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, st);
      g->steps_done += len;
      s += len;
      continue;
    }
    rc = janc_step(g, 1, dt, 0.0, nullptr, nullptr);
    if (rc) break;
    if (loss_kind == JANC_LOSS_ENDWALL_P) e = launch_loss_endwall(g->ns, sv(g, 0), g->gd, w_loss, q.small, st);
    ++s;
  }
  if (!rc && e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, q.small, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (!rc && e != cudaSuccess) rc = fail_cuda(e, "janc_adjoint_forward");
  if (rc) {
    if (own) cudaFree(ws);
    return rc;
  }
  g->adj.valid = true;
  g->adj.n_steps = n_steps;
  g->adj.ckpt_every = ckpt_every;
  g->adj.loss_kind = loss_kind;
  g->adj.mode = mode;
  g->adj.dt = dt;
  g->adj.ws = ws;
  g->adj.own = own;
  return JANC_OK;
}

int janc_adjoint_reverse(janc_grid_t g, const double* seed, double* dL_dU0, int where) {
  if (!g || !dL_dU0) return fail(JANC_E_INVALID, "null argument");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  if (!g->adj.valid) return fail(JANC_E_INVALID, "janc_adjoint_reverse: no pending janc_adjoint_forward");
  const int n_steps = g->adj.n_steps, ckpt_every = g->adj.ckpt_every, loss_kind = g->adj.loss_kind;
  const double dt = g->adj.dt;
  const AdjLayout L = adj_layout(g, n_steps, ckpt_every, g->adj.mode);
  const AdjPtrs q = adj_ptrs(g, L, g->adj.ws);
  cudaStream_t st = g->stream;
  const size_t n = (size_t)g->n;
  const int nv = g->nv;
  const size_t nvn = (size_t)nv * n;
  auto ckpt_state = [&](int c) { return StateView{(double*)(q.ckpt + (size_t)c * (L.state + 256))}; };
  auto ckpt_alpha = [&](int c) { return (unsigned long long*)(q.ckpt + (size_t)c * (L.state + 256) + L.state); };
  const bool chem = g->d.chemistry == JANC_CHEM_LIE;
  const bool src = g->d.chemistry == JANC_CHEM_EXPLICIT;
  const double w_loss = dt / g->gd.ny;
  const StepCtl ctl = adj_ctl(g, dt);
  double* cfx = q.cfx;
  double* cfy = q.cfy;
  double* small = q.small;
  double* lamN = q.lam[0];  // cotangent of U^{m+1}
  double* lamS = q.lam[1];  // of U*
  double* lam2 = q.lam[2];
  double* lam1 = q.lam[3];
  double* lam0 = q.lam[4];
  cudaError_t e = cudaSuccess;
  if (seed) e = cudaMemcpyAsync(lamN, seed, sizeof(double) * nvn,
                                where == JANC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
  else e = cudaMemsetAsync(lamN, 0, sizeof(double) * nvn, st);
  // the RHS VJPs of the sweep find the per-position sums and the alpha
  // cotangents zero and leave them zero
  if (e == cudaSuccess) e = cudaMemsetAsync(cfx, 0, L.cfx, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cfy, 0, L.cfy, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(small + 32, 0, 2 * sizeof(double), st);
  // The forward left its last nstore segments in the stores. The others are
  // recomputed from their checkpoints on a second stream, one segment ahead
  // of the reverse sweep: segment c - 2 goes into store c % 2 once segment
  // c's reverse has finished with it, and is recomputed while segment c - 1
  // is reversed.
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_rev = nullptr;
  auto seg_len = [&](int c) {
    const int m0 = c * ckpt_every;
    return (n_steps - m0) < ckpt_every ? (n_steps - m0) : ckpt_every;
  };
  auto recompute = [&](int c) {  // segment c into store c % 2, on s2
    const SegStore& sq = q.store[c % L.nstore];
    cudaError_t r = cudaMemcpyAsync(seg_S0(sq, L, 0).base, ckpt_state(c).base, L.state, cudaMemcpyDeviceToDevice, s2);
    if (r == cudaSuccess) r = cudaMemsetAsync(sq.alog, 0, L.alog, s2);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(sq.alog, ckpt_alpha(c), 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s2);
    if (r == cudaSuccess) r = adj_segment(g, L, sq, seg_len(c), ctl, nullptr, nullptr, 0.0, s2);
    if (r == cudaSuccess) r = cudaEventRecord(ev_rec[c % 2], s2);
    return r;
  };
  // With recomputation the sweep runs on an internal stream of the highest
  // priority and the recompute on one of the lowest.
  const int n_fwd = L.nstore;  // trailing segments the forward left in the stores
  cudaStream_t s1 = nullptr;
  if (e == cudaSuccess && L.ncp > n_fwd && n_steps > 0) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s1, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, least);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev_rec[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_rev, cudaEventDisableTiming);
    // both start after everything enqueued on the grid's stream so far
    if (e == cudaSuccess) e = cudaEventRecord(ev_rev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev_rev, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s1, ev_rev, 0);
    if (e == cudaSuccess) st = s1;
  }
  for (int c = L.ncp - 1; c >= 0 && e == cudaSuccess && n_steps > 0; --c) {
    const int len = seg_len(c);
    const SegStore& sq = q.store[c % L.nstore];
    const unsigned long long* alog = sq.alog;
    auto segS0 = [&](int m) { return seg_S0(sq, L, m); };
    auto segS = [&](int m, int which) { return seg_S(sq, L, m, which); };
    // the forward left the last n_fwd segments in their stores; the others come from s2
    if (c < L.ncp - n_fwd) e = cudaStreamWaitEvent(st, ev_rec[c % 2], 0);
    // reverse through the segment
    for (int m = len - 1; m >= 0 && e == cudaSuccess; --m) {
      const unsigned long long* a = alog + 10 * m;
      if (loss_kind == JANC_LOSS_ENDWALL_P)
        e = launch_seed_endwall(g->ns, segS0(m + 1), g->gd, g->mech, w_loss, lamN, st);
      if (e == cudaSuccess) {
        if (chem) e = launch_chem_vjp(g->ns, segS(m, 3), g->gd, g->mech, dt, lamN, lamS, seg_clin(sq, L, m), st);
        else e = cudaMemcpyAsync(lamS, lamN, sizeof(double) * nvn, cudaMemcpyDeviceToDevice, st);
      }
      // Each stage's RHS VJP takes mu = c dt lam directly and writes the
      // stage's combinations itself (VjpIO); in the explicit source-term form
      // its cell pass also adds the source's VJP at the stage state.
      // stage 3: U* = U^n/3 + 2/3 (U2 + dt L(U2)): lam2 = 2/3 lamS + L^T mu, lam0 = lamS / 3
      const VjpIO io3{lamS, 2.0 / 3.0 * dt, lam2, lamS, 2.0 / 3.0, 0, lam0, lamS, 1.0 / 3.0, 0};
      if (e == cudaSuccess)
        e = launch_rhs_vjp(g->ns, segS(m, 2), (const double*)(a + 4), io3, cfx, cfy, small + 32, g->gd, g->mech,
                           seg_lin(sq, L, m, 2), false, src, src ? seg_src(sq, L, m, 2) : nullptr, st);
      // stage 2: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1)): lam1 = lam2 / 4 + L^T mu, lam0 += 3/4 lam2
      const VjpIO io2{lam2, 0.25 * dt, lam1, lam2, 0.25, 0, lam0, lam2, 0.75, 1};
      if (e == cudaSuccess)
        e = launch_rhs_vjp(g->ns, segS(m, 1), (const double*)(a + 2), io2, cfx, cfy, small + 32, g->gd, g->mech,
                           seg_lin(sq, L, m, 1), false, src, src ? seg_src(sq, L, m, 1) : nullptr, st);
      // stage 1: U1 = U^n + dt L(U^n): lam0 += lam1 + L^T mu
      const VjpIO io1{lam1, dt, lam0, lam1, 1.0, 1, nullptr, nullptr, 0.0, 0};
      if (e == cudaSuccess)
        e = launch_rhs_vjp(g->ns, segS0(m), (const double*)a, io1, cfx, cfy, small + 32, g->gd, g->mech,
                           seg_lin(sq, L, m, 0), false, src, src ? seg_src(sq, L, m, 0) : nullptr, st);
      std::swap(lamN, lam0);
    }
    // segment c's store is free once its reverse is done: refill it with c - 2
    if (e == cudaSuccess && c - 2 >= 0) {
      e = cudaEventRecord(ev_rev, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev_rev, 0);
      if (e == cudaSuccess) e = recompute(c - 2);
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dL_dU0, lamN, sizeof(double) * nvn,
                        where == JANC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (s2) {
    const cudaError_t e2 = cudaStreamSynchronize(s2);  // nothing is left on it once st is done; a failure shows here
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(s2);
  }
  if (s1) {
    const cudaError_t e1 = cudaStreamSynchronize(s1);
    if (e == cudaSuccess) e = e1;
    cudaStreamDestroy(s1);
  }
  for (int k = 0; k < 2; ++k)
    if (ev_rec[k]) cudaEventDestroy(ev_rec[k]);
  if (ev_rev) cudaEventDestroy(ev_rev);
  adj_release(g);
  if (e != cudaSuccess) return fail_cuda(e, "janc_adjoint_reverse");
  return JANC_OK;
}

int janc_step_adjoint(janc_grid_t g, int n_steps, double dt, int ckpt_every, int loss_kind, const double* seed,
                      double* dL_dU0, double* loss_out, void* workspace, size_t workspace_bytes, int where) {
  if (!g || n_steps < 0 || !(dt > 0.0) || ckpt_every <= 0) return fail(JANC_E_INVALID, "bad argument");
  if (loss_kind != JANC_LOSS_ENDWALL_P && loss_kind != JANC_LOSS_SEEDED) return fail(JANC_E_INVALID, "loss kind");
  if (loss_kind == JANC_LOSS_SEEDED && !seed) return fail(JANC_E_INVALID, "seeded loss needs a seed");
  if (where != JANC_HOST && where != JANC_DEVICE) return fail(JANC_E_INVALID, "bad where");
  double loss = 0.0;
  int rc = janc_adjoint_forward(g, n_steps, dt, ckpt_every, loss_kind, &loss, workspace, workspace_bytes);
  if (rc) return rc;
  if (loss_kind == JANC_LOSS_SEEDED) {  // loss = <seed, U^N>
    const AdjLayout L = adj_layout(g, n_steps, ckpt_every, g->adj.mode);
    const AdjPtrs q = adj_ptrs(g, L, g->adj.ws);
    const size_t nvn = (size_t)g->nv * (size_t)g->n;
    double* dseed = q.lam[6];
    cudaError_t e = cudaMemcpyAsync(dseed, seed, sizeof(double) * nvn,
                                    where == JANC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q.small, 0, sizeof(double), g->stream);
    if (e == cudaSuccess) e = launch_dot((long long)nvn, dseed, g->S[0], q.small, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, q.small, sizeof(double), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
      adj_release(g);
      return fail_cuda(e, "janc_step_adjoint");
    }
  }
  if (loss_out) *loss_out = loss;
  if (!dL_dU0) {
    adj_release(g);
    return JANC_OK;
  }
  return janc_adjoint_reverse(g, loss_kind == JANC_LOSS_SEEDED ? seed : nullptr, dL_dU0, where);
}

int janc_primitive_T_vjp(janc_grid_t g, const double* T, const double* p, const double* u, const double* v,
                         const double* Y, const double* dL_dU, double* dL_dT) {
  if (!g || !T || !p || !u || !v || !Y || !dL_dU || !dL_dT) return fail(JANC_E_INVALID, "null argument");
  cudaError_t e = launch_prim_T_vjp(g->ns, T, p, u, v, Y, dL_dU, dL_dT, g->gd, g->mech, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  return e == cudaSuccess ? JANC_OK : fail_cuda(e, "janc_primitive_T_vjp");
}

}  // extern "C"
