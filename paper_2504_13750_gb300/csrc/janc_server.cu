// Continuous-batching server: many independent solves (grids of different
// sizes and mixtures, one mechanism) advanced together on one GPU.
//
// Requests wait in a FIFO queue and are admitted, in arrival order with
// skip-ahead, whenever their device footprint fits the free part of one HBM
// pool and a slot is free. Every admitted request keeps its whole state on
// the device. A macro-step advances every active request by one time step
// (advance_one_step, Sec. 4.3 of arXiv 2504.13750) with one persistent
// kernel per phase that walks a flattened (request, tile) list: the batched
// face-flux, stage-update and chemistry kernels run the same per-tile device
// code as the single-grid path, with per-request alpha, dt and status slots,
// so a request's result does not depend on what it shares the GPU with.
// A request that has done its steps leaves the active set at once; its final
// state is copied to pinned host memory on a second stream and its pool
// memory returns to the free list when that copy has finished. Requests that
// arrive meanwhile join at the next macro-step.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/janc.h"
#include "janc_device.cuh"
#include "janc_host.h"
#include "janc_internal.h"

using namespace janc;
using janc::host::Pool;

namespace {

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum RState { R_QUEUED = 0, R_ACTIVE = 1, R_COPYING = 2, R_DONE = 3, R_FAILED = 4, R_FETCHED = 5 };

struct Req {
  int id = 0;
  janc_grid_desc d;
  int n_steps = 0;
  double dt = 0.0, cfl = 0.0;
  int steps_done = 0;
  RState state = R_QUEUED;
  long long n = 0;
  double* host = nullptr;  // pinned: (4 + ns) planes of initial fields, later U and T, then t, status
  size_t host_doubles = 0;
  size_t footprint = 0, off = 0;
  BatchReq br;
  int fresh = 0;
  cudaEvent_t ev_done = nullptr, ev_copy = nullptr;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  bool reported = false;  // returned as finished by janc_server_run_until
};

// Device footprint of one request: 3 states, face fluxes, 5 alpha slots +
// clock + status in one 256-byte piece.
void req_layout(int nx, int ny, int nv, size_t* state, size_t* fx, size_t* gy, size_t* small, size_t* total) {
  const size_t n = (size_t)nx * ny;
  *state = a256(sizeof(double) * (size_t)(nv + 4) * n);
  *fx = a256(sizeof(double) * (size_t)nv * ny * (nx + 1));
  *gy = a256(sizeof(double) * (size_t)nv * (ny + 1) * nx);
  *small = 256;
  *total = 3 * *state + *fx + *gy + *small;
}

}  // namespace

struct janc_server_s {
  int ns = 0, nv = 0, chem = 0;
  MechDev* dmech = nullptr;
  bool chem_fixed = false;  // the mechanism has the compiled reaction structure
  char* pool_base = nullptr;
  bool owns_pool = false;
  Pool pool;
  int max_active = 0;
  long long cell_budget = 0;   // cap on the active set's cells (0: none)
  double max_skip_s = 0.0;     // how long later requests may pass a budget-blocked one
  long long active_cells = 0;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  std::vector<Req*> reqs;
  std::deque<int> queue;
  std::vector<int> active;
  bool dirty = true;
  BatchReq* d_reqs = nullptr;
  int* d_first = nullptr;  // 3 x (max_active + 1): flux, update, chemistry
  char* h_stage[2] = {nullptr, nullptr};
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  int stage_k = 0;
  int tot[3] = {0, 0, 0};
  long long macro_steps = 0;
  janc_grid_desc defaults;
  // janc_server_run_until keeps at most two macro-steps in flight: the event
  // of each macro-step's end, alternating
  cudaEvent_t step_ev[2] = {nullptr, nullptr};
  int step_k = 0;
};

namespace {

int sfail(int code, const std::string& m) {
  set_last_error(m.c_str());
  return code;
}
int scuda(cudaError_t e, const char* where) {
  return sfail(JANC_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t stage_bytes(int max_active) {
  return a256(sizeof(BatchReq) * max_active) + a256(sizeof(int) * 3 * (max_active + 1));
}

// Descriptor of an admitted request (pointers into its pool piece).
void fill_batchreq(janc_server_s* s, Req* r) {
  char* base = s->pool_base + r->off;
  size_t st, fx, gy, sm, tot;
  req_layout(r->d.nx, r->d.ny, s->nv, &st, &fx, &gy, &sm, &tot);
  BatchReq& b = r->br;
  std::memset(&b, 0, sizeof b);
  GridDev& g = b.g;
  g.nx = r->d.nx;
  g.ny = r->d.ny;
  g.n = r->n;
  g.dx = r->d.dx;
  g.dy = r->d.dy;
  g.rdx = 1.0 / r->d.dx;
  g.rdy = 1.0 / r->d.dy;
  for (int k = 0; k < 4; ++k) g.bc[k] = r->d.bc[k];
  g.eps4 = 4.0 * (r->d.weno_eps > 0.0 ? r->d.weno_eps : 1e-6);
  g.newton_tol = r->d.newton_tol > 0.0 ? r->d.newton_tol : 1e-12;
  g.newton_maxit = r->d.newton_maxit > 0 ? r->d.newton_maxit : 50;
  g.chem_fixed = s->chem_fixed ? 1 : 0;
  for (int k = 0; k < 3; ++k) b.S[k].base = (double*)(base + k * st);
  b.Fx = (double*)(base + 3 * st);
  b.Gy = (double*)(base + 3 * st + fx);
  char* small = base + 3 * st + fx + gy;
  b.alpha = (unsigned long long*)small;          // 5 slots = 80 B
  b.clock2 = (double*)(small + 80);               // 16 B
  b.status = (int*)(small + 96);                  // 4 B
  b.mech = s->dmech;
  b.ctl.dt_fixed = r->dt > 0.0 ? r->dt : 0.0;
  b.ctl.cfl = r->cfl > 0.0 ? r->cfl : 0.0;
  b.ctl.chem_frac = 1.0;
  b.ctl.source = 0;
  b.ctl.hmin = g.dx < g.dy ? g.dx : g.dy;
  int tot_f;
  face_flux_tiles(g, &b.nbx, &b.ntx_x, &b.ntx_y, &tot_f);
  update_blocks(g, &b.ubx, &b.uby);
}

int admit(janc_server_s* s, Req* r) {
  fill_batchreq(s, r);
  BatchReq& b = r->br;
  cudaError_t e = cudaMemsetAsync(b.alpha, 0, 128, s->stream);
  const size_t n = (size_t)r->n;
  double* stage = b.S[1].base;  // initial fields staged in S1
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(stage, r->host, sizeof(double) * (4 + s->ns) * n, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = launch_set_primitive(s->ns, b.S[0], stage, stage + n, stage + 2 * n, stage + 3 * n, stage + 4 * n, b.g,
                             s->dmech, b.alpha, b.status, s->stream);
  if (e != cudaSuccess) return scuda(e, "admission");
  r->state = R_ACTIVE;
  r->fresh = 1;
  r->t_admit = now_s();
  s->active.push_back(r->id);
  s->active_cells += r->n;
  s->dirty = true;
  return JANC_OK;
}

// One admission pass (janc_host.h): slots, cell budget with aging, pool.
void try_admit(janc_server_s* s) {
  janc::host::admission_pass(
      s->queue, s->pool, s->max_active, s->cell_budget, s->max_skip_s, now_s(),
      [&](int id) {
        const Req* r = s->reqs[id];
        return janc::host::Pending{r->n, r->footprint, r->t_submit};
      },
      [&] { return (int)s->active.size(); }, [&] { return s->active_cells; },
      [&](int id, size_t off) {
        Req* r = s->reqs[id];
        r->off = off;
        if (admit(s, r) == JANC_OK) return true;
        r->state = R_FAILED;
        return false;
      });
}

void reap(janc_server_s* s) {
  for (Req* r : s->reqs) {
    if (!r || r->state != R_COPYING) continue;
    if (cudaEventQuery(r->ev_copy) == cudaSuccess) {
      s->pool.release(r->off, r->footprint);
      const size_t un = (size_t)(s->nv + 1) * r->n;
      int st = 0;
      std::memcpy(&st, r->host + un + 2, sizeof(int));
      r->state = st ? R_FAILED : R_DONE;
      r->t_done = now_s();
    }
  }
}

int upload(janc_server_s* s) {
  const int na = (int)s->active.size();
  char* h = s->h_stage[s->stage_k];
  cudaError_t e = cudaEventSynchronize(s->stage_ev[s->stage_k]);  // previous use of this staging half
  if (e != cudaSuccess) return scuda(e, "staging wait");
  BatchReq* hb = (BatchReq*)h;
  int* hf = (int*)(h + a256(sizeof(BatchReq) * s->max_active));
  int acc[3] = {0, 0, 0};
  for (int q = 0; q < na; ++q) {
    Req* r = s->reqs[s->active[q]];
    r->br.fresh = r->fresh;
    hb[q] = r->br;
    int nbx, ntx, nty, tf;
    face_flux_tiles(r->br.g, &nbx, &ntx, &nty, &tf);
    hf[q] = acc[0];
    hf[(s->max_active + 1) + q] = acc[1];
    hf[2 * (s->max_active + 1) + q] = acc[2];
    acc[0] += tf;
    acc[1] += r->br.ubx * r->br.uby;
    acc[2] += chem_blocks(r->br.g);
  }
  for (int k = 0; k < 3; ++k) {
    hf[k * (s->max_active + 1) + na] = acc[k];
    s->tot[k] = acc[k];
  }
  const size_t bb = a256(sizeof(BatchReq) * s->max_active);
  e = cudaMemcpyAsync(s->d_reqs, hb, sizeof(BatchReq) * na, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_first, h + bb, sizeof(int) * 3 * (s->max_active + 1), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->stage_ev[s->stage_k], s->stream);
  if (e != cudaSuccess) return scuda(e, "descriptor upload");
  s->stage_k ^= 1;
  s->dirty = false;
  return JANC_OK;
}

int retire(janc_server_s* s, Req* r) {
  const size_t un = (size_t)(s->nv + 1) * r->n;
  cudaError_t e = cudaEventRecord(r->ev_done, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, r->ev_done, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->host, r->br.S[0].base, sizeof(double) * un, cudaMemcpyDeviceToHost, s->copy_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->host + un, r->br.clock2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->copy_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->host + un + 2, r->br.status, sizeof(int), cudaMemcpyDeviceToHost, s->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev_copy, s->copy_stream);
  if (e != cudaSuccess) return scuda(e, "retire copy");
  r->state = R_COPYING;
  s->active_cells -= r->n;
  return JANC_OK;
}

}  // namespace

extern "C" {

int janc_server_set_cell_budget(janc_server_t s, long long cells, double max_skip_s) {
  if (!s || cells < 0 || !(max_skip_s >= 0.0)) return sfail(JANC_E_INVALID, "janc_server_set_cell_budget: bad argument");
  s->cell_budget = cells;
  s->max_skip_s = max_skip_s;
  return JANC_OK;
}

int janc_server_create(const janc_mechanism* m, int chemistry, size_t pool_bytes, void* pool, int max_active,
                       void* cuda_stream, janc_server_t* out) {
  if (!m || !out || max_active <= 0) return sfail(JANC_E_INVALID, "janc_server_create: bad argument");
  if (chemistry == JANC_CHEM_STRANG || chemistry == JANC_CHEM_EXPLICIT)
    return sfail(JANC_E_UNSUPPORTED, "janc_server_create: the server runs the Lie order");
  // validate the mechanism through the grid checks on a small probe descriptor
  janc_grid_desc probe;
  std::memset(&probe, 0, sizeof probe);
  probe.nx = probe.ny = 4;
  probe.dx = probe.dy = 1.0;
  probe.chemistry = chemistry;
  size_t dummy;
  int rc = janc_workspace_bytes(&probe, m, &dummy);
  if (rc) return rc;
  janc_server_s* s = new janc_server_s();
  s->ns = m->ns;
  s->nv = m->ns + 3;
  s->chem = chemistry ? 1 : 0;
  s->max_active = max_active;
  s->stream = (cudaStream_t)cuda_stream;
  MechDev hm;
  rc = build_mech_table(m, &hm);
  s->chem_fixed = fixed_structure(m);
  if (rc) { delete s; return rc; }
  cudaError_t e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  const size_t mech_b = a256(sizeof(MechDev));
  const size_t desc_b = a256(sizeof(BatchReq) * max_active) + a256(sizeof(int) * 3 * (max_active + 1));
  // the pool's head holds the mechanism table and the descriptor arrays
  if (e == cudaSuccess) {
    if (pool) {
      if ((uintptr_t)pool & 255u || pool_bytes <= mech_b + desc_b) {
        delete s;
        return sfail(JANC_E_INVALID, "janc_server_create: pool too small or not 256-byte aligned");
      }
      s->pool_base = (char*)pool;
    } else {
      e = cudaMalloc(&s->pool_base, pool_bytes);
      s->owns_pool = true;
    }
  }
  if (e == cudaSuccess) {
    s->dmech = (MechDev*)s->pool_base;
    s->d_reqs = (BatchReq*)(s->pool_base + mech_b);
    s->d_first = (int*)(s->pool_base + mech_b + a256(sizeof(BatchReq) * max_active));
    s->pool_base += mech_b + desc_b;
    s->pool.init(pool_bytes - mech_b - desc_b);
    for (int k = 0; k < 2; ++k) {
      if (e == cudaSuccess) e = cudaMallocHost(&s->h_stage[k], stage_bytes(max_active));
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->stage_ev[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(s->stage_ev[k], s->stream);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->dmech, &hm, sizeof(MechDev), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    janc_server_destroy(s);
    return scuda(e, "janc_server_create");
  }
  *out = s;
  return JANC_OK;
}

int janc_server_footprint(janc_server_t s, const janc_grid_desc* d, size_t* bytes) {
  if (!s || !d || !bytes) return sfail(JANC_E_INVALID, "null argument");
  size_t st, fx, gy, sm, tot;
  req_layout(d->nx, d->ny, s->nv, &st, &fx, &gy, &sm, &tot);
  *bytes = tot;
  return JANC_OK;
}

int janc_server_submit(janc_server_t s, const janc_grid_desc* d, const double* T, const double* p, const double* u,
                       const double* v, const double* Y, int n_steps, double dt, double cfl, int* id) {
  if (!s || !d || !T || !p || !u || !v || !Y || !id) return sfail(JANC_E_INVALID, "janc_server_submit: null argument");
  if (n_steps <= 0) return sfail(JANC_E_INVALID, "janc_server_submit: n_steps must be > 0");
  if ((dt > 0.0) == (cfl > 0.0)) return sfail(JANC_E_INVALID, "janc_server_submit: give exactly one of dt, cfl");
  if (d->nx < 3 || d->ny < 3) return sfail(JANC_E_INVALID, "janc_server_submit: grids need nx, ny >= 3");
  if (!(d->dx > 0.0) || !(d->dy > 0.0)) return sfail(JANC_E_INVALID, "janc_server_submit: dx, dy must be > 0");
  for (int k = 0; k < 4; ++k)
    if (d->bc[k] < 0 || d->bc[k] > 2) return sfail(JANC_E_INVALID, "janc_server_submit: unknown boundary kind");
  if ((d->bc[0] == JANC_BC_PERIODIC) != (d->bc[1] == JANC_BC_PERIODIC) ||
      (d->bc[2] == JANC_BC_PERIODIC) != (d->bc[3] == JANC_BC_PERIODIC))
    return sfail(JANC_E_INVALID, "janc_server_submit: periodic boundaries must pair");
  if (d->chemistry == JANC_CHEM_STRANG || d->chemistry == JANC_CHEM_EXPLICIT)
    return sfail(JANC_E_UNSUPPORTED, "janc_server_submit: the server runs the Lie order");
  if ((d->chemistry != 0) != (s->chem != 0))
    return sfail(JANC_E_INVALID, "janc_server_submit: chemistry flag differs from the server's");
  Req* r = new Req();
  r->id = (int)s->reqs.size();
  r->d = *d;
  r->n_steps = n_steps;
  r->dt = dt;
  r->cfl = cfl;
  r->n = (long long)d->nx * d->ny;
  size_t st, fx, gy, sm;
  req_layout(d->nx, d->ny, s->nv, &st, &fx, &gy, &sm, &r->footprint);
  if (r->footprint > s->pool.size) {
    delete r;
    return sfail(JANC_E_NOMEM, "janc_server_submit: request larger than the whole pool");
  }
  const size_t n = (size_t)r->n;
  r->host_doubles = (size_t)(4 + s->ns) * n + 4;  // (ns + 4) planes, then t, dt, status
  cudaError_t e = cudaMallocHost(&r->host, sizeof(double) * r->host_doubles);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_copy, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (r->host) cudaFreeHost(r->host);
    delete r;
    return scuda(e, "janc_server_submit");
  }
  std::memcpy(r->host, T, sizeof(double) * n);
  std::memcpy(r->host + n, p, sizeof(double) * n);
  std::memcpy(r->host + 2 * n, u, sizeof(double) * n);
  std::memcpy(r->host + 3 * n, v, sizeof(double) * n);
  std::memcpy(r->host + 4 * n, Y, sizeof(double) * s->ns * n);
  r->t_submit = now_s();
  s->reqs.push_back(r);
  s->queue.push_back(r->id);
  *id = r->id;
  return JANC_OK;
}

}  // extern "C"

namespace {

// One macro-step: retire finished copies, admit, then one batched step of
// every active request and the retirement of those that are done. *ran is
// false when nothing was active after admission.
int macro_step(janc_server_s* s, bool* ran) {
  *ran = false;
  reap(s);
  try_admit(s);
  if (s->active.empty()) return JANC_OK;
  if (s->dirty) {
    int rc = upload(s);
    if (rc) return rc;
  }
  const int na = (int)s->active.size();
  const int* f0 = s->d_first;
  const int* f1 = s->d_first + (s->max_active + 1);
  const int* f2 = s->d_first + 2 * (s->max_active + 1);
  cudaError_t e = launch_batch_prep(s->d_reqs, na, s->stream);
  for (int stage = 1; stage <= 3 && e == cudaSuccess; ++stage) {
    e = launch_face_flux_batch(s->nv, s->d_reqs, f0, na, s->tot[0], stage - 1, s->stream);
    if (e == cudaSuccess) e = launch_rk_update_batch(s->ns, stage, s->d_reqs, f1, na, s->tot[1], s->chem, s->stream);
  }
  if (e == cudaSuccess && s->chem)
    e = launch_chem_batch(s->ns, s->d_reqs, f2, na, s->tot[2], s->chem_fixed, s->stream);
  if (e != cudaSuccess) return scuda(e, "batched step");
  ++s->macro_steps;
  *ran = true;
  std::vector<int> still;
  for (int id : s->active) {
    Req* r = s->reqs[id];
    r->fresh = 0;
    if (++r->steps_done >= r->n_steps) {
      int rc = retire(s, r);
      if (rc) return rc;
      s->dirty = true;
    } else {
      still.push_back(id);
    }
  }
  s->active.swap(still);
  return JANC_OK;
}

void fill_info(janc_server_s* s, janc_server_info* info) {
  if (!info) return;
  std::memset(info, 0, sizeof *info);
  info->n_queued = (int)s->queue.size();
  info->n_active = (int)s->active.size();
  for (Req* r : s->reqs) {
    if (!r) continue;
    if (r->state == R_COPYING) ++info->n_copying;
    if (r->state == R_DONE || r->state == R_FAILED) ++info->n_done;
  }
  info->pool_used = s->pool.used;
  info->pool_bytes = s->pool.size;
  info->macro_steps = s->macro_steps;
}

// Newly finished (done or failed, not yet returned) requests into ids[0..cap).
void collect_finished(janc_server_s* s, int* ids, int cap, int* n) {
  reap(s);
  for (Req* r : s->reqs) {
    if (*n >= cap) break;
    if (!r || r->reported || (r->state != R_DONE && r->state != R_FAILED)) continue;
    r->reported = true;
    ids[(*n)++] = r->id;
  }
}

}  // namespace

extern "C" {

int janc_server_run(janc_server_t s, int macro_steps, janc_server_info* info) {
  if (!s || macro_steps < 0) return sfail(JANC_E_INVALID, "janc_server_run: bad argument");
  for (int k = 0; k < macro_steps; ++k) {
    bool ran = false;
    const int rc = macro_step(s, &ran);
    if (rc) return rc;
    if (!ran) break;
  }
  reap(s);
  fill_info(s, info);
  return JANC_OK;
}

int janc_server_run_until(janc_server_t s, int max_macro_steps, double max_wall_s, int* done_ids, int cap,
                          int* n_done, janc_server_info* info) {
  if (!s || max_macro_steps < 0 || !(max_wall_s >= 0.0) || !n_done || cap < 0 || (cap > 0 && !done_ids))
    return sfail(JANC_E_INVALID, "janc_server_run_until: bad argument");
  *n_done = 0;
  const double t0 = now_s();
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < 2 && e == cudaSuccess; ++q)
    if (!s->step_ev[q]) e = cudaEventCreateWithFlags(&s->step_ev[q], cudaEventDisableTiming);
  if (e != cudaSuccess) return scuda(e, "janc_server_run_until");
  collect_finished(s, done_ids, cap, n_done);
  for (int k = 0; k < max_macro_steps && *n_done == 0; ++k) {
    // at most two macro-steps in flight: wait for the end of the one before
    // the previous, so that finished copies are seen about one step late
    e = cudaEventSynchronize(s->step_ev[s->step_k]);
    if (e != cudaSuccess) return scuda(e, "janc_server_run_until");
    bool ran = false;
    const int rc = macro_step(s, &ran);
    if (rc) return rc;
    if (ran) {
      e = cudaEventRecord(s->step_ev[s->step_k], s->stream);
      if (e != cudaSuccess) return scuda(e, "janc_server_run_until");
      s->step_k ^= 1;
    }
    collect_finished(s, done_ids, cap, n_done);
    if (*n_done > 0) break;
    if (!ran) {
      // nothing active: wait for the copies of retired requests (they hold
      // the pool memory a queued request may be waiting for)
      e = cudaStreamSynchronize(s->copy_stream);
      if (e != cudaSuccess) return scuda(e, "janc_server_run_until");
      collect_finished(s, done_ids, cap, n_done);
      if (*n_done > 0 || s->queue.empty()) break;
    }
    if (now_s() - t0 >= max_wall_s) break;
  }
  fill_info(s, info);
  return JANC_OK;
}

int janc_server_poll(janc_server_t s, int id, janc_request_info* ri) {
  if (!s || !ri || id < 0 || id >= (int)s->reqs.size() || !s->reqs[id])
    return sfail(JANC_E_INVALID, "janc_server_poll: unknown request");
  reap(s);
  Req* r = s->reqs[id];
  std::memset(ri, 0, sizeof *ri);
  ri->state = (int)r->state;
  ri->steps_done = r->steps_done;
  ri->n_steps = r->n_steps;
  ri->latency_s = (r->state == R_DONE || r->state == R_FAILED || r->state == R_FETCHED) ? r->t_done - r->t_submit : -1.0;
  ri->queue_s = r->t_admit > 0.0 ? r->t_admit - r->t_submit : -1.0;
  if (r->state == R_DONE || r->state == R_FAILED) {
    const size_t un = (size_t)(s->nv + 1) * r->n;
    ri->t = r->host[un];
    ri->dt_last = r->host[un + 1];
    std::memcpy(&ri->status, r->host + un + 2, sizeof(int));
  }
  return JANC_OK;
}

int janc_server_fetch(janc_server_t s, int id, double* U, double* T) {
  if (!s || id < 0 || id >= (int)s->reqs.size() || !s->reqs[id])
    return sfail(JANC_E_INVALID, "janc_server_fetch: unknown request");
  reap(s);
  Req* r = s->reqs[id];
  if (r->state != R_DONE && r->state != R_FAILED) return sfail(JANC_E_INVALID, "janc_server_fetch: not finished");
  const size_t n = (size_t)r->n;
  if (U) std::memcpy(U, r->host, sizeof(double) * s->nv * n);
  if (T) std::memcpy(T, r->host + (size_t)s->nv * n, sizeof(double) * n);
  int st = 0;
  std::memcpy(&st, r->host + (size_t)(s->nv + 1) * n + 2, sizeof(int));
  cudaFreeHost(r->host);
  r->host = nullptr;
  cudaEventDestroy(r->ev_done);
  cudaEventDestroy(r->ev_copy);
  r->ev_done = r->ev_copy = nullptr;
  r->state = R_FETCHED;
  if (st) return sfail(JANC_E_DEVICE, "janc_server_fetch: device status word " + std::to_string(st));
  return JANC_OK;
}

void janc_server_destroy(janc_server_t s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->copy_stream) {
    cudaStreamSynchronize(s->copy_stream);
    cudaStreamDestroy(s->copy_stream);
  }
  for (Req* r : s->reqs) {
    if (!r) continue;
    if (r->host) cudaFreeHost(r->host);
    if (r->ev_done) cudaEventDestroy(r->ev_done);
    if (r->ev_copy) cudaEventDestroy(r->ev_copy);
    delete r;
  }
  for (int k = 0; k < 2; ++k) {
    if (s->h_stage[k]) cudaFreeHost(s->h_stage[k]);
    if (s->stage_ev[k]) cudaEventDestroy(s->stage_ev[k]);
    if (s->step_ev[k]) cudaEventDestroy(s->step_ev[k]);
  }
  if (s->owns_pool && s->dmech) cudaFree((void*)s->dmech);
  delete s;
}

}  // extern "C"
