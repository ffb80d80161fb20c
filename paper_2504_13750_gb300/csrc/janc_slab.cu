// x-slab domain decomposition (arXiv 2504.13750, Sec. 4.4, Fig. 3).
//
// The domain's nx columns are cut into slabs of whole columns. Each slab is
// an ordinary grid object whose x sides shared with a neighbour read their 3
// ghost columns from halo buffers (BC_HALO in the face-flux tile load); its
// y sides and the domain's outer x sides keep their physical boundaries, and
// a periodic x axis joins the last slab to the first. After every phase of a
// step that produces a state a neighbour's next face-flux launch reads (the
// outputs of RK stages 1 and 2, the step's final state, and a loaded state),
// the exchange copies each slab's 3 edge columns of all nv + 4 planes into
// the neighbours' halos and makes the phase's LF speeds (Eq. 4.11) the max
// over all slabs; the CFL dt follows from those. Every face then sees the
// same stencil values and the same alpha as in the undivided grid, every cell
// runs the same arithmetic, and a max is exact, so the slabs reproduce the
// undivided grid bit for bit.
//
// Two forms:
//  * janc_split_*: n slabs in one process, on the current device, one
//    stream. The slabs share one array of alpha slots, so the atomic max of
//    every update kernel is already the max over all slabs, and the halo
//    exchange is a pack kernel per slab that writes straight into its
//    neighbours' halo buffers.
//  * janc_slab_create: one slab per process (a rank), exchanging through a
//    caller callback (e.g. NCCL send/recv and an all-reduce max): the
//    library packs its edge columns into the caller's send buffers and its
//    alpha pair into the caller's 2-value buffer, calls back on the stream,
//    and reads the halos from the caller's receive buffers.
#include <cstring>
#include <string>
#include <vector>

#include "../../include/janc.h"
#include "janc_device.cuh"
#include "janc_grid.h"
#include "janc_internal.h"

using namespace janc;

namespace {

int sfail(int code, const std::string& m) { return fail_msg(code, m.c_str()); }

bool periodic_x(const janc_grid_desc* d) { return d->bc[0] == JANC_BC_PERIODIC; }

// The halo exchange of a stand-alone slab through the caller's callback.
struct CallbackExchange : Exchanger {
  janc_grid_s* g = nullptr;
  janc_slab_exchange x{};
  int after(int k, unsigned long long* slot) override {
    cudaStream_t st = g->stream;
    cudaError_t e = launch_halo_pack(g->nv + 4, StateView{g->S[k]}, g->gd, g->halo_side[0] ? x.send_lo : nullptr,
                                     g->halo_side[1] ? x.send_hi : nullptr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x.alpha2, slot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail_cuda_at(e, "slab exchange");
    const int rc = x.fn(x.user, (void*)st);
    if (rc != 0) return sfail(JANC_E_EXCHANGE, "slab exchange: the callback returned " + std::to_string(rc));
    e = cudaMemcpyAsync(slot, x.alpha2, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? JANC_OK : fail_cuda_at(e, "slab exchange");
  }
};

// The halo exchange among the slabs of one process: each slab's edge
// columns go straight into its neighbours' halo buffers (the alpha slots
// are shared, so their max needs nothing).
struct SplitExchange : Exchanger {
  std::vector<janc_grid_s*>* slabs = nullptr;
  int after(int k, unsigned long long*) override {
    const int n = (int)slabs->size();
    for (int i = 0; i < n; ++i) {
      janc_grid_s* g = (*slabs)[i];
      double* lo = g->halo_side[0] ? (*slabs)[(i + n - 1) % n]->halo[1] : nullptr;
      double* hi = g->halo_side[1] ? (*slabs)[(i + 1) % n]->halo[0] : nullptr;
      const cudaError_t e = launch_halo_pack(g->nv + 4, StateView{g->S[k]}, g->gd, lo, hi, g->stream);
      if (e != cudaSuccess) return fail_cuda_at(e, "split exchange");
    }
    return JANC_OK;
  }
};

int partition(int nx, int n, int k, int* x0, int* nxl) {
  if (n < 1 || k < 0 || k >= n) return sfail(JANC_E_INVALID, "slab index out of range");
  const int base = nx / n, rem = nx % n;
  if (base < 3) return sfail(JANC_E_INVALID, "every slab needs at least 3 columns (its neighbour's halo)");
  *nxl = base + (k < rem ? 1 : 0);
  *x0 = k * base + (k < rem ? k : rem);
  return JANC_OK;
}

// 2D copy of `rows` rows of `w` doubles between a whole-domain array
// (row pitch nx) and a slab array (row pitch w) starting at column x0.
cudaError_t copy_rows(double* dst, size_t dpitch, const double* src, size_t spitch, int w, size_t rows, cudaMemcpyKind kind,
                      cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  return cudaMemcpy2DAsync(dst, dpitch * sizeof(double), src, spitch * sizeof(double), (size_t)w * sizeof(double), rows,
                           kind, st);
}

}  // namespace

struct janc_split_s {
  janc_grid_desc d;
  int ns = 0, nv = 0;
  std::vector<janc_grid_s*> slabs;
  std::vector<int> x0, nxl;
  unsigned long long* alpha = nullptr;
  cudaStream_t stream = nullptr;
  SplitExchange ex;
};

extern "C" {

int janc_slab_partition(int nx, int n_slabs, int k, int* x0, int* nx_local) {
  if (!x0 || !nx_local) return sfail(JANC_E_INVALID, "null output");
  return partition(nx, n_slabs, k, x0, nx_local);
}

int janc_slab_halo_doubles(const janc_grid_desc* d, const janc_mechanism* m, size_t* count) {
  size_t ws = 0;
  const int rc = janc_workspace_bytes(d, m, &ws);  // validates d and m
  if (rc) return rc;
  if (!count) return sfail(JANC_E_INVALID, "null output");
  *count = (size_t)(m->ns + 7) * d->ny * 3;
  return JANC_OK;
}

int janc_slab_create(const janc_grid_desc* d, const janc_mechanism* m, int x0, int nx_local,
                     const janc_slab_exchange* x, void* workspace, size_t workspace_bytes, void* cuda_stream,
                     janc_grid_t* out) {
  size_t ws = 0;
  int rc = janc_workspace_bytes(d, m, &ws);
  if (rc) return rc;
  if (!x || !x->fn || !x->alpha2 || !out) return sfail(JANC_E_INVALID, "janc_slab_create: null argument");
  if (x0 < 0 || nx_local < 3 || x0 + nx_local > d->nx)
    return sfail(JANC_E_INVALID, "janc_slab_create: the slab must be >= 3 columns inside the domain");
  SlabOpts so;
  so.halo_lo = x0 > 0 || periodic_x(d);
  so.halo_hi = x0 + nx_local < d->nx || periodic_x(d);
  if ((so.halo_lo && (!x->send_lo || !x->recv_lo)) || (so.halo_hi && (!x->send_hi || !x->recv_hi)))
    return sfail(JANC_E_INVALID, "janc_slab_create: a shared side needs its send and receive buffers");
  so.halo_ext[0] = so.halo_lo ? x->recv_lo : nullptr;
  so.halo_ext[1] = so.halo_hi ? x->recv_hi : nullptr;
  janc_grid_desc local = *d;
  local.nx = nx_local;
  janc_grid_s* g = nullptr;
  rc = create_grid(&local, m, workspace, workspace_bytes, cuda_stream, &so, &g);
  if (rc) return rc;
  CallbackExchange* cx = new CallbackExchange();
  cx->g = g;
  cx->x = *x;
  g->ex = cx;
  *out = g;
  return JANC_OK;
}

void janc_split_destroy(janc_split_t s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (janc_grid_s* g : s->slabs) janc_destroy_grid(g);
  if (s->alpha) cudaFree(s->alpha);
  delete s;
}

int janc_split_create(const janc_grid_desc* d, const janc_mechanism* m, int n_slabs, void* cuda_stream,
                      janc_split_t* out) {
  size_t ws = 0;
  int rc = janc_workspace_bytes(d, m, &ws);
  if (rc) return rc;
  if (!out) return sfail(JANC_E_INVALID, "null output handle");
  if (n_slabs < 1) return sfail(JANC_E_INVALID, "n_slabs must be >= 1");
  janc_split_s* s = new janc_split_s();
  s->d = *d;
  s->ns = m->ns;
  s->nv = m->ns + 3;
  s->stream = (cudaStream_t)cuda_stream;
  for (int k = 0; k < n_slabs; ++k) {
    int a = 0, w = 0;
    rc = partition(d->nx, n_slabs, k, &a, &w);
    if (rc) {
      delete s;
      return rc;
    }
    s->x0.push_back(a);
    s->nxl.push_back(w);
  }
  const size_t abytes = sizeof(unsigned long long) * 2 * (SLOTS_PER_STEP * CHUNK + 1);
  if (cudaMalloc(&s->alpha, abytes) != cudaSuccess) {
    delete s;
    return sfail(JANC_E_NOMEM, "janc_split_create: cudaMalloc of the alpha slots failed");
  }
  cudaError_t e = cudaMemsetAsync(s->alpha, 0, abytes, s->stream);
  if (e != cudaSuccess) {
    janc_split_destroy(s);
    return fail_cuda_at(e, "janc_split_create");
  }
  for (int k = 0; k < n_slabs; ++k) {
    SlabOpts so;
    so.halo_lo = k > 0 || periodic_x(d);
    so.halo_hi = k < n_slabs - 1 || periodic_x(d);
    so.alpha = s->alpha;
    janc_grid_desc local = *d;
    local.nx = s->nxl[k];
    janc_grid_s* g = nullptr;
    rc = create_grid(&local, m, nullptr, 0, cuda_stream, &so, &g);
    if (rc) {
      janc_split_destroy(s);
      return rc;
    }
    s->slabs.push_back(g);
  }
  s->ex.slabs = &s->slabs;
  *out = s;
  return JANC_OK;
}

// Shared start of the two state loads: clear the alpha pair of the loaded
// state and every slab's status word.
static cudaError_t split_reset(janc_split_t s) {
  cudaError_t e = cudaMemsetAsync(s->alpha, 0, 2 * sizeof(unsigned long long), s->stream);
  for (janc_grid_s* g : s->slabs)
    if (e == cudaSuccess) e = cudaMemsetAsync(g->status, 0, sizeof(int), s->stream);
  return e;
}

int janc_split_set_state(janc_split_t s, const double* U, const double* T0, int where) {
  if (!s || !U) return sfail(JANC_E_INVALID, "null argument");
  if (where != JANC_HOST && where != JANC_DEVICE) return sfail(JANC_E_INVALID, "bad where");
  const cudaMemcpyKind kind = where == JANC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const int nx = s->d.nx, ny = s->d.ny;
  cudaError_t e = split_reset(s);
  for (size_t k = 0; k < s->slabs.size() && e == cudaSuccess; ++k) {
    janc_grid_s* g = s->slabs[k];
    const int w = s->nxl[k];
    e = copy_rows(g->S[0], w, U + s->x0[k], nx, w, (size_t)s->nv * ny, kind, s->stream);
    double* t0 = nullptr;
    if (e == cudaSuccess && T0) {  // warm start staged in S1's T plane
      t0 = g->S[1] + (size_t)s->nv * g->n;
      e = copy_rows(t0, w, T0 + s->x0[k], nx, w, (size_t)ny, kind, s->stream);
    }
    if (e == cudaSuccess)
      e = launch_set_conserved(s->ns, StateView{g->S[0]}, t0, g->gd, g->mech, s->alpha, g->status, s->stream);
  }
  if (e != cudaSuccess) return fail_cuda_at(e, "janc_split_set_state");
  const int rc = s->ex.after(0, s->alpha);
  if (rc) return rc;
  if (where == JANC_HOST) {
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return fail_cuda_at(e, "janc_split_set_state");
  }
  return JANC_OK;
}

int janc_split_set_state_primitive(janc_split_t s, const double* T, const double* p, const double* u, const double* v,
                                   const double* Y, int where) {
  if (!s || !T || !p || !u || !v || !Y) return sfail(JANC_E_INVALID, "null argument");
  if (where != JANC_HOST && where != JANC_DEVICE) return sfail(JANC_E_INVALID, "bad where");
  const cudaMemcpyKind kind = where == JANC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const int nx = s->d.nx, ny = s->d.ny;
  cudaError_t e = split_reset(s);
  for (size_t k = 0; k < s->slabs.size() && e == cudaSuccess; ++k) {
    janc_grid_s* g = s->slabs[k];
    const int w = s->nxl[k];
    const size_t n = (size_t)g->n;
    double* base = g->S[1];  // the fields staged in S1 (ns + 4 of its nv + 4 planes)
    const double* src[4] = {T, p, u, v};
    for (int f = 0; f < 4 && e == cudaSuccess; ++f)
      e = copy_rows(base + f * n, w, src[f] + s->x0[k], nx, w, (size_t)ny, kind, s->stream);
    if (e == cudaSuccess) e = copy_rows(base + 4 * n, w, Y + s->x0[k], nx, w, (size_t)s->ns * ny, kind, s->stream);
    if (e == cudaSuccess)
      e = launch_set_primitive(s->ns, StateView{g->S[0]}, base, base + n, base + 2 * n, base + 3 * n, base + 4 * n,
                               g->gd, g->mech, s->alpha, g->status, s->stream);
  }
  if (e != cudaSuccess) return fail_cuda_at(e, "janc_split_set_state_primitive");
  const int rc = s->ex.after(0, s->alpha);
  if (rc) return rc;
  if (where == JANC_HOST) {
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return fail_cuda_at(e, "janc_split_set_state_primitive");
  }
  return JANC_OK;
}

int janc_split_step(janc_split_t s, int n_steps, double dt, double cfl, double* t_out, double* dt_last_out) {
  if (!s) return sfail(JANC_E_INVALID, "null split");
  return step_grids(s->slabs.data(), (int)s->slabs.size(), &s->ex, n_steps, dt, cfl, t_out, dt_last_out);
}

int janc_split_get_state(janc_split_t s, double* U, double* T, int where) {
  if (!s) return sfail(JANC_E_INVALID, "null split");
  if (where != JANC_HOST && where != JANC_DEVICE) return sfail(JANC_E_INVALID, "bad where");
  const cudaMemcpyKind kind = where == JANC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const int nx = s->d.nx, ny = s->d.ny;
  cudaError_t e = cudaSuccess;
  std::vector<int> st(s->slabs.size(), 0);
  for (size_t k = 0; k < s->slabs.size() && e == cudaSuccess; ++k) {
    janc_grid_s* g = s->slabs[k];
    const int w = s->nxl[k];
    if (U) e = copy_rows(U + s->x0[k], nx, g->S[0], w, w, (size_t)s->nv * ny, kind, s->stream);
    if (e == cudaSuccess && T)
      e = copy_rows(T + s->x0[k], nx, g->S[0] + (size_t)s->nv * g->n, w, w, (size_t)ny, kind, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st[k], g->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return fail_cuda_at(e, "janc_split_get_state");
  int any = 0;
  for (int v : st) any |= v;
  if (any) return sfail(JANC_E_DEVICE, "device status word " + std::to_string(any));
  return JANC_OK;
}

int janc_split_status(janc_split_t s, janc_status_info* info) {
  if (!s || !info) return sfail(JANC_E_INVALID, "null argument");
  janc_status_info first{};
  int any = 0;
  for (size_t k = 0; k < s->slabs.size(); ++k) {
    janc_status_info one{};
    const int rc = janc_status(s->slabs[k], &one);
    if (rc) return rc;
    any |= one.status;
    if (k == 0) first = one;
  }
  *info = first;
  info->status = any;
  return JANC_OK;
}

int janc_split_slab(janc_split_t s, int k, janc_grid_t* slab) {
  if (!s || !slab || k < 0 || k >= (int)s->slabs.size()) return sfail(JANC_E_INVALID, "bad argument");
  *slab = s->slabs[k];
  return JANC_OK;
}

}  // extern "C"
