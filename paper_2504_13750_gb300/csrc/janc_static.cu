// janc_rhs_static: the right-hand side of janc_rhs for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or arena (where a raw allocation would bypass the
// pool's accounting and can fail once the pool has reserved the device),
// real-time or embedded loops that forbid allocation after start-up, and
// plug-ins that only receive device buffers from their host. This entry point
// needs no workspace from them: its scratch (one state buffer with the
// auxiliary planes, the x- and y-face flux arrays, the LF-speed slot, the
// status word and the mechanism table) lives in the file-scope device array
// below, of fixed size JANC_STATIC_SCRATCH_BYTES, which every GPU that loads
// this library holds until the process exits.
//
// Host code must not hand the array's name to a kernel: in host code that
// name is a host-side stand-in, not a device address. The device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device; that first call should
// therefore come before any stream capture. The address is kept until the
// process exits: a device reset (which destroys the primary context) leaves
// it stale, and this entry point must not be used on that device again. All
// calls share the one array
// and it keeps the previous call's contents: the LF-speed slot and the status
// word are cleared on every call, everything else is overwritten before it is
// read. Calls that overlap on the GPU (different streams or threads without
// ordering) race on the array and must be serialised by the caller.
#include <mutex>
#include <string>

#include "../../include/janc.h"
#include "janc_device.cuh"
#include "janc_internal.h"

using namespace janc;

static __device__ __align__(256) unsigned char g_static_scratch[JANC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex s_mu;
unsigned char* s_addr[kMaxDevices] = {};

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

int fail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

// Device address of the scratch array on the current device (looked up once).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(JANC_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(JANC_E_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lk(s_mu);
  if (!s_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(JANC_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    s_addr[dev] = (unsigned char*)p;
  }
  *out = s_addr[dev];
  return JANC_OK;
}

}  // namespace

extern "C" {

int janc_rhs_static(const janc_grid_desc* d, const janc_mechanism* m, const double* U, const double* T,
                    double* L, double* alpha, void* cuda_stream) {
  if (!d || !m || !U || !T || !L) return fail(JANC_E_INVALID, "janc_rhs_static: null argument");
  // Validate through the regular descriptor check (it allocates nothing).
  size_t ws = 0;
  int rc = janc_workspace_bytes(d, m, &ws);
  if (rc) return fail(rc, std::string("janc_rhs_static: ") + janc_last_error());
  const int nv = m->ns + 3;
  const long long n = (long long)d->nx * d->ny;
  const size_t state = a256(sizeof(double) * (size_t)(nv + 4) * n);
  const size_t fx = a256(sizeof(double) * (size_t)nv * d->ny * (d->nx + 1));
  const size_t gy = a256(sizeof(double) * (size_t)nv * (d->ny + 1) * d->nx);
  const size_t slots = 256, mech = a256(sizeof(MechDev));
  const size_t need = state + fx + gy + slots + mech;
  if (need > (size_t)JANC_STATIC_SCRATCH_BYTES)
    return fail(JANC_E_INVALID, "janc_rhs_static: grid needs " + std::to_string(need) +
                                    " bytes of scratch, more than JANC_STATIC_SCRATCH_BYTES = " +
                                    std::to_string((size_t)JANC_STATIC_SCRATCH_BYTES));
  // Mechanism table in kernel form (same conversion as janc_create_grid).
  MechDev hm;
  rc = build_mech_table(m, &hm);
  if (rc) return fail(rc, std::string("janc_rhs_static: ") + janc_last_error());
  unsigned char* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* S = (double*)base;
  double* Fx = (double*)(base + state);
  double* Gy = (double*)(base + state + fx);
  unsigned long long* a = (unsigned long long*)(base + state + fx + gy);
  int* status = (int*)(a + 2);
  MechDev* dm = (MechDev*)(base + state + fx + gy + slots);

  GridDev g = {};
  g.nx = d->nx;
  g.ny = d->ny;
  g.n = n;
  g.dx = d->dx;
  g.dy = d->dy;
  g.rdx = 1.0 / d->dx;
  g.rdy = 1.0 / d->dy;
  for (int s = 0; s < 4; ++s) g.bc[s] = d->bc[s];
  g.eps4 = 4.0 * (d->weno_eps > 0.0 ? d->weno_eps : 1e-6);
  g.newton_tol = d->newton_tol > 0.0 ? d->newton_tol : 1e-12;
  g.newton_maxit = d->newton_maxit > 0 ? d->newton_maxit : 50;

  cudaError_t e = cudaMemcpyAsync(dm, &hm, sizeof(MechDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, 2 * sizeof(unsigned long long) + sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S, U, sizeof(double) * (size_t)nv * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_set_conserved(m->ns, StateView{S}, T, g, dm, a, status, st);
  if (e == cudaSuccess) e = launch_face_flux(nv, StateView{S}, a, Fx, Gy, g, st);
  if (e == cudaSuccess) e = launch_rhs_L(nv, Fx, Gy, L, g, st);
  if (e == cudaSuccess && alpha) e = cudaMemcpyAsync(alpha, a, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  int hst = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  // The host table and status word are used by the copies above: wait.
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(JANC_E_CUDA, std::string("janc_rhs_static: ") + cudaGetErrorString(e));
  if (hst) return fail(JANC_E_DEVICE, "janc_rhs_static: device status word " + std::to_string(hst));
  return JANC_OK;
}

}  // extern "C"
