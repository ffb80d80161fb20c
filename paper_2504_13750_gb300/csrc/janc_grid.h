// The grid object behind janc_grid_t, shared by the translation units that
// drive grids directly: janc_capi.cu (single grids, the step loop, the
// adjoint) and janc_slab.cu (the x-slab decomposition of Sec. 4.4).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/janc.h"
#include "janc_device.cuh"
#include "janc_internal.h"

namespace janc {

constexpr int CHUNK = 256;  // steps per alpha-slot chunk
constexpr int SLOTS_PER_STEP = 5;

// Pieces of one grid's workspace, each 256-byte aligned: 3 state buffers,
// the two face-flux arrays, the alpha slots of a chunk of steps, the clock,
// the status word, the mechanism table and, for a slab whose halo buffers
// live in its own workspace, two halos of (nv + 4) x ny x 3 doubles.
struct Layout {
  size_t state, fx, gy, alpha, clock, status, mech, halo, total;
};
Layout layout_of(int nx, int ny, int nv, bool halos);

// Exchange of an x-slab decomposition (Sec. 4.4, Fig. 3). The step loop runs
// it after every phase whose output state a neighbour's next face-flux launch
// reads (and the state loads run it once): k is that state's buffer (0, 1, 2)
// and slot its pair of LF speeds. It fills the neighbours' halo buffers with
// the slab's 3 edge columns and makes slot hold the max over all slabs, all
// in stream order. Returns a JANC_* code (the error text already set).
struct Exchanger {
  virtual ~Exchanger() = default;
  virtual int after(int k, unsigned long long* slot) = 0;
};

}  // namespace janc

struct janc_grid_s {
  janc_grid_desc d;
  int ns, nv, nr;
  long long n;
  janc::GridDev gd;
  janc::Layout L;
  char* ws;
  bool owns_ws;
  cudaStream_t stream;
  double* S[3];
  double* Fx;
  double* Gy;
  unsigned long long* alpha;
  double* clock2;
  int* status;
  janc::MechDev* mech;
  int steps_done;
  // x-slab decomposition (Sec. 4.4): the x sides whose ghost columns come
  // from a halo buffer (gd.bc = BC_HALO there), the halo buffers, and the
  // exchange a stand-alone slab runs after its state-producing phases (null
  // for a plain grid and for the slabs of a janc_split, whose exchange the
  // split object runs). A split's slabs share one array of alpha slots.
  bool halo_side[2] = {false, false};
  double* halo[2] = {nullptr, nullptr};
  janc::Exchanger* ex = nullptr;  // owned by the grid
  bool alpha_shared = false;
  // trajectory of the last janc_adjoint_forward, for janc_adjoint_reverse
  int adj_mode = 0;  // JANC_ADJ_RECOMPUTE or JANC_ADJ_STORE_FACES (janc_set_adjoint_mode)
  struct AdjPending {
    bool valid = false;
    int n_steps = 0, ckpt_every = 1, loss_kind = 0, mode = 0;
    double dt = 0.0;
    char* ws = nullptr;
    bool own = false;
  } adj;
  // per-kernel event timing (janc_profile)
  bool prof_on = false;
  struct Mark { cudaEvent_t a, b; int cls; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
};

namespace janc {

// Options of a grid that is one slab of an x-slab decomposition.
struct SlabOpts {
  bool halo_lo = false, halo_hi = false;   // x sides shared with a neighbouring slab
  unsigned long long* alpha = nullptr;     // shared alpha slots (a split), else the workspace's
  double* halo_ext[2] = {nullptr, nullptr};  // caller halo buffers, else the workspace's
};

// Creates a grid; with `so` a slab (its desc's x boundaries must be those of
// the whole domain: the shared sides become BC_HALO). Returns a JANC_* code.
int create_grid(const janc_grid_desc* d, const janc_mechanism* m, void* workspace, size_t workspace_bytes,
                void* cuda_stream, const SlabOpts* so, janc_grid_s** out);

// n_steps steps of advance_one_step (Sec. 4.3) on ng grids in lockstep: the
// slabs of one domain, or a single grid (ng = 1). Every phase is launched on
// each grid in turn; `ex` (may be null) runs after each state-producing
// phase. All grids share gs[0]'s stream and, when ng > 1, its alpha slots.
int step_grids(janc_grid_s* const* gs, int ng, Exchanger* ex, int n_steps, double dt, double cfl, double* t_out,
               double* dt_last_out);

// Fails with a CUDA error text / a message (sets janc_last_error).
int fail_cuda_at(cudaError_t e, const char* where);
int fail_msg(int code, const char* msg);

}  // namespace janc
