/*
 * janc.h - C ABI of the GB300 (sm_103a) reacting-flow step.
 *
 * The library advances the 2D reactive Euler equations (arXiv 2504.13750,
 * Sec. 4.1, Eq. 4.1) on a uniform Cartesian grid with the scheme of Sec. 4.2:
 * global Lax-Friedrichs flux splitting (Eq. 4.11) with WENO5 reconstruction
 * and 3 ghost layers, 3rd-order TVD Runge-Kutta for the flux terms, Newton
 * recovery of T from the energy, and the first-order point-implicit chemistry
 * update (Eq. 4.12-4.13) with Arrhenius and equilibrium rates (Eq. 4.6-4.9).
 * One call of janc_step runs advance_one_step of Sec. 4.3 n times.
 *
 * Conventions shared by every entry point:
 *  - Return value: 0 on success, a negative JANC_E_* code on failure. Nothing
 *    throws across the ABI; janc_last_error() gives a text for the calling
 *    thread's most recent failure.
 *  - Arithmetic is IEEE FP64 throughout.
 *  - State layout: structure of arrays, U[nv][ny][nx] with x fastest,
 *    nv = ns + 3 planes in the order rho, rho u, rho v, E, rho Y_1 ..
 *    rho Y_{ns-1} (SI units: kg/m^3, kg/(m^2 s), J/m^3); T[ny][nx] in K.
 *    The ns-th species is not carried (Y_ns = 1 - sum of the others).
 *  - Pointer arguments marked "host or device" are read or written according
 *    to the `where` argument (JANC_HOST / JANC_DEVICE). Host copies are
 *    synchronous with respect to the caller; device pointers are used in
 *    order on the grid's stream. All buffers passed in stay owned by the
 *    caller and may be released once the call returns (host) or once the
 *    stream has passed the call (device).
 *  - Work is enqueued on the CUDA stream given at creation (NULL = legacy
 *    default stream). janc_step is asynchronous; device-side failures are
 *    recorded in a status word that janc_status / janc_get_state report.
 *  - A grid handle must not be used from two host threads at once.
 */
#ifndef JANC_H_
#define JANC_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define JANC_OK 0
#define JANC_E_INVALID (-1)     /* bad argument (null pointer, size, mode) */
#define JANC_E_UNSUPPORTED (-2) /* valid but not built (e.g. species count) */
#define JANC_E_CUDA (-3)        /* a CUDA runtime call failed */
#define JANC_E_NOMEM (-4)       /* device allocation failed or workspace too small */
#define JANC_E_DEVICE (-5)      /* the device status word reports a failure */
#define JANC_E_EXCHANGE (-6)    /* an x-slab exchange callback reported a failure */

/* Boundary kinds (user boundary hooks of Sec. 4.3 reduced to three forms). */
#define JANC_BC_WALL 0      /* slip wall: mirror ghosts, wall-normal momentum negated */
#define JANC_BC_ZEROGRAD 1  /* non-reflecting: zero-gradient copy of the edge cell */
#define JANC_BC_PERIODIC 2  /* periodic wrap (both sides of an axis must agree) */

#define JANC_HOST 0
#define JANC_DEVICE 1

/* Device status bits (OR-ed by the kernels, read by janc_status). */
#define JANC_ST_NONFINITE 1      /* a NaN or Inf appeared in the state */
#define JANC_ST_NONPOSITIVE 2    /* rho, T or p <= 0 */
#define JANC_ST_NEWTON_FAIL 4    /* T recovery did not converge in newton_maxit */
#define JANC_ST_SINGULAR 8       /* zero pivot in the point-implicit solve */

typedef struct janc_grid_s* janc_grid_t;

/* Operator splitting of one step (Sec. 4.3). advance_one_step as written
 * there runs the flux RK3 over dt and then the point-implicit chemistry
 * (Eq. 4.12-4.13) over dt (JANC_CHEM_LIE); the text of the same section names
 * Strang splitting, chemistry over dt/2, flux over dt, chemistry over dt/2
 * (JANC_CHEM_STRANG). dt is the step's, from the CFL of its starting state. */
#define JANC_CHEM_OFF 0
#define JANC_CHEM_LIE 1
#define JANC_CHEM_STRANG 2
/* No splitting: the production rates of the mechanism are a source term of
 * the semi-discrete equation, advanced with the fluxes by the same TVD-RK3
 * (the user source_terms path of Sec. 4.3, for a weakly stiff global
 * reaction); advance_source_term is not run. */
#define JANC_CHEM_EXPLICIT 3

/* Grid description.
 * nx, ny >= 1 cells; dx, dy > 0 m; bc = {left, right, bottom, top};
 * chemistry = JANC_CHEM_* (above): JANC_CHEM_OFF runs the flux terms only,
 * the explicit variant of advance_one_step (Sec. 4.3). The server and AMR
 * take JANC_CHEM_OFF or JANC_CHEM_LIE only, the adjoint also
 * JANC_CHEM_EXPLICIT (otherwise JANC_E_UNSUPPORTED);
 * weno_eps = epsilon of the WENO5-JS weights (1e-6 if <= 0);
 * newton_tol / newton_maxit = stop when |dT| <= tol * T (1e-12 / 50 if <= 0). */
typedef struct {
  int nx, ny;
  double dx, dy;
  int bc[4];
  int chemistry;
  double weno_eps;
  double newton_tol;
  int newton_maxit;
} janc_grid_desc;

/* Mechanism and thermodynamic data (Eq. 4.3-4.9), all SI, copied at creation.
 * ns species (the last one is not carried in U), nr reactions.
 * M[ns] kg/mol; nasa[ns*7] NASA-7 coefficients a_0..a_6 (single range);
 * A[nr], b[nr], Ea[nr]: k_f = A T^b exp(-Ea / (Ru T)), Ea in J/mol;
 * nuf[nr*ns], nub[nr*ns]: reactant / product stoichiometric coefficients;
 * tb[nr] = 1 when reaction i carries the third-body factor sum_j eff[i*ns+j] X_j
 * (1 otherwise). Supported: ns in {1, 3, 9}, nr <= 32, at most 3 distinct
 * species on each side of a reaction, coefficients 0..3. */
typedef struct {
  int ns, nr;
  const double* M;
  const double* nasa;
  const double* A;
  const double* b;
  const double* Ea;
  const int* nuf;
  const int* nub;
  const int* tb;
  const double* eff;
} janc_mechanism;

typedef struct {
  int status;          /* OR of JANC_ST_* since creation or the last reset */
  int steps_done;      /* steps completed since creation */
  double t;            /* simulated time since creation, s */
  double dt_last;      /* dt of the most recent step, s */
  double alpha[2];     /* LF speeds (Eq. 4.11) of the current state, m/s */
} janc_status_info;

/* Bytes of device workspace janc_create_grid needs for this grid. */
int janc_workspace_bytes(const janc_grid_desc* d, const janc_mechanism* m, size_t* bytes);

/* Create a grid. `workspace` is a device allocation of at least
 * janc_workspace_bytes(d, m) bytes, 256-byte aligned, owned by the caller and
 * kept alive until janc_destroy_grid; pass NULL to let the library allocate
 * (and free) its own. `cuda_stream` is a cudaStream_t (NULL = default). The
 * state is undefined until janc_set_state or janc_set_state_primitive. */
int janc_create_grid(const janc_grid_desc* d, const janc_mechanism* m, void* workspace, size_t workspace_bytes,
                     void* cuda_stream, janc_grid_t* out);

/* Load the conserved state U[nv][ny][nx] (host or device). With T0 non-NULL
 * it is the warm start of the Newton T recovery (end of Sec. 4.2); with NULL
 * the recovery starts from 1000 K. Resets the status word. */
int janc_set_state(janc_grid_t g, const double* U, const double* T0, int where);

/* Load the state from primitive fields T, p, u, v [ny][nx] and mass
 * fractions Y[ns][ny][nx] of all ns species (host or device), through the
 * equation of state of Eq. 4.2. Resets the status word. */
int janc_set_state_primitive(janc_grid_t g, const double* T, const double* p, const double* u, const double* v,
                             const double* Y, int where);

/* Advance n_steps steps of advance_one_step (Sec. 4.3). Exactly one of
 * dt > 0 (fixed step) or cfl > 0 must be given; with cfl each step uses
 * dt = cfl * min(dx, dy) / max(alpha_x, alpha_y) of its starting state,
 * computed on the device. t_out / dt_last_out (host, may be NULL) receive the
 * simulated time of the call and the last dt; giving either synchronises the
 * stream. */
int janc_step(janc_grid_t g, int n_steps, double dt, double cfl, double* t_out, double* dt_last_out);

/* Copy out U[nv][ny][nx] and T[ny][nx] (either may be NULL), host or device.
 * Host copies synchronise the stream. Returns JANC_E_DEVICE (after copying)
 * when the status word is non-zero. */
int janc_get_state(janc_grid_t g, double* U, double* T, int where);

/* Right-hand side of the current state, for checking: the split WENO5 face
 * fluxes Fx[nv][ny][nx+1] (x-face i-1/2 at index i) and Gy[nv][ny+1][nx]
 * (y-face j-1/2 at index j) of Eq. 4.10-4.11, L = -(dF/dx + dG/dy)
 * [nv][ny][nx], and alpha[2] (any may be NULL), host or device. */
int janc_rhs(janc_grid_t g, double* Fx, double* Gy, double* L, double* alpha, int where);

/* Per-kernel timing. While enabled, janc_step brackets every kernel launch
 * with CUDA events on the grid's stream. janc_profile_read synchronises,
 * returns per kernel class (0 = face fluxes, 1 = RK stage update, 2 =
 * chemistry) the summed device time in ms and the launch count, and clears
 * the counters. Arrays have 3 entries. */
int janc_profile(janc_grid_t g, int enable);
int janc_profile_read(janc_grid_t g, double* ms, long long* launches);

/* advance_source_term of Sec. 4.3 alone, n_steps times over dt: the
 * point-implicit chemistry (Eq. 4.12-4.13) and the Newton T of every cell,
 * no flux terms (so every cell is an independent constant-volume reactor, the
 * 0-D ignition case of Sec. 5.1(2)). The simulated clock is not advanced.
 * Asynchronous on the grid's stream; JANC_E_INVALID without chemistry. */
int janc_source_step(janc_grid_t g, int n_steps, double dt);

/* Read the status word and counters (synchronises the stream). */
int janc_status(janc_grid_t g, janc_status_info* s);

/* Text of the calling thread's most recent error ("" if none). */
const char* janc_last_error(void);

/* Release the grid (waits for its stream). */
void janc_destroy_grid(janc_grid_t g);

/* FP64 pipe throughput probe: runs n_iter dependent-chain DFMA loops on
 * every SM and reports the DFMA lane operations per second it sustained
 * (a measured FP64 peak for roofline fractions). Synchronous. */
int janc_fp64_peak(void* cuda_stream, int n_iter, double* dfma_per_s);

/* Accuracy check of the library's FP64 reciprocal (MUFU seed refined by one
 * third-order iteration step) against IEEE division on the device, over the n host
 * values x (positive normal doubles): max_ulp receives the largest distance
 * in units in the last place. Synchronous; allocates scratch. */
int janc_selfcheck_rcp(const double* x, int n, long long* max_ulp);

/* Accuracy check of the library's FP64 exponential (P. T. P. Tang's
 * table-driven method, used by the chemistry kernel) against CUDA's exp on
 * the device, over the n host values x: max_ulp receives the largest
 * distance in units in the last place. Synchronous; allocates scratch. */
int janc_selfcheck_exp(const double* x, int n, long long* max_ulp);

/* ------------------------------------------------------------------------
 * Discrete adjoint. The gradient of a loss of a fixed-dt trajectory of
 * advance_one_step (Sec. 4.3) with respect to its initial conserved state,
 * by reverse-mode differentiation of every operation the forward kernels do
 * (flux splitting and WENO5, the global LF speeds through their arg-max
 * cells, Newton T recovery by its implicit derivative, TVD-RK3, point-
 * implicit chemistry), with checkpoint-and-recompute: the state is stored
 * every ckpt_every steps and each segment is recomputed (bit for bit) during
 * the reverse sweep. Memory: ceil(n/ckpt_every) + 4 ckpt_every + 1 states of
 * (nv + 4) planes (twice the 4 ckpt_every + 1 when there is more than one
 * segment: the next segment is recomputed on a second stream while the
 * current one is reversed), 7 cotangent arrays and the face-contribution
 * buffers; see janc_adjoint_workspace_bytes. The continuous adjoint of Sec. 6.1 (Eq. 6.5)
 * is replaced by this exact discrete one.
 * ---------------------------------------------------------------------- */
#define JANC_LOSS_ENDWALL_P 0  /* L = sum_n dt * mean_j p(nx-1, j) of U^{n+1} */
#define JANC_LOSS_SEEDED 1     /* L = <seed, U^N> (seed: nv planes) */

/* How the reverse sweep gets the linearisation of the forward operators.
 * JANC_ADJ_RECOMPUTE (the default): the face pass of each RHS
 * vector-Jacobian product recomputes the derivatives of the WENO5
 * reconstructions (Eq. 4.10) from the stage state, and the chemistry VJP
 * forms the rates, J'' and the LU factors of Eq. 4.13 again.
 * JANC_ADJ_STORE_FACES: the steps that fill a segment store (the forward's
 * last two segments, every recomputed segment) run a face-flux kernel that also
 * stores, per face, variable and split sign, the four partials of the
 * reconstruction with respect to its window's differences, and (with
 * JANC_CHEM_LIE) a chemistry kernel that also keeps, per cell, the rate
 * constants k_f and k_b, the LU factors, the pivots and the solution, or
 * (with JANC_CHEM_EXPLICIT) stage updates that keep k_f and k_b of the
 * explicit source at each stage input; the reverse face pass then only
 * weights the partials by the cotangent, and the chemistry or source VJP
 * starts from the kept values. That moves most of the reverse work into the
 * recompute, which runs on its own stream beside the sweep, at a memory cost
 * per step of a segment store of 3 x 8 nv ((nx+1) ny + (ny+1) nx) doubles
 * (faces) plus (2 nr + (ns-1)^2 + ns) nx ny doubles (JANC_CHEM_LIE) or
 * 6 nr nx ny doubles (JANC_CHEM_EXPLICIT), ckpt_every steps per store, two
 * stores when there is more than one segment. The face fluxes,
 * the trajectory and the loss are the same bit for bit in both modes; the
 * gradients agree to rounding. The mode is read when
 * janc_adjoint_workspace_bytes and janc_adjoint_forward run; a pending
 * forward keeps the mode it started with. JANC_E_INVALID for another mode.
 * The paper has no counterpart: it is a memory-for-work trade of this
 * implementation of the discrete adjoint. */
#define JANC_ADJ_RECOMPUTE 0
#define JANC_ADJ_STORE_FACES 1
int janc_set_adjoint_mode(janc_grid_t g, int mode);

/* Device bytes janc_step_adjoint needs as workspace: checkpoints every
 * ckpt_every steps, the stage states of one segment of ckpt_every steps (two
 * such stores when n_steps > ckpt_every), cotangent and face buffers. The
 * forward writes the last two segments' stages directly (one per store), so
 * the reverse recomputes every segment but those; with ckpt_every >= n_steps the
 * whole trajectory is kept and nothing is recomputed (about
 * (4 n_steps + 2) (nv + 4) nx ny doubles, plus the face derivatives and
 * chemistry factors of n_steps steps in mode JANC_ADJ_STORE_FACES). */
int janc_adjoint_workspace_bytes(janc_grid_t g, int n_steps, int ckpt_every, size_t* bytes);

/* From the grid's current state U^0 (set beforehand), run n_steps fixed-dt
 * steps, computing the loss (*loss_out, host, may be NULL) and, when dL_dU0
 * is not NULL, the cotangent dL/dU^0 [nv][ny][nx] (host or device, `where`).
 * seed: nv planes for JANC_LOSS_SEEDED, else ignored (host or device).
 * workspace: device memory of janc_adjoint_workspace_bytes (256-byte
 * aligned), or NULL to let the call allocate and free it. On return the
 * grid holds U^N. Synchronous. */
int janc_step_adjoint(janc_grid_t g, int n_steps, double dt, int ckpt_every, int loss_kind, const double* seed,
                      double* dL_dU0, double* loss_out, void* workspace, size_t workspace_bytes, int where);

/* The two halves of janc_step_adjoint, for losses that need U^N first (the
 * cotangent dL/dU^N of a nonlinear loss, e.g. an autograd graph on U^N).
 * janc_adjoint_forward runs n_steps fixed-dt steps from the grid's state with
 * checkpoints in `workspace` (janc_adjoint_workspace_bytes; null: an internal
 * allocation) and leaves U^N in the grid. With JANC_LOSS_ENDWALL_P it returns
 * that loss in *loss_out (may be null); with JANC_LOSS_SEEDED nothing is
 * accumulated. A later forward on the same grid replaces the pending one. */
int janc_adjoint_forward(janc_grid_t g, int n_steps, double dt, int ckpt_every, int loss_kind, double* loss_out,
                         void* workspace, size_t workspace_bytes);
/* janc_adjoint_reverse: dL/dU^0 of the pending forward, for the cotangent
 * seed = dL/dU^N ([nv][ny][nx]; null: zero) plus the end-wall loss's own
 * cotangents when the forward used JANC_LOSS_ENDWALL_P. The workspace must be
 * the forward's and untouched; the grid's own state may have changed since.
 * Synchronous; ends the pending forward (and frees an internal workspace).
 * JANC_E_INVALID without a pending forward. */
int janc_adjoint_reverse(janc_grid_t g, const double* seed, double* dL_dU0, int where);

/* Vector-Jacobian product of the right-hand side L(U) (Eq. 4.10-4.11 with
 * WENO5, the ghost layers and the global LF speeds) at the grid's current
 * state: nu = (dL/dU)^T mu, both [nv][ny][nx], host or device. workspace:
 * device memory for 2 nv planes plus 10 nv values per x- and y-face, each
 * piece rounded up to 256 bytes, plus 256 bytes and 24 bytes per 32 x 8
 * block of cells rounded up to 256 (NULL: allocated here); a smaller
 * workspace returns JANC_E_NOMEM. Synchronous. */
int janc_rhs_vjp(janc_grid_t g, const double* mu, double* nu, void* workspace, size_t workspace_bytes, int where);

/* dL/dT [ny][nx] of the primitive initialisation of Eq. 4.2 at fixed p, u,
 * v, Y (device pointers, the layout of janc_set_state_primitive), given
 * dL/dU [nv][ny][nx] (device). Synchronous. */
int janc_primitive_T_vjp(janc_grid_t g, const double* T, const double* p, const double* u, const double* v,
                         const double* Y, const double* dL_dU, double* dL_dT);

/* ------------------------------------------------------------------------
 * Continuous-batching server: many independent solves of one mechanism on
 * one GPU. Each request is a grid (janc_grid_desc) with primitive initial
 * fields, a step count and dt or cfl; it advances by advance_one_step
 * (Sec. 4.3) exactly as janc_step would run it alone. Requests are queued,
 * admitted in arrival order (skipping ahead over ones that do not fit) when
 * their device footprint fits the free part of the server's HBM pool and one
 * of max_active slots is free, then advanced together: every janc_server_run
 * macro-step moves each active request one step with one batched persistent
 * kernel per phase over all of them. A finished request leaves the active set
 * at once; its result goes to pinned host memory on a second stream and its
 * pool memory is reused when that copy is done. Single host thread.
 * ---------------------------------------------------------------------- */
typedef struct janc_server_s* janc_server_t;

#define JANC_REQ_QUEUED 0
#define JANC_REQ_ACTIVE 1
#define JANC_REQ_COPYING 2
#define JANC_REQ_DONE 3
#define JANC_REQ_FAILED 4
#define JANC_REQ_FETCHED 5

typedef struct {
  int n_queued, n_active, n_copying, n_done;
  size_t pool_used, pool_bytes;
  long long macro_steps;
} janc_server_info;

typedef struct {
  int state;          /* JANC_REQ_* */
  int steps_done, n_steps;
  int status;         /* device status word of the finished request */
  double t, dt_last;  /* simulated time and last dt of the finished request */
  double latency_s;   /* completion - submission (host clock), -1 before */
  double queue_s;     /* admission - submission, -1 before */
} janc_request_info;

/* Create a server. pool_bytes of device memory hold all admitted requests
 * (pass a 256-byte aligned caller allocation in `pool`, or NULL to let the
 * server allocate it); max_active bounds the active set; chemistry as in
 * janc_grid_desc and shared by every request. */
int janc_server_create(const janc_mechanism* m, int chemistry, size_t pool_bytes, void* pool, int max_active,
                       void* cuda_stream, janc_server_t* out);

/* Cap on the summed cells of the active set (0, the default: none). A
 * queued request that would take the active set past the cap waits until the
 * active set has room or is empty (a request larger than the cap runs alone).
 * Later requests may pass it until it has waited max_skip_s seconds since its
 * submission; after that nothing behind it is admitted, so the active set
 * drains for it (max_skip_s = 0: strict arrival order under the cap). Bounds
 * how many solves share the GPU at once, so that a solve runs near full speed
 * instead of being time-shared with every admitted one. */
int janc_server_set_cell_budget(janc_server_t s, long long cells, double max_skip_s);

/* Device bytes a request of this grid occupies while active. */
int janc_server_footprint(janc_server_t s, const janc_grid_desc* d, size_t* bytes);

/* Queue a request: primitive initial fields (host) T, p, u, v [ny][nx] and
 * Y [ns][ny][nx] (copied at once), n_steps > 0 and exactly one of dt > 0 or
 * cfl > 0. *id receives the request id. JANC_E_NOMEM if the request can
 * never fit the pool. */
int janc_server_submit(janc_server_t s, const janc_grid_desc* d, const double* T, const double* p, const double* u,
                       const double* v, const double* Y, int n_steps, double dt, double cfl, int* id);

/* Run up to macro_steps macro-steps (admission, one batched step of every
 * active request, retirement); stops early when nothing is active or queued.
 * Asynchronous with respect to the GPU except for admission bookkeeping. */
int janc_server_run(janc_server_t s, int macro_steps, janc_server_info* info);

/* Run macro-steps as janc_server_run does until a request finishes: returns
 * once at least one request is done or failed that no earlier call returned
 * (its id in done_ids[0 .. *n_done), at most cap of them; any others come
 * with the next call), or after max_macro_steps macro-steps, or once
 * max_wall_s seconds of host time have passed since the call (checked after
 * each macro-step; give the time to the next expected arrival), or when
 * nothing is active or queued (after the last results have reached host
 * memory). At most two macro-steps are in flight on the GPU, so a finished
 * request is seen within about one macro-step. Lets a caller serve a stream
 * without polling every request. */
int janc_server_run_until(janc_server_t s, int max_macro_steps, double max_wall_s, int* done_ids, int cap,
                          int* n_done, janc_server_info* info);

/* State and timing of one request. */
int janc_server_poll(janc_server_t s, int id, janc_request_info* r);

/* Copy a finished request's final U [nv][ny][nx] and T [ny][nx] to host
 * memory (either may be NULL) and release it. JANC_E_DEVICE if its status
 * word was non-zero (after copying). */
int janc_server_fetch(janc_server_t s, int id, double* U, double* T);

/* Release the server (waits for its streams). */
void janc_server_destroy(janc_server_t s);

/* ------------------------------------------------------------------------
 * x-slab domain decomposition (Sec. 4.4, Fig. 3). The domain's nx columns
 * are cut into slabs of whole columns. Each slab is a grid whose x sides
 * shared with a neighbour read their 3 ghost columns from halo buffers; its
 * y sides and the domain's outer x sides keep the physical boundaries of the
 * descriptor, and a periodic x axis joins the last slab to the first. After
 * every phase of a step whose output state a neighbour's next face fluxes
 * read (RK stages 1 and 2, the step's final state) and after a state load,
 * the exchange fills each neighbour's halo with the slab's 3 edge columns of
 * all ns + 7 stored planes and makes the LF speeds of Eq. 4.11 the max over
 * all slabs (the CFL dt follows). The slabs together give the undivided
 * grid's result bit for bit: every face sees the same stencil values and
 * alpha, every cell runs the same arithmetic, and a max is exact. The
 * adjoint, the server and AMR take whole grids only.
 * ---------------------------------------------------------------------- */

/* Columns [*x0, *x0 + *nx_local) of slab k of n_slabs over nx columns: the
 * first nx % n_slabs slabs take one column more. JANC_E_INVALID unless
 * every slab has at least 3 columns (a halo is 3 columns of one neighbour).
 * Host arithmetic only. */
int janc_slab_partition(int nx, int n_slabs, int k, int* x0, int* nx_local);

/* Doubles in one halo buffer of a slab of the domain d: (ns + 7) ny 3,
 * laid out [plane][ny][3] (planes: the nv conserved variables, T, u, v, p;
 * column c of a low-side buffer is ghost column c - 3 of the receiving slab,
 * of a high-side buffer its column nx_local + c). */
int janc_slab_halo_doubles(const janc_grid_desc* d, const janc_mechanism* m, size_t* count);

/* Exchange callback of a stand-alone slab (one slab per process or rank).
 * Before each call the library has enqueued on cuda_stream the packing of
 * the slab's columns 0..2 into send_lo and nx_local-3..nx_local-1 into
 * send_hi (shared sides only) and the copy of the slab's LF speeds into
 * alpha2. The callback must enqueue, on cuda_stream or in a way ordered
 * with it (e.g. NCCL on that stream, or synchronously), the transfer of the
 * low neighbour's send_hi into recv_lo and of the high neighbour's send_lo
 * into recv_hi, and the replacement of alpha2[0..1] by the max over all
 * slabs (bit patterns of non-negative doubles: an unsigned 64-bit max).
 * It must not reuse send buffers before those transfers are done. Returns
 * 0, or non-zero to fail the library call with JANC_E_EXCHANGE. */
typedef int (*janc_exchange_fn)(void* user, void* cuda_stream);

typedef struct {
  double* send_lo;             /* device, janc_slab_halo_doubles each; the  */
  double* send_hi;             /* buffers of a side without a neighbour may */
  double* recv_lo;             /* be NULL. recv_lo / recv_hi are the slab's */
  double* recv_hi;             /* halos, read by every face-flux launch.    */
  unsigned long long* alpha2;  /* device, 2 values */
  janc_exchange_fn fn;
  void* user;                  /* passed to fn */
} janc_slab_exchange;

/* Create slab [x0, x0 + nx_local) of the domain d (nx_local >= 3) as a grid
 * of nx_local x d->ny cells: janc_set_state / janc_set_state_primitive take
 * and janc_get_state gives the slab's own arrays, and janc_step runs the
 * step with the exchange of *x after every state-producing phase (the loads
 * run it once too). Buffers of *x are owned by the caller and must stay
 * valid until janc_destroy_grid. workspace as janc_create_grid, sized by
 * janc_workspace_bytes of d with nx = nx_local (NULL: allocated here). */
int janc_slab_create(const janc_grid_desc* d, const janc_mechanism* m, int x0, int nx_local,
                     const janc_slab_exchange* x, void* workspace, size_t workspace_bytes, void* cuda_stream,
                     janc_grid_t* out);

/* Single-process split: the domain d cut into n_slabs slabs on the current
 * device (janc_slab_partition), all on cuda_stream. The slabs share one set
 * of alpha slots (so every update kernel's max already covers all slabs) and
 * exchange halos by a pack kernel that writes each slab's edge columns
 * straight into its neighbours' halo buffers. Set-up allocates each slab's
 * workspace (janc_workspace_bytes of its own size plus two halos). */
typedef struct janc_split_s* janc_split_t;
int janc_split_create(const janc_grid_desc* d, const janc_mechanism* m, int n_slabs, void* cuda_stream,
                      janc_split_t* out);
/* Whole-domain state in, as janc_set_state / janc_set_state_primitive. */
int janc_split_set_state(janc_split_t s, const double* U, const double* T0, int where);
int janc_split_set_state_primitive(janc_split_t s, const double* T, const double* p, const double* u, const double* v,
                                   const double* Y, int where);
/* n_steps steps of all slabs in lockstep, as janc_step. */
int janc_split_step(janc_split_t s, int n_steps, double dt, double cfl, double* t_out, double* dt_last_out);
/* Whole-domain state out, as janc_get_state (status: OR over the slabs). */
int janc_split_get_state(janc_split_t s, double* U, double* T, int where);
/* Status as janc_status: OR of the slabs' status words, slab 0's clock. */
int janc_split_status(janc_split_t s, janc_status_info* info);
/* Handle of slab k (owned by the split: never pass it to janc_destroy_grid),
 * e.g. for janc_profile. */
int janc_split_slab(janc_split_t s, int k, janc_grid_t* slab);
void janc_split_destroy(janc_split_t s);

/* Size of the device array behind janc_rhs_static (32 MiB per GPU). */
#define JANC_STATIC_SCRATCH_BYTES (32u << 20)

/* Right-hand side without device allocation. The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc, such as code running
 * inside another framework's memory pool, loops that forbid allocation after
 * start-up, and plug-ins that only receive device buffers.
 * Same result as janc_rhs for the state (U, T): U[nv][ny][nx] and T[ny][nx]
 * (the Newton warm start) are device inputs, L[nv][ny][nx] and alpha[2]
 * (may be NULL) device outputs; the caller owns all four. Scratch comes from
 * one file-scope device array of JANC_STATIC_SCRATCH_BYTES that every GPU
 * loading the library holds until exit; a grid whose scratch
 * ((nv + 4) nx ny + nv (2 nx ny + nx + ny) doubles plus small tables) does
 * not fit is rejected with JANC_E_INVALID. No allocation of any kind. The
 * first call on each device looks up the array's device address, so make it
 * before any stream capture. That address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys the primary
 * context) it is stale, so a process that resets a device must not call this
 * entry point on that device again. All calls share the array: calls that overlap
 * on the GPU race and must be serialised by the caller. Synchronises
 * cuda_stream before returning; JANC_E_DEVICE if the state's Newton T
 * recovery flagged a bad cell. */
int janc_rhs_static(const janc_grid_desc* d, const janc_mechanism* m, const double* U, const double* T,
                    double* L, double* alpha, void* cuda_stream);

/* ---- Block-structured adaptive mesh refinement (Sec. 3) -------------------------------------
 * Layer 0 is the base grid of the descriptor (physical boundaries). Layer i
 * (1 <= i <= levels) holds blocks of 16 x 16 cells at twice the resolution of
 * layer i-1, at fixed positions (block (bx, by) covers the layer-i cells
 * [16 bx, 16 bx + 16) x [16 by, 16 by + 16)), nested in the blocks of layer
 * i-1 (Sec. 3.1.1). A block is refined where a cell of layer i-1 within
 * n_buffer cells of its parent region has |grad T| > threshold (K/m; central
 * differences, Sec. 3.1.2). Per base step (Algorithm 2): regrid every
 * regrid_every steps (blocks kept across a regrid keep their data, new blocks
 * copy their parent one-to-four), the crossover advance (layer i+1 takes two
 * steps of dt/2 before each step of layer i), each layer solved as in
 * Algorithm 3 (ghost blocks from the same-layer neighbours or the physical
 * boundary; cells within 3 of a side with no neighbour take the layer-(i-1)
 * values after every RK stage; chemistry over the layer's dt), then the
 * four-to-one mean from the deepest layer up, onto the parent cells none of
 * whose children lies in an external band. The base dt is fixed or the CFL
 * of layer 0 at the step's start (computed on the device); layer i uses
 * dt / 2^i. A step makes no host round trip; a regrid reads back one block
 * count per layer. Layer buffers grow as needed and are kept until
 * janc_amr_destroy. Chemistry: JANC_CHEM_OFF or JANC_CHEM_LIE. nx, ny of the
 * base must be multiples of 8. */
typedef struct janc_amr_s* janc_amr_t;

typedef struct {
  int levels;         /* refined layers above the base, 0..6 */
  int block;          /* block edge in cells; must be 16 */
  double threshold;   /* refinement criterion |grad T| > threshold, K/m */
  int n_buffer;       /* buffer cells around the masked cells (layer i-1 cells) */
  int regrid_every;   /* base steps between regrids (>= 1); step 0 builds the layers */
  int synchronous;    /* 0: crossover advance (Fig. 2a); 1: synchronous advance (Fig. 2b): every
                         layer takes the step's dt (the CFL dt of layer 0 / 2^levels when the CFL
                         drives it), deepest first */
} janc_amr_desc;

/* Create an AMR hierarchy over the base grid `base` (device memory owned by
 * the object; the layers grow and shrink with the block count). */
int janc_amr_create(const janc_grid_desc* base, const janc_mechanism* m, const janc_amr_desc* a, void* cuda_stream,
                    janc_amr_t* out);
/* Base-layer state from primitive fields, as janc_set_state_primitive; the
 * refined layers are rebuilt at the next step. */
int janc_amr_set_state_primitive(janc_amr_t a, const double* T, const double* p, const double* u, const double* v,
                                 const double* Y, int where);
/* n steps with a fixed dt (> 0) or the CFL number (> 0); t_out (may be
 * null) receives the simulated time advanced. A crossover step advances the
 * base dt; a synchronous step advances dt (or the CFL dt of layer 0 / 2^levels). */
int janc_amr_step(janc_amr_t a, int n_steps, double dt, double cfl, double* t_out);
/* The block-list builder of the regrid, run on the device for checking:
 * from flags[nby][nbx] (host; non-zero = the candidate block is refined) the
 * blocks in (by, bx) order, *nblk of them, with pos[2 b] = bx and
 * pos[2 b + 1] = by, map[by nbx + bx] = the block number or -1, and
 * nbr[4 b + s] = the block across side s (north, south, west, east; the
 * periodic partner on a periodic side of bc = {left, right, bottom, top}),
 * -2 on a non-periodic domain side, -1 where the layer has no block (an
 * external side). Host outputs; pos, map and nbr sized for every candidate.
 * Synchronous; allocates scratch. */
int janc_amr_block_lists(const unsigned char* flags, int nbx, int nby, const int* bc, int* pos, int* map, int* nbr,
                         int* nblk);
/* Blocks of layer `level` (1..levels). */
int janc_amr_layer_blocks(janc_amr_t a, int level, int* nblk);
/* Host copy of layer `level`: pos[2 b] = bx, pos[2 b + 1] = by of block b
 * (blocks in (by, bx) order), U [nblk][nv][16][16], T [nblk][16][16]; any
 * pointer may be null. Synchronous. */
int janc_amr_get_layer(janc_amr_t a, int level, int* pos, double* U, double* T);
/* Base-layer state (after the last step's four-to-one means), as janc_get_state. */
int janc_amr_get_base(janc_amr_t a, double* U, double* T, int where);
/* OR of the JANC_ST_* bits of every layer since creation. Synchronous. */
int janc_amr_status(janc_amr_t a, int* status);
/* Cell updates of the last step: base cells + sum over layers of 2^i x cells
 * (crossover) or of the cells once (synchronous). */
int janc_amr_cell_updates(janc_amr_t a, long long* per_step);
void janc_amr_destroy(janc_amr_t a);

#ifdef __cplusplus
}
#endif

#endif /* JANC_H_ */
