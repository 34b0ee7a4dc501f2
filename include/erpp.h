/*
 * erpp.h -- C ABI of the GB300 implementation of the Exact Regularized Point
 * Particle (ERPP) two-way coupling step (Gualtieri, Picano, Sardina &
 * Casciola, arXiv 1405.6969).
 *
 * The library computes, on one GPU, the coupling between point particles and
 * an Eulerian fluid grid:
 *   - the regularised momentum source of Sec. 2.4, Eq. ns_regularized_filtered:
 *       S(x) = -(1/rho_f) sum_p D_p g(x - x_p, eps_R),
 *     with g the heat kernel of App. A.1 (Eq. fundamental_phys): a Gaussian
 *     of width sigma_R = sqrt(2 nu eps_R), truncated at cutoff * sigma_R on
 *     every axis and (by default) normalised to unit discrete mass per axis;
 *   - the matching kernel gather of the fluid velocity at the particles;
 *   - the removal of each particle's own regularised disturbance
 *     (Sec. 2.5 and the closed form of App. A.5, Eq. disturbance_velo);
 *   - the Stokes drag of Sec. 2.5 (Eq. force_stokes_drag) and one explicit
 *     Euler step of Eq. particle_motion.
 *
 * Conventions shared by every entry point
 *   Grid: periodic box [0,Lx) x [0,Ly) x [0,Lz), nodes at j * L / N.  Grid
 *     fields are three contiguous components, each nz*ny*nx values with x
 *     fastest: index ((c*nz + k)*ny + j)*nx + i.  Element type: float with
 *     ERPP_FP32, double with ERPP_FP64 (fixed at erpp_init).
 *   Particles: structure of arrays, one device array of n doubles per
 *     component.  Positions must lie in [0, L) on each axis.
 *   Pointers: device pointers unless stated otherwise; the caller owns every
 *     grid and particle buffer.  The context owns only its scratch memory.
 *   Streams: every call is asynchronous on the given CUDA stream (NULL = the
 *     legacy default stream) unless stated otherwise.  Calls that share one
 *     context share its scratch: issue them on one stream, in order.
 *   Errors: argument errors are reported synchronously by the return value
 *     and nothing is launched.  Data errors found on the device (NaN or
 *     out-of-box positions) set a sticky device error word that
 *     erpp_check() or erpp_momentum() report.  No call aborts or traps.
 */
#ifndef ERPP_H
#define ERPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (the same object as cudaStream_t). */
typedef struct CUstream_st* erpp_stream;

typedef enum {
  ERPP_OK = 0,
  ERPP_EINVAL = 1,   /* invalid argument or parameter                      */
  ERPP_ENOMEM = 2,   /* device allocation failed                           */
  ERPP_ECUDA = 3,    /* a CUDA runtime call failed (no device, launch ...)  */
  ERPP_ERANGE = 4,   /* a particle position was NaN/Inf or outside [0, L)  */
  ERPP_EBOUNDS = 5,  /* an internal capacity or index check failed         */
  ERPP_ETIMEOUT = 6, /* a bounded device-side wait gave up                 */
  ERPP_ESTATE = 7    /* call not valid in the context's current state      */
} erpp_status;

/* erpp_params.flags */
enum {
  ERPP_FP32 = 1u << 0,         /* float grids; FP32 kernel evaluation and
                                  accumulation; FP64 particle integration    */
  ERPP_FP64 = 1u << 1,         /* double grids; plain FP64 kernels           */
  ERPP_NORMALIZE = 1u << 2,    /* unit discrete mass per axis (recommended)  */
  ERPP_SELF_REMOVAL = 1u << 3, /* subtract the closed-form self disturbance  */
  ERPP_KAHAN = 1u << 4,        /* FP32 only: compensated scatter: each
                                  contribution's 64-bit fixed-point product
                                  summed per tile as a high and a low 32-bit
                                  word (about 46 bits below the tile's force
                                  bound, order independent), converted to
                                  FP32 once per tile; twice the shared memory
                                  of the default form                        */
  ERPP_PIC = 1u << 5,          /* classical particle-in-cell coupling instead
                                  of the regularised kernel (see below)      */
  ERPP_POINT_GATHER = 1u << 6, /* point-value gather (see below); the source
                                  stays the regularised kernel               */
  ERPP_LAG = 1u << 7,          /* delay the source by eps_R (see below)      */
  ERPP_FULL_FORCE = 1u << 8    /* the general force of Eq. force_particle   */
};

/* ERPP_FULL_FORCE: erpp_step computes the general hydrodynamic force of
 * Eq. force_particle instead of the Stokes drag: the Faxen terms (the
 * Laplacian of the gathered velocity, with the Laplacian of the removed self
 * disturbance, 2 d/ds2 of App. A.5's closed form), the fluid-acceleration and
 * added-mass terms and the Basset memory over the last step (Sec. 2.5).
 * With q = u~ + (a^2/6) lap u~, m_f = rho_f (4/3) pi a^3 and
 * c_B = 12 mu a^2 sqrt(pi / (nu dt)):
 *   F = 6 pi mu a (q - v) + m_f du~/dt + (m_f/2) d(u~ + (a^2/10) lap u~)/dt
 *       + c_B dq,    (du~/dt etc. the change over the last step / dt)
 *   [(m_p + m_f/2)/dt + c_B] (v' - v) = F + (m_p - m_f) g,
 *   D = F - [(m_f/2)/dt + c_B] (v' - v)  (what the fluid receives, negated).
 * The context keeps u~ and lap u~ of the previous step (48 bytes per
 * particle); a first step takes no time derivatives.  Gaussian weights only,
 * not with ERPP_LAG, not in the batched step (ERPP_EINVAL); dt must be
 * positive; the particle count must not change between first steps, and
 * after erpp_set_tiling or any call with more particles than the context has
 * held so far the next step must be a first step (ERPP_ESTATE).
 * Other calls (erpp_interpolate, erpp_particle_advance, ...) are unchanged. */

/* ERPP_LAG: the literal time delay of Eq. ns_regularized_filtered.  The
 * source of step n is D^(n-L) spread at x^(n-L), L = round(eps_R / dt) >= 1
 * steps earlier, instead of the step's own D^n at x^n; the first L steps
 * after a first_step have no source (S = 0).  The self disturbance removed
 * at step n is that of the previous step's source, D^(n-1-L) at x^(n-1-L)
 * (none while n < L + 1).  The context keeps the positions and forces of
 * the last L + 1 steps (48 bytes per particle and step, (L + 1) * 48 bytes
 * per particle in all).  Applies to erpp_step and erpp_step_host (the other
 * calls work on what they are given); with the Gaussian weights only
 * (ERPP_PIC / ERPP_POINT_GATHER: ERPP_EINVAL), not in the batched step
 * (ERPP_EINVAL); dt must be positive; the particle count must not change
 * between first steps, and after erpp_set_tiling or any call with more
 * particles than the context has held so far the next step must be a first
 * step (else ERPP_ESTATE). */

/* Other weights on the same grid (the comparisons of Sec. 3.2.1-3.2.2 and the
 * interpolation question of Sec. 2.5).  At most one of the two flags.
 *
 * ERPP_PIC (cloud in cell): a particle at grid coordinates s = x N / L (one
 *   rounding per axis), cell j0 = floor(s), f = s - j0, gives its force to the
 *   8 nodes j0 .. j0 + 1 (wrapped) with the trilinear weights
 *   w = prod_a (1 - f_a or f_a), as the source density
 *   S_j = -(1/rho_f) sum_p D_p w_p(j) / dV, and the fluid velocity is
 *   interpolated at the particle with the same weights.  The self
 *   disturbance of PIC has no closed form: ERPP_SELF_REMOVAL and ERPP_KAHAN
 *   are rejected with it (ERPP_EINVAL).  The scatter adds with device atomics:
 *   in FP32 the rounding of a node's sum depends on the order of arrival.
 * ERPP_POINT_GATHER: the fluid velocity at the particle is the separable
 *   4-point Lagrange (cubic) interpolant over the nodes j0 - 1 .. j0 + 2; the
 *   self disturbance is removed at the variance the particle's point sees,
 *   s2 = 2 nu (eps_R + dt), without the gather's own sigma_R^2.
 * Both keep eps_R and cutoff subject to the stencil requirements below.  They
 * apply to erpp_interpolate, erpp_particle_advance, erpp_scatter_source,
 * erpp_step, erpp_step_host and erpp_momentum; the adjoints, the batched step
 * and erpp_interpolate_noalloc return ERPP_EINVAL for such a context or
 * parameter set. */

/* Physical and numerical parameters (Sec. 2.3-2.5).  sigma_R =
 * sqrt(2 nu eps_R); the stencil keeps, per axis, the nodes within
 * r_c = cutoff * sigma_R of the particle.  Requirements: 2 r_c smaller than
 * every box side, r_c at least one grid spacing and at most 15.5 grid
 * spacings on every axis (windows of at most 31 nodes).  mu = rho_f nu. */
typedef struct {
  int32_t nx, ny, nz;  /* grid nodes per axis (>= 1)                          */
  uint32_t flags;      /* exactly one of ERPP_FP32 / ERPP_FP64, plus options  */
  double Lx, Ly, Lz;   /* box sides                                          */
  double nu;           /* kinematic viscosity                                */
  double rho_f;        /* fluid density                                      */
  double eps_R;        /* regularisation time                                */
  double cutoff;       /* stencil radius in units of sigma_R (paper: 3)      */
  double dt;           /* time step                                          */
  double gravity[3];   /* acceleration of gravity                            */
  double shear_rate;   /* mean flow shear_rate * y along x, added at the
                          particles (the grid holds the fluctuation)          */
} erpp_params;

/* Particle state: n particles, device arrays of n doubles per component. */
typedef struct {
  int64_t n;
  double* x[3];        /* position, in [0, L)                                */
  double* v[3];        /* velocity                                           */
  double* x_prev[3];   /* position one step earlier                          */
  double* D[3];        /* hydrodynamic force of the previous step            */
  const double* radius;/* particle radius a_p                                */
  const double* rho_p; /* particle density                                   */
} erpp_particles;

typedef struct erpp_ctx erpp_ctx;

/* Creates a context for one grid and parameter set on the current CUDA
 * device.  Validates params (EINVAL before any CUDA call), then allocates
 * the context's scratch (tile tables, device error word).  *out receives the
 * context; on failure *out is set to NULL. */
erpp_status erpp_init(const erpp_params* params, erpp_ctx** out);

/* Frees the context and its scratch (synchronises the device first).  NULL
 * is accepted. */
erpp_status erpp_destroy(erpp_ctx* ctx);

/* Static, NUL-terminated description of a status code. */
const char* erpp_status_string(erpp_status status);

/* Matching kernel gather: u_p[c][i] = sum_j dV W_i(j) u[c][j] (+ shear_rate *
 * y_i for c = x), W the truncated (normalised) Gaussian of the scatter.
 * x: n positions per component; u: grid field (float/double per mode);
 * u_p: n doubles per component (output). */
erpp_status erpp_interpolate(erpp_ctx* ctx, const void* u, int64_t n,
                             const double* const x[3], double* const u_p[3],
                             erpp_stream stream);

/* Self-disturbance removal, Stokes drag and one explicit Euler step
 * (Sec. 2.5).  In: u_p = fluid velocity gathered at P->x.  With self
 * removal and first_step == 0, the disturbance the particle left in the
 * previous step, v_self(x - x_prev; D), is subtracted first (App. A.5 closed
 * form at variance 2 nu (eps_R + dt) + sigma_R^2: one step of diffusion,
 * plus the gather's own filtering).  Out: P->D = 6 pi mu a (u_p - v_self - v),
 * P->v += dt (D / m_p + (1 - rho_f / rho_p) g), P->x += dt v (old v, wrapped
 * into [0, L)), P->x_prev = old x.  m_p = (4/3) pi a^3 rho_p. */
erpp_status erpp_particle_advance(erpp_ctx* ctx, const double* const u_p[3],
                                  const erpp_particles* P, int first_step,
                                  erpp_stream stream);

/* Regularised momentum source of forces D at positions x (Eq.
 * ns_regularized_filtered): S[c][j] = -(1/rho_f) sum_i D[c][i] W_i(j).
 * S (grid field) is overwritten entirely. */
erpp_status erpp_scatter_source(erpp_ctx* ctx, int64_t n, const double* const x[3],
                                const double* const D[3], void* S, erpp_stream stream);

/* Adjoint of the source (Eq. ns_regularized_filtered) for a scalar loss L of
 * S: given the cotangent R = dL/dS (grid field, float/double per mode),
 *   dD[c][i] = dL/dD_ic = -(1/rho_f) sum_j R[c][j] W_i(j),
 *   dx[a][i] = dL/dx_ia = -(1/rho_f) sum_j (R_j . D_i) dW_i(j)/dx_ia,
 * with dw/dx_p = w d / sigma_R^2 per axis factor (d = x_j - x_p) for raw
 * weights and w (d - dx sum_k w_k d_k) / sigma_R^2 for normalised ones (the
 * normalising sum depends on x_p too).  x, D: n positions and forces per
 * component; dD (may be NULL) and dx: n doubles per component (outputs,
 * overwritten).  Weights and sums in the context's precision (FP32 or FP64). */
erpp_status erpp_scatter_backward(erpp_ctx* ctx, int64_t n, const double* const x[3],
                                  const double* const D[3], const void* R, double* const dD[3],
                                  double* const dx[3], erpp_stream stream);

/* Adjoint of the kernel gather (erpp_interpolate) for a scalar loss L of u_p:
 * given g = dL/du_p (n doubles per component),
 *   du[c][j] = dL/du_cj = dV sum_i g[c][i] W_i(j)      (grid, overwritten;
 *                                                        a scatter of g),
 *   dx[a][i] = dL/dx_ia = dV sum_j (u_j . g_i) dW_i(j)/dx_ia
 *                         + shear_rate g[0][i] (a = y only).
 * du or dx may be NULL (not both).  u: the grid field the gather read. */
erpp_status erpp_gather_backward(erpp_ctx* ctx, int64_t n, const double* const x[3],
                                 const void* u, const double* const g[3], void* du,
                                 double* const dx[3], erpp_stream stream);

/* One coupling step: gather u at P->x, remove the self disturbance, drag,
 * Euler advance (as erpp_particle_advance), then scatter the new forces at
 * the positions they were evaluated at (P->x_prev after the call) into S
 * (overwritten).  The fluid field u is held fixed during the call. */
erpp_status erpp_step(erpp_ctx* ctx, const void* u, const erpp_particles* P, void* S,
                      int first_step, erpp_stream stream);

/* erpp_step on HOST data: u, S and every array of P (n doubles per
 * component, radius and rho_p included) are host memory, page-locked for the
 * copies to run asynchronously (pageable memory works, without overlap).
 * The call copies u and P in once the work already on `stream` is done,
 * runs the step on streams of its own and copies S (overwritten) and P's
 * x, v, x_prev, D (updated) back, then returns without waiting: the host
 * arrays must stay untouched, and the results are valid only after
 * erpp_step_host_wait(ctx, s) and a synchronisation of s.  Successive calls
 * overlap their copies with the neighbouring steps' computation (device
 * staging in two slots, owned by the context: 2 x (2 grids + 14 n doubles));
 * a call's particle upload waits for the previous call's particle download,
 * the host arrays being the state of record.  The Python binding's
 * Context.step_host is the user entry point. */
erpp_status erpp_step_host(erpp_ctx* ctx, const void* u, const erpp_particles* P, void* S,
                           int first_step, erpp_stream stream);
/* Makes `stream` wait until every erpp_step_host call on ctx so far has
 * copied its results back. */
erpp_status erpp_step_host_wait(erpp_ctx* ctx, erpp_stream stream);

/* Momentum bookkeeping (the impulse of Sec. 3.1): out[0..2] = dV sum_j S[c][j]
 * and out[3..5] = -(1/rho_f) sum_i M_i D[c][i], M_i the discrete kernel mass
 * (1 when normalised); both summed in FP64.  out is a HOST array of 6
 * doubles.  Synchronises the stream, then reports the sticky device error
 * word like erpp_check. */
erpp_status erpp_momentum(erpp_ctx* ctx, const void* S, int64_t n, const double* const x[3],
                          const double* const D[3], double out[6], erpp_stream stream);

/* Synchronises the stream and returns (and clears) the sticky device error:
 * ERPP_ERANGE for NaN/Inf/out-of-box positions seen since the last check,
 * ERPP_EBOUNDS for a failed internal index check, ERPP_ETIMEOUT for a
 * bounded device wait that gave up (see erpp_debug_set_wait), else ERPP_OK. */
erpp_status erpp_check(erpp_ctx* ctx, erpp_stream stream);

/* Stencil windows as the kernels compute them: for each particle and axis,
 * the first and last node index (unwrapped, may be < 0 or >= N) whose
 * distance from x is at most cutoff * sigma_R (Sec. 2.4, truncated support).
 * jlo, jhi: device int32 arrays of 3*n (component-major).  The binning takes
 * the window with one FP64 product and exact integer/FP32 work; this call
 * also evaluates the plain FP64 form and writes INT32_MIN to both ends of any
 * axis where the two disagree in the home cell, the ends or the fractional
 * position (a self-check that is never expected to fire). */
erpp_status erpp_debug_windows(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               int32_t* jlo, int32_t* jhi, erpp_stream stream);

/* Bounded device-side waits (a tracing and testing aid, not part of the
 * method).  The FP32 tile gather stages each tile by asynchronous copies
 * completed on a shared-memory barrier; one thread of the block waits for it
 * for at most limit_ns nanoseconds of the GPU's global timer, after which the
 * block records ERPP_ETIMEOUT in the context's error word (reported by
 * erpp_check) and returns, leaving no copy in flight.
 * limit_ns: 0 = the default (250 ms), else 1e3 .. 1e10.  stall: 1 makes
 * every such block, once its copies have landed, also wait on a barrier that
 * nothing ever completes, so that the wait runs out (for tests of the
 * timeout path); 0 = normal operation.  Takes effect for the context's next
 * launches; ERPP_EINVAL for values out of range. */
erpp_status erpp_debug_set_wait(erpp_ctx* ctx, int64_t limit_ns, int32_t stall);

/* Kernel gather without any allocation, for callers that must not allocate
 * device memory: code running while a memory pool is frozen or exhausted,
 * plugins handed a fixed device budget by their host application, or paths
 * that must never enter the allocator.  The paper has no counterpart; this is
 * a deployment convenience.
 * Computes exactly what erpp_interpolate computes with an ERPP_FP32 context
 * made from the same params (u is a float grid, u_p n doubles per component),
 * but takes the parameters directly and needs no context: its scratch lives
 * in one fixed 7.2 MiB array inside the library image, which every GPU that
 * loads the library holds until the process exits.  No cudaMalloc, cudaFree
 * or other allocating call is made.
 * Limits: n <= 16384 particles, at most 131072 stencil pieces (n times the
 * largest number of tiles one window can touch) and 4096 grid tiles; larger
 * problems, an ERPP_FP64 flag or invalid params return ERPP_EINVAL before any
 * launch.  Asynchronous on `stream`.  The first call in each CUDA context
 * (per device, and again in a context created later, e.g. after a device
 * reset) looks up the array's device address with that device current; make
 * that first call before any stream capture.  With lazy module loading (the
 * CUDA default) that first call is also when the array is actually placed
 * in device memory: make a first (warm-up) call before the phase in which
 * the device memory may be exhausted.  Every call, from any thread or
 * stream, uses the same array and leaves its contents behind: calls that
 * overlap on the GPU race and must be serialised (one stream, or events).
 * Positions outside [0, L) are not reported (no error word is readable);
 * their u_p is zero. */
erpp_status erpp_interpolate_noalloc(const erpp_params* params, const void* u, int64_t n,
                                     const double* const x[3], double* const u_p[3],
                                     erpp_stream stream);

/* ---- Batched boxes ---------------------------------------------------
 * Many independent periodic boxes (each with its own grid, parameters and
 * particles) stepped together.  The paper treats one box; stepping many
 * small ones at once is a throughput form of the same step. */

#define ERPP_MAX_BOXES 4096

/* One box: its parameters, its grid fields and its particle state (device
 * pointers, caller-owned, as for erpp_step).  u is read, S overwritten and
 * the particle arrays advanced by every step. */
typedef struct {
  erpp_params params;
  const void* u;
  erpp_particles particles;
  void* S;
} erpp_box_desc;

typedef struct erpp_batch erpp_batch;

/* Creates a batch over nbox (1..ERPP_MAX_BOXES) box descriptors (copied):
 * one context per box, with its scratch allocated now for the box's particle
 * count.  The descriptors' buffers must stay allocated and in place until
 * erpp_batch_destroy: the batch keeps their addresses (their contents may
 * change between steps).  *out is NULL on failure. */
erpp_status erpp_batch_init(int32_t nbox, const erpp_box_desc* boxes, erpp_batch** out);

/* One coupling step (erpp_step) of every box, asynchronous on `stream`.
 * use_graph != 0: the first call for each value of first_step captures the
 * step into one CUDA graph and every call replays it with a single graph
 * launch on `stream`; the graph's form is set by erpp_batch_set_form.
 * use_graph == 0: each box's erpp_step, one box after another on `stream`.
 * All forms compute the same thing. */
erpp_status erpp_step_batched(erpp_batch* batch, int first_step, int use_graph,
                              erpp_stream stream);

/* The form of the batched graph (not in the paper, which treats one box):
 *   ERPP_BATCH_BRANCHES (default): one independent branch per box with the
 *     box's own launches; the boxes run concurrently.
 *   ERPP_BATCH_MULTI: nine kernels for all boxes together: the binning in
 *     four (counts cleared, counted, scanned per box, records filled), a
 *     persistent gather whose blocks pull (box, tile) work items, densest
 *     boxes first, from a counter, the advance, a persistent scatter and the
 *     two halo merges.  Needs every box on the FP32 step with x/y-halo tiles,
 *     the fixed-point scatter and windows of the same longest length, else
 *     the branches are captured.  The first graph call in this form builds
 *     the boxes' device descriptors (a small device allocation, before the
 *     capture).
 * Discards captured graphs.  ERPP_EINVAL for other values. */
enum { ERPP_BATCH_BRANCHES = 0, ERPP_BATCH_MULTI = 1 };
erpp_status erpp_batch_set_form(erpp_batch* batch, int32_t form);

/* erpp_set_tiling for one box (0 <= box < nbox) of the batch; the box's
 * scratch is reallocated at once and captured graphs are discarded (the next
 * erpp_step_batched with a graph captures again). */
erpp_status erpp_batch_set_tiling(erpp_batch* batch, int32_t box, int32_t tile_y,
                                  int32_t tile_z, int32_t threads);

/* erpp_get_tiling of box `box` (0 <= box < nbox, else ERPP_EINVAL); out is a
 * HOST array of 5. */
erpp_status erpp_batch_get_tiling(erpp_batch* batch, int32_t box, int32_t out[5]);

/* The kernels of one batched step, written to the HOST int *n: the sum over
 * the boxes of erpp_last_step_launches, plus the nine multi-box kernels when
 * the graph holds them (a captured graph replays what was recorded at
 * capture). */
erpp_status erpp_batch_last_step_launches(erpp_batch* batch, int32_t* n);

/* erpp_check over every box: synchronises `stream`, returns the first error
 * found (and clears each box's error word). */
erpp_status erpp_batch_check(erpp_batch* batch, erpp_stream stream);

/* Frees the batch, its contexts and graphs (synchronises the device first).
 * NULL is accepted. */
erpp_status erpp_batch_destroy(erpp_batch* batch);

/* ---- Fluid stand-in ---------------------------------------------------
 * One exact step of the periodic unsteady Stokes equations forced by the
 * source, with the forcing / projection / diffusion split App. A.5 uses for
 * one step (the linear disturbance problem of Sec. 2.2):
 *   u_hat <- exp(-nu |k|^2 dt) P(k) (u_hat + dt S_hat),
 * P(k) = I - k k^T / |k|^2 (identity on the mean mode), k_a = 2 pi m_a / L_a.
 * It closes the two-way coupling loop in place of the paper's DNS solver
 * (Sec. 3-4), which is not part of this library. */

typedef struct erpp_fluid erpp_fluid;

/* Creates the stand-in for the grid, nu and dt of params (precision from
 * ERPP_FP32 / ERPP_FP64; other flags ignored; every axis needs >= 2 nodes).
 * Allocates the spectral scratch (3 nz ny (nx/2+1) complex values) and the
 * FFT plans on the current device. */
erpp_status erpp_fluid_init(const erpp_params* params, erpp_fluid** out);

/* u <- one Stokes step of u forced by S (both grid fields of the fluid's
 * precision, [3][nz][ny][nx]); u is overwritten (also used as the transform
 * input), S is read.  Asynchronous on `stream`. */
erpp_status erpp_fluid_stokes_step(erpp_fluid* fluid, void* u, const void* S,
                                   erpp_stream stream);

/* Frees the stand-in (synchronises the device first).  NULL is accepted. */
erpp_status erpp_fluid_destroy(erpp_fluid* fluid);

/* ---- Tiling (performance tuning; results do not depend on it beyond
 * floating-point summation order) ---------------------------------------
 * FP32 contexts whose windows span at most 16 nodes in x and y use tiles of
 * W x T_y x T_z nodes staged with x- and y-halos, processed by one block of
 * 256 or 512 threads; the default is T_y = 16, T_z = 4, 256 threads.
 * erpp_set_tiling requests T_y in 1..32, T_z in {1, 2, 4} and threads in
 * {256, 512} (0 = default each); T_y is raised to the halo depth and T_z
 * reduced when the staged tile would not fit in shared memory.  Synchronises
 * the device and frees the context's scratch (reallocated on the next call);
 * EINVAL for other values.  Contexts outside that scope accept the call and
 * keep their own tiling. */
erpp_status erpp_set_tiling(erpp_ctx* ctx, int32_t tile_y, int32_t tile_z, int32_t threads);

/* How the FP32 scatter (x/y-halo tiles) adds each tile's halo to its
 * neighbours (a tuning option: every mode computes the same sums up to the
 * order of FP32 additions, and each is reproducible bit for bit):
 *   ERPP_SCATTER_MERGE (default): one block per tile writes its interior to S
 *     and its halo to strips in a context buffer; two merge kernels then add
 *     the strips onto the neighbouring tiles' rims.
 *   ERPP_SCATTER_CLUSTER: the x-tiles of each (y, z) tile row run as one
 *     thread-block cluster, and every tile adds its x-neighbours' halo columns
 *     to its own rim straight from their shared memory (fixed order: own,
 *     left, right); the y-halo still goes through strips and one merge kernel.
 *     Needs rows of at most 8 x-tiles starting on multiples of 4 nodes (nx a
 *     multiple of 4) and a 16-byte aligned S, and enough resources for a
 *     cluster to be resident; otherwise the MERGE form runs.
 *   ERPP_SCATTER_XCLIP: the binning cuts every x-window at x-tile boundaries
 *     (a window that crosses one becomes two pieces, one per tile), so no
 *     tile adds to its x-halo; only the y-halo goes through strips and one
 *     merge kernel.  The gather uses the same pieces.
 * ERPP_EINVAL for other values. */
enum { ERPP_SCATTER_MERGE = 0, ERPP_SCATTER_CLUSTER = 1, ERPP_SCATTER_XCLIP = 2 };
erpp_status erpp_set_scatter_mode(erpp_ctx* ctx, int32_t mode);

/* out[0] = tile design in use (4: x/y-halo tiles, 3: x-halo tiles cut in y
 * and z), out[1..3] = tile size W, T_y, T_z, out[4] = threads per block.
 * out is a HOST array of 5. */
erpp_status erpp_get_tiling(erpp_ctx* ctx, int32_t out[5]);

/* Number of kernels the most recent erpp_step on ctx launched (0 before the
 * first; memsets and event records are not kernels), written to the HOST
 * int *n.  A tracing aid for launch-count accounting. */
erpp_status erpp_last_step_launches(erpp_ctx* ctx, int32_t* n);

/* Per-phase timing (a tracing aid, not part of the method).  After
 * erpp_profile_enable(ctx, 1) every erpp_step records CUDA events on its
 * stream around its phases: 0 binning (count, scan, fill), 1 gather,
 * 2 removal + drag + advance, 3 scatter.  erpp_profile_read synchronises the
 * device, writes the accumulated milliseconds per phase to the HOST array
 * ms[4] and the number of timed steps to *steps, and resets the counters.
 * Up to 1024 steps are kept between two reads (older ones are dropped). */
erpp_status erpp_profile_enable(erpp_ctx* ctx, int enable);
erpp_status erpp_profile_read(erpp_ctx* ctx, double ms[4], int64_t* steps);

/* Measured peak of the scatter's accumulating operation (a measurement aid,
 * not part of the method).  In the scatter (Sec. 2.4, Eq.
 * ns_regularized_filtered) each stencil node of each particle receives one
 * contribution per force component, which the tile kernels add to the
 * staged tile with one shared-memory atomic add: a 32-bit fixed-point
 * integer (ERPP_RATE_SHARED_S32), or an FP32 value on tiles of more than
 * 1024 pieces (ERPP_RATE_SHARED_F32).  erpp_shared_add_rate times that add
 * on the current device with nothing else limiting it (every SM full of
 * 256-thread blocks whose lanes add to 32 distinct banks, 16 adds unrolled
 * per loop iteration; the fastest of three timed launches after one
 * warm-up) and writes the lane adds completed per second to the HOST
 * double *adds_per_s.  Synchronous: it allocates 4 bytes of device memory,
 * a stream and two events, and frees them before returning.  ERPP_EINVAL
 * for another kind or a null pointer (*adds_per_s is then untouched),
 * ERPP_ECUDA or ERPP_ENOMEM when a CUDA call fails (*adds_per_s = 0). */
enum { ERPP_RATE_SHARED_S32 = 0, ERPP_RATE_SHARED_F32 = 1 };
erpp_status erpp_shared_add_rate(int32_t kind, double* adds_per_s);

#ifdef __cplusplus
}
#endif

#endif /* ERPP_H */
