/*
 * lbm_elastic.h -- C ABI of the GB300 (sm_103a) library for the
 * single-relaxation-time D2Q9 lattice Boltzmann method for wave propagation
 * in isotropic linear elastic solids (Escande, Kolluru, Cleon, Sagaut,
 * arXiv 2009.06404).
 *
 * One time step (Sec. 2, Eq. 18, with Eqs. 9-15) per cell:
 *   1. pull streaming  f_i(x) = f*_i(x - c_i), with the wall rules below;
 *   2. moments         rho = sum f, m = sum f c, P = sum f c c;
 *   3. density gradient by centred differences (Eq. 10);
 *   4. source          S = (mu - lambda)/rho0 grad rho + F - A j   (Eqs. 9, 44),
 *                      physical flux j = (m + (S_elastic + F)/2) / (1 + A/2);
 *   5. equilibrium     f^eq = w (rho + c.j/b^2 + P^n:(cc - b^2 I)/(2 b^4)),
 *                      P^n = P - rho b^2 I                       (Eqs. 14-15);
 *   6. BGK + forcing   f* = f - (f - f^eq)/tau + (1 - 1/(2 tau)) w c.S/b^2 (Eqs. 11, 18);
 *   7. displacement    u += j / rho0 (Delta t = 1), receivers record (u, j/rho0).
 * Lattice units: Delta x = Delta t = 1, b^2 = 1/3 (the S-wave speed).
 *
 * Boundaries (Sec. 6): periodic (must pair top/bottom or left/right), rigid
 * wall by half-way bounce-back (Eq. 36), free surface by anti-bounce-back with
 * rho_air and the tangential stress extrapolated to the wall, the normal and
 * shear stress set to zero (Eqs. 37-42), and absorbing layers
 * A(x) = A_max (d/L)^2 on any side (Sec. 6.4, Eq. 44).  Body force: sum over sources of
 * amplitude * dir * exp(-|x-x_s|^2/(2 sigma^2)) * ricker(n) inside r_cut
 * (Sec. 5), evaluated at t = n for step n.
 *
 * Grid layout seen by callers: row-major [ny][nx], x fastest; row y = 0 is the
 * TOP row.  Population order: c_0 = (0,0); c_1..4 = (1,0),(0,1),(-1,0),(0,-1);
 * c_5..8 = (1,1),(-1,1),(-1,-1),(1,-1).  Populations are deviations from a
 * rest state with zero density (the step is linear-affine, so this is exact).
 *
 * Memory ownership: the caller owns ALL device memory.  It passes one device
 * workspace of lbm_elastic_workspace_bytes() bytes to lbm_elastic_create and
 * keeps it alive until lbm_elastic_destroy.  The library never calls
 * cudaMalloc/cudaFree; the handle itself holds only host memory.
 *
 * Streams: every call enqueues its device work on the stream given at create
 * (0 = the legacy default stream).  lbm_elastic_step is asynchronous.  Calls
 * that return data to the host synchronise that stream.
 *
 * Errors: every function returns an lbm_status; nothing is thrown across the
 * ABI.  Argument errors are reported synchronously.  A non-finite value met by
 * the step kernel (an unstable run, Sec. 4) sets a device flag that the next
 * synchronising call reports as LBM_ERR_NONFINITE.  lbm_elastic_last_error
 * gives a message for the last failing call on a handle.
 *
 * Threads: one handle must not be used by two host threads at once.
 */
#ifndef LBM_ELASTIC_H
#define LBM_ELASTIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ELASTIC_ABI_VERSION 1

typedef struct lbm_elastic lbm_elastic_t;

typedef enum {
  LBM_OK = 0,
  /* set_material: mu/rho0 differs from b^2 = 1/3 somewhere.  The lattice fixes
   * v_S = b (Sec. 2, after Eq. 12); Lambda = (mu - lambda)/(rho0 b^2) (Eq. 32)
   * is still used as given.  Not an error. */
  LBM_WARN_VS_NOT_B = 1,
  LBM_ERR_ARG = -1,         /* invalid argument, size or pointer            */
  LBM_ERR_UNSUPPORTED = -2, /* a valid request this build does not support  */
  LBM_ERR_WORKSPACE = -3,   /* workspace too small or misaligned            */
  LBM_ERR_CUDA = -4,        /* a CUDA runtime call failed                   */
  LBM_ERR_NONFINITE = -5,   /* NaN/Inf met by a step (unstable run)         */
  LBM_ERR_TIMEOUT = -6,     /* a bounded device wait gave up                */
  LBM_ERR_CAPACITY = -7     /* more sources/receivers than reserved at create */
} lbm_status;

/* Storage type of the populations.  F64 computes in FP64; the others compute
 * in FP32 (F16/BF16 store deviations from rest times 2^store_scale_log2,
 * rounded to the 16-bit type at every step). */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 } lbm_storage;

/* Boundary kinds (Sec. 6). */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_FREE = 1, LBM_BC_RIGID = 2 } lbm_bc;

typedef struct {
  int nx, ny;            /* grid size; both >= 3                              */
  int storage;           /* lbm_storage                                       */
  int u_fp64;            /* 1: accumulate the displacement in FP64            */
  double tau;            /* BGK relaxation time (> 0.5), Eq. 18               */
  int bc_top, bc_bottom, bc_left, bc_right;             /* lbm_bc             */
  int sponge_top, sponge_bottom, sponge_left, sponge_right; /* layer cells, >= 0 */
  double sponge_amax;    /* A_max of every layer; <= 0 selects 12.8 / L       */
  int free_surface_order; /* extrapolation of rho_air and the tangential stress
                           * to a free surface: 1 = linear, 1.5 x_b - 0.5 x_in
                           * as printed (Eq. 39; it has growing modes: up to
                           * x1.046 per step at tau = 1), 0 = constant, the
                           * boundary cell's own values (neutrally stable).
                           * The density-gradient ghost follows the same
                           * order: 2 rho_b - rho_in, or rho_b.               */
  int material_per_cell; /* 0: material given per row (ny values); 1: per cell */
  int max_sources;       /* capacity reserved in the workspace (>= 0)         */
  int max_receivers;     /* capacity reserved in the workspace (>= 0)         */
  int max_steps_traced;  /* receiver samples kept: steps [0, max) after reset */
  int kernel_variant;    /* step kernel: 0 = default, 1 = one thread per cell
                          * with direct loads (the only variant; 0 selects
                          * it) */
  int store_scale_log2;  /* 16-bit storage keeps f * 2^k (k in [-60, 60]) so
                          * that the populations' range fits FP16; ignored
                          * for FP32/FP64 */
} lbm_elastic_config;

/* One Ricker x Gaussian body-force source (Sec. 5).  Position in cells (may be
 * fractional), sigma and r_cut in cells, force direction (used as given, not
 * normalised), amplitude, Ricker peak frequency f_peak (1/steps) and delay t0
 * (steps): r(t) = (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2). */
typedef struct {
  double x, y, sigma, dir_x, dir_y, amplitude, f_peak, t0, r_cut;
} lbm_source;

/* Bytes of device workspace a configuration needs (0 for an invalid one).
 * The workspace must start on a 256-byte boundary. */
size_t lbm_elastic_workspace_bytes(const lbm_elastic_config *cfg);

/* Creates a handle over a caller-owned device workspace and resets the state
 * to rest (f* = 0, u = 0, step 0).  The material defaults to a homogeneous
 * Poisson solid with rho0 = 1 (lambda = mu = 1/3); no sources; no receivers.
 * cuda_stream is a cudaStream_t (NULL for the default stream).  Synchronous. */
lbm_status lbm_elastic_create(const lbm_elastic_config *cfg, void *d_workspace,
                              size_t workspace_bytes, void *cuda_stream,
                              lbm_elastic_t **out);

/* Material (Sec. 2, Eqs. 9 and 32): rho0, lambda and mu, FP64, each with ny
 * entries (material_per_cell = 0, one value per row) or nx*ny entries
 * ([ny][nx]).  Pointers are device pointers if on_device, else host pointers.
 * The kernel forms Lambda = (mu - lambda)/(rho0 b^2) and 1/rho0.  Returns
 * LBM_WARN_VS_NOT_B (still applied) if |mu/(rho0 b^2) - 1| > 1e-9 anywhere,
 * LBM_ERR_ARG if some rho0 <= 0 or a value is not finite.  Synchronous. */
lbm_status lbm_elastic_set_material(lbm_elastic_t *h, const double *rho0,
                                    const double *lambda, const double *mu,
                                    int on_device);

/* Replaces the source list (host array of n <= max_sources entries; n = 0
 * removes every source).  sigma > 0, r_cut >= 0 required. */
lbm_status lbm_elastic_set_sources(lbm_elastic_t *h, const lbm_source *src, int n);

/* Replaces the receivers: host array xy[2n] of cell coordinates (x, y), n <=
 * max_receivers, each inside the grid.  Clears the recorded traces; steps
 * taken afterwards are recorded from trace slot 0. */
lbm_status lbm_elastic_set_receivers(lbm_elastic_t *h, const int *xy, int n);

/* Replaces the absorbing layers (Sec. 6.4, Eq. 44) of a running simulation:
 * thicknesses in cells (>= 0, each opposite pair at most the grid's extent)
 * and A_max (<= 0: 12.8 / L per layer).  The state is kept; the next step
 * uses the new layers.  The boundary kinds of the edges stay as created
 * (the paper's surface-wave experiment of Sec. 7 removes the lateral layers
 * of a laterally periodic grid after 400 steps). */
lbm_status lbm_elastic_set_sponges(lbm_elastic_t *h, int top, int bottom, int left, int right,
                                   double amax);

/* Back to rest: f* = 0, u = 0, step index 0, traces cleared, error flag
 * cleared.  Material, sources and receivers are kept.  Asynchronous. */
lbm_status lbm_elastic_reset(lbm_elastic_t *h);

/* Advances nsteps >= 0 time steps (asynchronous; nsteps = 0 is a no-op).  Each
 * step also records the receivers while fewer than max_steps_traced steps
 * have been recorded since the last reset / set_receivers / set_state. */
lbm_status lbm_elastic_step(lbm_elastic_t *h, int nsteps);

/* Time steps per kernel launch in lbm_elastic_step: 1, or 2, which advances
 * two steps per launch with the intermediate populations kept in on-chip
 * shared memory (each population then crosses HBM once per two steps).
 * Until set, the handle chooses: 2 for FP32, and for 16-bit storage when
 * every Lambda is zero; 1 for FP64 (bound by the FP64 arithmetic rather
 * than by memory) and for 16-bit storage with the density-gradient force
 * (issue-bound, where the larger two-step window costs more than the bytes
 * it saves).  An odd remainder takes a one-step launch.  Both settings give
 * bit-identical states and traces.  Returns LBM_ERR_ARG for any other
 * value. */
lbm_status lbm_elastic_set_steps_per_launch(lbm_elastic_t *h, int steps);

/* Index n of the next step (number of steps taken since reset or the step
 * given to set_state). */
long long lbm_elastic_step_index(const lbm_elastic_t *h);

/* Fields of the current state, FP64, each [ny][nx]: displacement u, velocity
 * v = j/rho0 with j the physical flux that the next step will use (with the
 * half-force shift), density rho and second moment P = -sigma (Sec. 2) of the
 * streamed populations.  Any pointer may be NULL to skip that field.  Device
 * pointers if on_device, else host pointers.  Synchronises; returns
 * LBM_ERR_NONFINITE if a step met a non-finite value. */
lbm_status lbm_elastic_read_fields(lbm_elastic_t *h, double *ux, double *uy,
                                   double *vx, double *vy, double *rho,
                                   double *pxx, double *pxy, double *pyy,
                                   int on_device);

/* Number of steps recorded in the trace buffer so far. */
int lbm_elastic_traces_recorded(const lbm_elastic_t *h);

/* Copies the recorded traces, FP64 [T][R][4] with T = traces_recorded and R =
 * the receiver count; the four values are (u_x, u_y, v_x, v_y) after each
 * step.  Synchronises. */
lbm_status lbm_elastic_read_traces(lbm_elastic_t *h, double *out, int on_device);

/* Sets the state from FP64 arrays: post-collision populations f9 [9][ny][nx]
 * (the state a step streams from) and displacement u2 [2][ny][nx] (NULL: zero).
 * The step index becomes `step`; traces are cleared.  Values are rounded to
 * the storage type.  Synchronous. */
lbm_status lbm_elastic_set_state(lbm_elastic_t *h, const double *f9,
                                 const double *u2, long long step, int on_device);

/* Reads the state as FP64 arrays (either pointer may be NULL).  Synchronises. */
lbm_status lbm_elastic_get_state(lbm_elastic_t *h, double *f9, double *u2,
                                 int on_device);

/* Checkpoint in the storage type: lbm_elastic_checkpoint_bytes() bytes holding
 * the populations, the displacement and the step index.  save/load copy to or
 * from a caller buffer (device if on_device).  load clears the traces.  A
 * checkpoint only loads into a handle of the same configuration. */
size_t lbm_elastic_checkpoint_bytes(const lbm_elastic_t *h);
lbm_status lbm_elastic_save(lbm_elastic_t *h, void *buf, int on_device);
lbm_status lbm_elastic_load(lbm_elastic_t *h, const void *buf, int on_device);

/* Deterministic FP64 sums over the grid of the current post-collision state:
 * out[0..6] = sum rho, sum m_x, sum m_y, sum P_xx, sum P_xy, sum P_yy,
 * sum (u_x^2 + u_y^2).  Fixed summation order (per-block partials in the
 * workspace, then one block), so repeated calls give identical bits.
 * Synchronises. */
lbm_status lbm_elastic_moment_sums(lbm_elastic_t *h, double out[7]);

/* Waits for the handle's stream; reports LBM_ERR_NONFINITE / LBM_ERR_CUDA. */
lbm_status lbm_elastic_sync(lbm_elastic_t *h);

/* Releases the handle (host memory only; the workspace stays the caller's). */
lbm_status lbm_elastic_destroy(lbm_elastic_t *h);

/* Message of the last failing call on h ("" if none).  Valid until the next
 * call on h.  With h == NULL: the last failure, on the calling thread, of a
 * call made without a handle (lbm_elastic_create,
 * lbm_elastic_moment_sums_noalloc); each thread keeps its own message. */
const char *lbm_elastic_last_error(const lbm_elastic_t *h);

/* Static name of a status code. */
const char *lbm_elastic_status_string(int status);

/* Number of kernel launches this handle has issued (for launch accounting). */
long long lbm_elastic_kernel_launches(const lbm_elastic_t *h);

/* ---- Moment sums without a workspace (no counterpart in the paper) -------
 *
 * The same deterministic sums as lbm_elastic_moment_sums, for callers that
 * can neither hand the library a workspace nor let it allocate: code whose
 * device memory is entirely pre-reserved by another allocator (a framework's
 * caching pool or a fixed arena), or code running where a cudaMalloc could
 * fail, or stall the whole device, at a bad moment.  This entry point
 * allocates nothing: its scratch (the per-block partial sums) is a fixed
 * array of LBM_NOALLOC_SCRATCH_BYTES bytes inside the library image, which
 * every GPU that loads the library holds until the process exits.
 *
 *   f9      9 population planes, each [ny][pitch] elements, plane after plane
 *           (plane stride pitch * ny), in the storage type (FP64 or FP32);
 *   u2      2 displacement planes in the same layout, FP64 if storage is
 *           LBM_F64 or u_fp64 is set, else FP32;
 *   out7    sum rho, sum m_x, sum m_y, sum P_xx, sum P_xy, sum P_yy,
 *           sum (u_x^2 + u_y^2) over the nx x ny cells, FP64; a host pointer
 *           (the call then waits for the stream) or, with out_on_device, a
 *           device pointer written asynchronously on the stream.
 * All pointers are the caller's; work runs on cuda_stream (NULL: default).
 * Sizes: nx, ny >= 1, pitch >= nx and 9 * pitch * ny <= LBM_NOALLOC_MAX_ELEMENTS;
 * anything else returns LBM_ERR_ARG (storage other than F64/F32:
 * LBM_ERR_UNSUPPORTED) with a message in lbm_elastic_last_error(NULL).
 * The first call on a device looks up the array's device address on that
 * (current) device; make that first call before any stream capture.  All
 * calls on a device share the one array, and each call overwrites every part
 * of it that it reads, so nothing carries over; calls whose work overlaps on
 * the GPU (e.g. on two streams at once) race on the array and must be
 * ordered by the caller. */
#define LBM_NOALLOC_SCRATCH_BYTES 19520
#define LBM_NOALLOC_MAX_ELEMENTS 2147483647LL
lbm_status lbm_elastic_moment_sums_noalloc(const void *f9, const void *u2, int storage,
                                           int u_fp64, int nx, int ny, int pitch,
                                           double *out7, int out_on_device,
                                           void *cuda_stream);


/* ------------------------------------------------------------------------
 * Batches: many independent grids ("shots") advanced together.
 *
 * A batch references existing handles (each keeps its own workspace,
 * material, sources, receivers and traces) and advances all of them by the
 * same number of steps with one launch per step, or with one persistent
 * launch for many steps.  The step of every cell is the single-grid step
 * (Sec. 2, Eq. 18, with the boundaries of Sec. 6 and the sources of Sec. 5),
 * so a shot advanced in a batch gives the same result as the shot advanced
 * alone.  Each step is split into tiles of 32 x rows cells of all shots, or
 * each pair of steps into the tiles of the two-step kernels (the
 * intermediate step in shared memory); how the tiles are launched is the
 * batch's launch configuration, which lbm_batch_autotune chooses by timing
 * the candidates on the batch itself.
 *
 * Requirements: every shot has the same storage type and u_fp64 setting.
 * The shots must not be stepped or changed by other calls while a batched
 * call is in flight; changes made between batched calls (sources, material,
 * receivers, state) are picked up by the next batched call.  The caller owns
 * the batch workspace (lbm_batch_workspace_bytes, 256-byte aligned) and
 * keeps it and the shots alive until lbm_batch_destroy.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch_t;

typedef enum {
  LBM_BATCH_AUTO = 0,       /* tune on the first lbm_batch_step of >= 96 steps */
  LBM_BATCH_STREAM = 1,     /* one launch per step (programmatic dependent launch) */
  LBM_BATCH_GRAPH = 2,      /* the same launches captured in a CUDA graph   */
  LBM_BATCH_PERSISTENT = 3  /* one cooperative launch for steps_per_launch steps:
                               blocks claim tiles from an atomic queue and meet at a
                               grid barrier after every step */
} lbm_batch_mode;

typedef struct {
  int mode;              /* lbm_batch_mode                                    */
  int rows;              /* tile height: 4 or 8 (tiles are 32 cells wide)     */
  int order;             /* 0: tiles shot by shot, row-major; 1: tiles near an
                            edge, a source or a receiver first (the expensive
                            ones), then the rest                               */
  int graph_steps;       /* GRAPH: steps per captured graph, >= 1             */
  int steps_per_launch;  /* PERSISTENT: steps per cooperative launch, >= 1    */
  int ctas_per_sm;       /* PERSISTENT: resident blocks per SM, 0 = all that fit */
  long long barrier_cycles; /* PERSISTENT: grid-barrier wait limit in SM clock
                               cycles (0 = 4e9); past it the kernel stops and
                               lbm_batch_sync returns LBM_ERR_TIMEOUT           */
  int barrier_extra;     /* PERSISTENT, for tests of the time-out: arrivals each
                            barrier waits for beyond the grid size (> 0: every
                            wait runs out).  Normally 0.                        */
  int steps_per_tile;    /* 1: one time step per launch (PERSISTENT: per grid
                            barrier) on tiles of 32 x rows cells; 2: two time
                            steps per launch on the tiles of the two-step
                            kernels (30 x 14 cells, 28 x 12 with the
                            density-gradient force; rows unused), the
                            intermediate populations in shared memory, and an
                            odd remainder as one one-step launch.  GRAPH's
                            graph_steps then counts launches; PERSISTENT's
                            steps_per_launch still counts time steps.        */
} lbm_batch_launch;

/* Workspace bytes for a batch of these n shots. */
size_t lbm_batch_workspace_bytes(lbm_elastic_t *const *shots, int n);

/* Creates a batch of n >= 1 shots.  d_workspace: device memory of at least
 * lbm_batch_workspace_bytes bytes, 256-byte aligned.  cuda_stream: the
 * stream every batched call uses (0 = legacy default).  Errors: LBM_ERR_ARG
 * (null shot, n < 1, mixed storage types), LBM_ERR_WORKSPACE; the message is
 * then in lbm_batch_last_error(NULL) (kept per calling thread). */
lbm_status lbm_batch_create(lbm_elastic_t *const *shots, int n, void *d_workspace, size_t bytes,
                            void *cuda_stream, lbm_batch_t **out);

/* Sets / reads the launch configuration (LBM_ERR_ARG for values outside the
 * ranges above). */
lbm_status lbm_batch_set_launch(lbm_batch_t *b, const lbm_batch_launch *l);
lbm_status lbm_batch_get_launch(const lbm_batch_t *b, lbm_batch_launch *l);

/* Times each candidate configuration (the three modes x both orders x
 * {one step per tile with rows 4 or 8, two steps per tile}: 18) on the batch
 * itself, two untimed steps and then steps_per_trial steps (rounded up to
 * even) timed, and keeps the fastest.  This ADVANCES every shot by
 * 18 x (2 + steps_per_trial rounded up to even) steps.  *us_per_step (may
 * be NULL) receives the best time per step in microseconds.  Synchronises
 * the stream.  LBM_BATCH_AUTO runs it with steps_per_trial 2 (72 steps) on
 * the first call of at least 96 steps. */
lbm_status lbm_batch_autotune(lbm_batch_t *b, int steps_per_trial, double *us_per_step);

/* Advances every shot by nsteps >= 0 steps (asynchronous). */
lbm_status lbm_batch_step(lbm_batch_t *b, int nsteps);

/* Synchronises the stream; reports a grid-barrier time-out (LBM_ERR_TIMEOUT)
 * or a non-finite value met in any shot (LBM_ERR_NONFINITE). */
lbm_status lbm_batch_sync(lbm_batch_t *b);

/* Kernel launches made by batched calls so far, and cells over all shots. */
long long lbm_batch_kernel_launches(const lbm_batch_t *b);
long long lbm_batch_cells(const lbm_batch_t *b);

lbm_status lbm_batch_destroy(lbm_batch_t *b);
const char *lbm_batch_last_error(const lbm_batch_t *b);


/* ------------------------------------------------------------------------
 * Adjoint (reverse mode): gradients of a function J of the receiver traces
 * with respect to Lambda = (mu - lambda)/(rho0 b^2) per cell (hence lambda
 * and mu, Eq. 32; rho0 held fixed) and to each source amplitude (Sec. 5).
 *
 * The adjoint step is the exact transpose of the step's linear part (pull
 * streaming with the wall rules of Sec. 6, the centred density gradient of
 * Eq. 10 with its wall ghosts, the absorbing layer of Eq. 44, the collision
 * with forcing of Eqs. 11-18 and u += j/rho0).  lbm_adjoint_forward runs
 * nsteps steps from the handle's current state and saves a checkpoint every
 * checkpoint_every steps; lbm_adjoint_backward walks the segments backwards,
 * recomputes each one from its checkpoint (storing its density gradients)
 * and runs its adjoint steps in reverse.  Supported for F32 and F64 storage
 * (u in the storage precision); the adjoint state is in the storage
 * precision, the gradient sums in FP64.
 *
 * All array arguments of the lbm_adjoint_* calls are DEVICE pointers.  Trace
 * adjoints: [nsteps][nrec][4], the derivative of J with respect to the
 * traces the forward run recorded (u_x, u_y after the step, v_x, v_y of the
 * step), by receiver index.  Output fields are dense [ny][nx] FP64.  The
 * calls run on the handle's stream; the handle must not be used by other
 * calls meanwhile.  After lbm_adjoint_backward the handle is back in the
 * state lbm_adjoint_forward left it in.
 * ------------------------------------------------------------------------ */
typedef struct lbm_adjoint lbm_adjoint_t;

/* Workspace bytes: three adjoint population sets and a few planes, the
 * density gradients of one segment, and ceil(nsteps / checkpoint_every) + 1
 * state checkpoints.  0 for invalid arguments. */
size_t lbm_adjoint_workspace_bytes(const lbm_elastic_t *h, int nsteps, int checkpoint_every);

/* Errors: LBM_ERR_ARG, LBM_ERR_UNSUPPORTED (F16/BF16 storage, or FP64 u with
 * FP32 populations), LBM_ERR_WORKSPACE (too small or not 256-byte aligned);
 * message in lbm_adjoint_last_error(NULL) (kept per calling thread). */
lbm_status lbm_adjoint_create(lbm_elastic_t *h, int nsteps, int checkpoint_every,
                              void *d_workspace, size_t bytes, lbm_adjoint_t **out);

/* nsteps forward steps with checkpoints; the handle records traces as
 * lbm_elastic_step does. */
lbm_status lbm_adjoint_forward(lbm_adjoint_t *a);

/* The reverse sweep for trace adjoints d_dtraces (may be NULL without
 * receivers).  Accumulates the gradients read by lbm_adjoint_gradients. */
lbm_status lbm_adjoint_backward(lbm_adjoint_t *a, const double *d_dtraces);

/* dJ/dlambda, dJ/dmu, dJ/dLambda per cell and dJ/d amplitude per source
 * (any output may be NULL).  Synchronises the stream. */
lbm_status lbm_adjoint_gradients(lbm_adjoint_t *a, double *d_g_lambda, double *d_g_mu,
                                 double *d_g_Lambda, double *d_g_amp);

/* For tests of the transpose: the adjoint state (adjoint of the
 * post-collision populations [9][ny][nx] and of u [2][ny][nx]; NULL reads
 * as zero), and one adjoint step of the linear part at the handle's step
 * index (no trace adjoint, no gradient sums). */
lbm_status lbm_adjoint_set_state(lbm_adjoint_t *a, const double *d_abar9, const double *d_ubar2);
lbm_status lbm_adjoint_get_state(lbm_adjoint_t *a, double *d_abar9, double *d_ubar2);
lbm_status lbm_adjoint_step_linear(lbm_adjoint_t *a);

/* 1 (default): each adjoint step is one fused kernel that stages the local
 * transposes of a tile and a two-cell ring in shared memory; 0: three
 * kernels (local transpose, density adjoint, push) through global memory.
 * Both compute the same transpose. */
lbm_status lbm_adjoint_set_fused(lbm_adjoint_t *a, int fused);

long long lbm_adjoint_kernel_launches(const lbm_adjoint_t *a);
lbm_status lbm_adjoint_destroy(lbm_adjoint_t *a);
const char *lbm_adjoint_last_error(const lbm_adjoint_t *a);

#ifdef __cplusplus
}
#endif

#endif /* LBM_ELASTIC_H */
