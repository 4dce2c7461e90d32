/*
 * sif.h -- C-ABI of libsif: GB300-native (sm_103a, FP64) conservative
 * sharp-interface solver for compressible two-fluid flow with
 * multi-time-step sub-cycling, after Long, Cai & Pan, "An accelerated
 * sharp-interface method for multiphase flows simulations" (arXiv
 * 1905.03917).
 *
 * Two stiffened-gas fluids share a uniform Cartesian grid: fluid N fills
 * phi < 0, fluid P fills phi >= 0 (phi the level set of Sec. 2.3).  Each
 * fluid k carries its conservative cut-cell variables (alpha U)_k of
 * Eq. 2 -- mass, x-momentum, y-momentum, total energy -- and is advanced
 * by the cut-cell finite-volume update of Eq. 2 with WENO5 Lax-Friedrichs
 * face fluxes weighted by face apertures, plus the interface exchange flux
 * X from an exact two-material Riemann problem (Sec. 2.1).
 *
 * Conventions for every entry point:
 *  - return 0 on success or a negative SIF_E* code; no exception crosses
 *    the ABI; sif_last_error() gives a one-line reason;
 *  - host/device arrays are caller-owned, borrowed for the duration of the
 *    call only, and always copied; mem_kind tells which memory a pointer
 *    refers to (SIF_HOST or SIF_DEVICE, the latter on the context's device);
 *  - grid arrays are x-fastest (index i + j*nx); "planes" are stacked
 *    component after component (component m at offset m*nx*ny);
 *  - all device work is issued on the context's stream; calls that return
 *    results to the host (integrals, get_state with SIF_HOST, step calls
 *    that fill a sif_cycle_info) synchronise that stream;
 *  - non-physical states (rho <= 0 or p + p_inf <= 0 in a cell that holds
 *    the fluid) are never clipped: the step reports SIF_ENONPHYS.
 */
#ifndef SIF_H
#define SIF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIF_OK 0
#define SIF_EINVAL -1    /* bad argument or configuration */
#define SIF_ECUDA -2     /* a CUDA call failed (no device, out of memory, ...) */
#define SIF_ENONPHYS -3  /* rho <= 0 or p + p_inf <= 0 in a real cell */
#define SIF_ENOCONV -4   /* interface Riemann Newton iteration did not converge */
#define SIF_ETIMEOUT -5  /* a bounded device wait gave up */
#define SIF_ESTATE -6    /* call out of order (e.g. step before init) */

#define SIF_HOST 0
#define SIF_DEVICE 1

#define SIF_BC_REFLECT 0   /* slip wall: normal velocity odd, rest even */
#define SIF_BC_ZEROGRAD 1  /* zero-gradient outflow */
#define SIF_BC_PERIODIC 2  /* periodic (both sides of the axis) */

typedef struct sif_ctx sif_ctx;

/* Configuration (all lengths in the units of the initial data). */
typedef struct {
  int dim;               /* 1 or 2 (dim 1 requires ny == 1) */
  int nx, ny;            /* cells; nx >= 3 and, in 2D, ny >= 3 */
  double x0, y0;         /* lower-left corner of the domain */
  double dx, dy;         /* cell sizes */
  int bc[4];             /* SIF_BC_* for the -x, +x, -y, +y sides */
  double gamma[2];       /* stiffened gas p = (gamma-1) rho e - gamma p_inf; [0] = N, [1] = P */
  double pinf[2];
  double cfl;            /* CFL number, 0.6 in the paper (Sec. 4) */
  int rk_order;          /* 2 = TVD-RK2 (the paper, Sec. 3); 3 = SSP-RK3 (both methods; the
                            adjoint calls require 2) */
  double weno_eps;       /* WENO5 epsilon, 1e-6; at least 1e-20 */
  double mix_alpha;      /* small-cell mixing threshold, 0.5 */
  double ratio_threshold;/* time-step-ratio truncation threshold, 0.7 (Sec. 3.1) */
  int ext_iters;         /* extension Jacobi sweeps per interaction step, 10 */
  int reinit_iters;      /* reinitialisation sweeps per level-set step, 2 */
  double band;           /* narrow-band half-width in cells, 6 */
  int flux_correction;   /* 1 = interfacial flux correction on (Eq. 8-9); 0 for tests */
  int force_ratio_one;   /* test switch: run the multi-dt cycle with dt1 = dt2 */
  void *cuda_stream;     /* cudaStream_t to issue work on; NULL = a private stream of the
                            context, created blocking (ordered with the legacy default
                            stream; a stream capture needs a non-legacy stream) */
  int device;            /* CUDA device ordinal */
  int weno_char;         /* 0 = WENO5 on each conserved component (the paper's WENO-LF,
                            Sec. 4); 1 = on the characteristic fields of the face state
                            (the mean of the two adjacent cells' stencil states), mapped
                            back by the right eigenvectors.  The adjoint calls require 0. */
  double sigma;          /* surface tension coefficient (Eq. 10), >= 0; 0 = none.  The
                            interface Riemann problem then carries the pressure jump
                            p_N - p_P = sigma kappa, kappa = div(grad phi / |grad phi|)
                            (positive where fluid N is convex), and each fluid receives
                            the exchange flux of its own interface pressure (Eq. 11-12
                            follow from recording fluid 1's).  2D only has curvature;
                            the adjoint calls require 0. */
  double mu[2];          /* dynamic viscosities of fluids N and P (Eq. 3, 5), >= 0; 0 =
                            inviscid.  Face viscous fluxes by central differences of the
                            stencil states times the apertures; each fluid's viscous
                            traction on its interface boundary through S; the explicit
                            viscous limit 2 nu (1/dx^2 + 1/dy^2) joins the CFL rate.  The
                            adjoint calls require 0. */
  int tait[2];           /* 1 = fluid k follows Tait's equation (Eq. 4, the weakly
                            compressible model's closure, Sec. 2.2): p = tait_B ((rho /
                            tait_rho0)^gamma - 1) + tait_p0, the pressure a function of
                            the density alone (the energy component is carried but does
                            not enter it); the interface Riemann problem takes such a
                            side's shock from mass and momentum alone.  pinf[k] is then
                            ignored: the sound speed is c^2 = gamma (p + tait_B - tait_p0)
                            / rho.  0 = stiffened gas.  Requires weno_char 0; the adjoint
                            calls require 0. */
  double tait_B[2], tait_rho0[2], tait_p0[2];  /* > 0, > 0, finite */
  int flux;              /* face flux of the finite-volume stage (Eq. 2): 0 = WENO5 on
                            Lax-Friedrichs split fluxes, per conserved component or field
                            (the paper's WENO-LF); 1 = HLLC (Toro's contact-restoring
                            approximate Riemann solver, Davis wave-speed bounds) between
                            WENO5 reconstructions of the primitive state (rho, u, v, p)
                            from either side, a reconstruction with rho <= 0 or
                            p + pinf <= 0 replaced by its cell's state.  1 requires
                            weno_char 0; the adjoint calls require 0. */
} sif_config;

/* Per-cycle record of the multi-time-step schedule (Sec. 3.1). */
typedef struct {
  double t;          /* time after the call */
  double dt1, dt2;   /* step of fluid 1 (larger) and first step of fluid 2 */
  double n_raw;      /* dt1/dt2 before truncation */
  double n_used;     /* ratio after the 0.7 truncation (1 = single step) */
  int role_fluid1;   /* 0 = N, 1 = P, -1 for single-dt steps */
  int substeps;      /* fluid-2 sub-steps in the last cycle */
  long long cell_updates; /* (cell, fluid) RK stage updates computed by the call's
                             finite-volume stages (every cell of a fluid's active
                             tiles, see sif_set_tile_shape) */
  long long open_updates; /* of those, the (cell, fluid) pairs with at least one
                             face open to the fluid (aperture A_k > 0, Eq. 2): the
                             cells whose update Eq. 2 computes.  open_updates /
                             rk_order is the call's work in fluid cell-updates
                             (RK steps), independent of the tile shape */
} sif_cycle_info;

/* Create a context on cfg->device; allocates all device memory it needs.
 * Errors: SIF_EINVAL for a bad configuration, SIF_ECUDA on allocation
 * failure (nothing is leaked; *out is set to NULL). */
int sif_create(const sif_config *cfg, sif_ctx **out);

/* Initial data (Sec. 2.3, Eq. 2): level set phi (nx*ny, a signed distance)
 * and the primitive fields of both fluids over the whole grid, prim_k =
 * 4 planes (rho, u, v, p).  Computes the geometry, sets (alpha U)_k =
 * alpha_k U(prim_k), mixes small cells and resets t = 0. */
int sif_init_fluids(sif_ctx *ctx, const double *phi, const double *prim_N,
                    const double *prim_P, int mem_kind);

/* nsteps steps of the original single-time-step method (Sec. 3.1, "the
 * original method"): both fluids and the level set advance with the
 * smaller CFL step; t_end > 0 caps the final time.  info (nullable) gets
 * the last step's record and the call's cell-update count. */
int sif_step_single_dt(sif_ctx *ctx, int nsteps, double t_end, sif_cycle_info *info);

/* ncycles cycles of the accelerated method (Sec. 3.1 steps 1-5): the fluid
 * with the larger CFL step (fluid 1) takes one RK step of dt1 while the
 * other sub-cycles against Eq. 7 interpolated states, with the Eq. 8-9
 * correction applied to fluid 1 at the end of the cycle.  With rk_order 3
 * (SSP-RK3, the paper's scheme carried to three stages): fluid 1's second
 * stage shares the last sub-step's evaluation at t1, its third stage is
 * evaluated at t^n + dt1/2 on the level set interpolated between the two
 * sub-step boundaries around that time, and the correction quantities
 * take RK3's stage weights 1/6, 1/6, 2/3; that third evaluation carries no
 * exchange flux, which the correction would remove from fluid 1 anyway. */
int sif_step_multi_dt(sif_ctx *ctx, int ncycles, double t_end, sif_cycle_info *info);

/* out[k*4+m] = sum over cells of (alpha U)_{k,m} dx dy (k = N, P; m = mass,
 * x-mom, y-mom, energy), reduced on the device in a fixed order.  Host
 * pointer; synchronises. */
int sif_integrals(sif_ctx *ctx, double *out);

/* Copy out the state: q_N, q_P as 4 planes each, phi as one plane; any
 * pointer may be NULL. */
int sif_get_state(sif_ctx *ctx, double *q_N, double *q_P, double *phi, int mem_kind);

/* Replace the state (checkpoint restore); geometry is recomputed, nothing
 * is mixed.  t is set to the given time. */
int sif_set_state(sif_ctx *ctx, const double *q_N, const double *q_P,
                  const double *phi, double t, int mem_kind);

/* Current simulation time. */
int sif_get_time(sif_ctx *ctx, double *t);

/* Checkpoint: serialise everything a bitwise-identical continuation needs
 * -- (alpha U) of both fluids, phi, the stencil states of both fluids
 * (the extension of Sec. 2.3 warm-starts from them) and t -- into a
 * caller-owned host buffer.  With buf == NULL only *len is set to the
 * size needed.  Errors: SIF_EINVAL if *len is too small. Synchronises. */
int sif_save(sif_ctx *ctx, void *buf, size_t *len);

/* Restore a checkpoint written by sif_save for the same grid size;
 * SIF_EINVAL if the buffer does not match. */
int sif_load(sif_ctx *ctx, const void *buf, size_t len);

/* Tile shape (output cells per CTA) of the finite-volume kernel: one of
 * 32x8 (default), 32x4, 16x8, 16x16, 64x4.  Results do not depend on it;
 * the autotuner (paper_1905_03917_gb300/autotune.py) picks the fastest
 * per grid-size bucket.  SIF_EINVAL for other shapes.  Synchronises. */
int sif_set_tile_shape(sif_ctx *ctx, int tx, int ty);
int sif_get_tile_shape(const sif_ctx *ctx, int *tx, int *ty);

/* Limits of the two bounded loops of a step (no counterpart in the paper,
 * whose method has no iteration limits): max_substeps, the fluid-2
 * sub-steps one accelerated cycle may take (default 4096; Sec. 3.1's
 * sub-cycle loop), and newton_iters, the Newton iterations of each
 * interface Riemann problem (default 50).  A cycle that reaches
 * max_substeps before its last sub-step stops with SIF_ETIMEOUT and leaves
 * the state undefined (restore a checkpoint); a Riemann problem that has
 * not converged after newton_iters iterations makes the step return
 * SIF_ENOCONV.  A value <= 0 keeps that limit; SIF_EINVAL above 1000000
 * sub-steps or 10000 iterations.  The captured graphs are rebuilt on the
 * next step.  Synchronises. */
int sif_set_limits(sif_ctx *ctx, int max_substeps, int newton_iters);

/* ---------------------------------------------------------------------
 * Batches of independent problems (uneven grid sizes) advanced together:
 * every instance's accelerated cycle is one device-driven CUDA graph
 * (conditional nodes follow each instance's own schedule), and a batch
 * cycle launches all of them as parallel branches of one graph.  Each
 * instance is an ordinary context (sif_batch_instance) for initial data,
 * state access, tile shape and integrals. */
typedef struct sif_batch sif_batch;

/* n contexts from cfgs[0..n-1] (their cuda_stream fields are ignored: the
 * batch owns its streams).  SIF_EINVAL / SIF_ECUDA as for sif_create. */
int sif_batch_create(int n, const sif_config *cfgs, sif_batch **out);

/* The i-th instance's context (owned by the batch: do not destroy). */
int sif_batch_instance(sif_batch *b, int i, sif_ctx **out);

/* ncycles accelerated cycles of every instance (each at its own time
 * step and sub-step count).  *cell_updates and *open_updates (nullable)
 * receive the sums over all instances of sif_cycle_info's counters of the
 * same names.  Every instance must have
 * been initialised.  Synchronises at the end; the first error of any
 * instance is returned (sif_batch_last_error names the instance). */
int sif_batch_step_multi_dt(sif_batch *b, int ncycles, long long *cell_updates,
                            long long *open_updates);

const char *sif_batch_last_error(const sif_batch *b);

/* 1 if the last batch step ran as one graph launch per batch cycle, 0 if
 * it fell back to one graph launch per instance and cycle. */
int sif_batch_one_graph(const sif_batch *b);
void sif_batch_destroy(sif_batch *b);

/* ---------------------------------------------------------------------
 * Discrete adjoint of the single-time-step method (rk_order 2) with each
 * step's schedule frozen.  The paper defines the forward step only
 * (Eq. 2 with the interface exchange of Sec. 2.1, mixing of Sec. 2.2,
 * extension of Sec. 2.3, TVD-RK2 of Sec. 4); the frozen step takes that
 * step's dt, its Lax-Friedrichs speeds of both stages and its level sets
 * after stage 1 and after the step as given, so that the geometry
 * (volume fractions, apertures, interface vectors, extension and mixing
 * targets and weights) is fixed and the step is a differentiable map of
 * the conserved states; the adjoint applies the transpose of its
 * Jacobian (WENO5 weights, LF splitting, the interface Riemann problem by
 * the implicit-function theorem, the aperture-weighted update, mixing,
 * extension, primitive recovery).
 *
 * Adjoint and state arrays in these calls are 8 planes of nx*ny doubles,
 * x fastest: the 4 components (mass, x-momentum, y-momentum, energy) of
 * (alpha U)_N, then those of (alpha U)_P.  mem_kind says whether the
 * caller's pointers are host or device memory; the context only reads
 * and writes them during the call. */

/* Start recording: every later sif_step_single_dt step (up to capacity in
 * total) records what its frozen replay needs (state, stencil states, level
 * sets, dt, LF speeds, both stages' stencil states and cut-cell flags:
 * 36 planes and 9 scalars per step, device memory
 * owned by the context).  Resets the tape to length 0.  capacity 0 stops
 * recording and frees the tape.  While recording, steps run without the
 * captured graphs (same kernels, same results) and sif_step_multi_dt
 * returns SIF_ESTATE.  SIF_EINVAL for rk_order != 2, weno_char != 0,
 * sigma != 0, mu != 0 or capacity < 0;
 * SIF_ECUDA if the tape cannot be allocated.  A step beyond capacity fails
 * with SIF_EINVAL before anything runs. */
int sif_tape_reset(sif_ctx *ctx, int capacity);
/* Number of steps recorded since the last sif_tape_reset. */
int sif_tape_length(const sif_ctx *ctx, int *len);

/* Frozen replay of recorded step `step` (0-based) from the state q_in,
 * written to q_out (may alias q_in).  From the recorded state it
 * reproduces the recorded step bitwise.  The context's own state is left
 * unchanged.  SIF_EINVAL for a step not on the tape; SIF_ENONPHYS if the
 * replayed state is non-physical in a real cell. */
int sif_replay_step(sif_ctx *ctx, int step, const double *q_in, double *q_out, int mem_kind);

/* lam_out = J^T lam_in with J the Jacobian of the frozen replay of
 * recorded step `step` at its recorded state: lam_in is the adjoint of
 * the state after the step, lam_out that of the state before it (may
 * alias lam_in).  The context's own state is left unchanged.
 * SIF_EINVAL for a step not on the tape or bad pointers. */
int sif_adjoint_step(sif_ctx *ctx, int step, const double *lam_in, double *lam_out,
                     int mem_kind);

/* Transpose of sif_init_fluids (conversion to (alpha U) and mixing, with
 * the geometry of phi) with respect to the primitive fields: lam_q (8
 * planes, adjoint of the initial state) -> lam_prim (8 planes: rho, u, v,
 * p of fluid N, then of fluid P).  phi, prim_N, prim_P as given to
 * sif_init_fluids.  The context's own state is left unchanged. */
int sif_adjoint_init(sif_ctx *ctx, const double *phi, const double *prim_N,
                     const double *prim_P, const double *lam_q, double *lam_prim,
                     int mem_kind);

/* Measurement counters of one context (no counterpart in the paper). */
typedef struct {
  long long kernel_launches;  /* libsif kernels launched on this context */
  long long fv_launches;      /* cut-cell finite-volume stage launches among them */
  double fv_ms;               /* summed CUDA-event time of those launches */
  long long fv_cell_updates;  /* (cell, fluid) stage updates they performed */
  long long fv_open_updates;  /* of those, cells with a face open to the fluid */
} sif_profile;

/* enable != 0 resets the counters and starts recording a pair of CUDA
 * events around every finite-volume stage launch on the context's stream
 * (at most 65536 pairs; later launches are counted but not timed);
 * enable == 0 stops recording. */
int sif_profile_enable(sif_ctx *ctx, int enable);

/* Read the counters (synchronises the stream to resolve the events). */
int sif_profile_read(sif_ctx *ctx, sif_profile *out);

/* FP64 fused multiply-add throughput of `device` in TFLOP/s (2 flops per
 * FMA), measured with independent FMA chains on every SM for a few tens of
 * milliseconds: the ceiling of the FP64-bound finite-volume kernel.  No
 * counterpart in the paper.  Allocates a small scratch buffer. */
int sif_measure_fp64_peak(int device, double *tflops);

/* The reciprocal the finite-volume kernel uses for its WENO5 face values
 * (one per face and component, Eq. 2's numerical flux): r[i] = 1 / d[i]
 * by Newton's iteration to third order from the device's approximate
 * reciprocal, within 1 ulp of the correctly rounded value.  d and r are
 * device pointers to n doubles (n >= 0; r may equal d); d[i] must be
 * positive, normal and below 2^1000, other inputs give unspecified values
 * (the kernel divides instead outside that range).  Launched on `stream`
 * (a cudaStream_t, NULL = default) and not synchronised.  SIF_EINVAL for
 * n < 0 or a null pointer with n > 0, SIF_ECUDA for a launch failure.  No
 * counterpart in the paper: it exists so that tests can hold the kernel's
 * arithmetic to IEEE division. */
int sif_probe_reciprocal(const double *d, double *r, long long n, void *stream);

/* Conserved totals of caller-provided device planes without allocating
 * anything -- for callers that cannot allocate device memory when they
 * need the totals (e.g. a host framework whose caching allocator already
 * holds the GPU's free memory, or a hook inside a time-stepping loop where
 * an allocation would synchronise the device).  The paper has no
 * counterpart; this is a variant of the reduction behind sif_integrals.
 *   q_N, q_P: device pointers, 4 planes (mass, x-mom, y-mom, energy) of
 *             nx*ny doubles each, x fastest, no ghost cells (the layout
 *             sif_get_state writes);
 *   out:      device pointer to 8 doubles, out[k*4+m] = sum q_k,m dx dy;
 *   stream:   cudaStream_t (NULL = legacy default stream); asynchronous.
 * Scratch: a 1 MiB file-scope device array holds the row partial sums, so
 * ny may not exceed 16384 (SIF_EINVAL beyond that, or for nx, ny < 1).
 * Every GPU that loads the library keeps that array until the process
 * exits.  The call works on the current device: q_N, q_P and out must
 * live there.  The first call on a device looks up the array's device
 * address with that device current and caches it; make that first call
 * before any stream capture.  The cached address is not valid after a
 * cudaDeviceReset (which unloads the module); first calls on one device
 * from several host threads at once are safe (they store the same
 * address).  Each GPU has its own copy of the array: calls that overlap
 * on the same GPU (on any streams) race on it and must be ordered by the
 * caller; calls on different GPUs share nothing.  Each call overwrites
 * every partial sum it reads, so nothing needs clearing between calls.
 * Calls no cudaMalloc/cudaFree. */
int sif_integrals_noalloc(const double *q_N, const double *q_P, int nx, int ny, double dx,
                          double dy, double *out, void *stream);

/* One-line description of the last error on this context (never NULL). */
const char *sif_last_error(const sif_ctx *ctx);

/* Free all device memory of the context. NULL is ignored. */
void sif_destroy(sif_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
