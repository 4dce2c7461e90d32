/*
 * sif3d.h -- C-ABI of the three-dimensional solver in libsif (sm_103a,
 * FP64): the conservative sharp-interface method with multi-time-step
 * sub-cycling of Long, Cai & Pan (arXiv 1905.03917) on a uniform grid of
 * cubes, the paper's "Uniform grid - 3D" rows (Tables 1, 3, 4).
 *
 * The method is the two-dimensional one with a third pair of faces: Eq. 2
 * sums six aperture-weighted WENO5 Lax-Friedrichs face fluxes per cut cell
 * plus the interface exchange X (Sec. 2.1); the level set moves by Eq. 6
 * and is reinitialised (Sec. 2.3); the accelerated cycle is Sec. 3.1's
 * steps 1-5 with Eq. 7 interpolation and the Eq. 8-9 correction.  The
 * cut-cell geometry of a cube: corner values are the mean of the eight
 * cells sharing the corner, each face's aperture is the area fraction of
 * the polygon through its positive corners and edge crossings, S_d = (A_d+
 * - A_d-) times the face area, and alpha follows from the divergence
 * theorem with the interface patch planar through the mean of its edge
 * crossings.  Small cells mix into up to seven neighbours toward their
 * fluid (x, y, z, the face and cube diagonals) weighted n_x^2, n_y^2,
 * n_z^2, |n_x n_y|, |n_x n_z|, |n_y n_z|, |n_x n_y n_z|^(2/3).
 *
 * Scope: stiffened-gas or Tait fluids (Eq. 1, 4) with or without surface
 * tension (Eq. 10) and viscosity (Eq. 3, 5), component-wise WENO5 on
 * Lax-Friedrichs split fluxes, TVD-RK2.  The other options of the 2D solver
 * (characteristic WENO5, HLLC, RK3, adjoint) are not available in 3D.
 *
 * Conventions are those of sif.h: 0 or a negative SIF_E* code, the reason
 * from sif3_last_error(); arrays are caller-owned and copied; mem_kind is
 * SIF_HOST or SIF_DEVICE; grid arrays are (nz, ny, nx) with x fastest,
 * "planes" stacked component after component (component m at offset
 * m*nx*ny*nz).  Every call that returns a result or a cycle record
 * synchronises the context's stream; the cycle's control (time steps, the
 * sub-step loop) is taken on the host from device-reduced maxima.
 */
#ifndef SIF3D_H
#define SIF3D_H

#include "sif.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sif3_ctx sif3_ctx;

typedef struct {
  int nx, ny, nz;        /* cells, each >= 3; (nx+6)(ny+6)(nz+6) < 2^31 */
  double x0, y0, z0;     /* lower corner of the domain */
  double dx, dy, dz;     /* cell sizes */
  int bc[6];             /* SIF_BC_* for the -x, +x, -y, +y, -z, +z sides */
  double gamma[2];       /* [0] fluid N (phi < 0), [1] fluid P */
  double pinf[2];        /* stiffened gas p_inf (ignored for a Tait fluid) */
  double cfl;            /* CFL number (Sec. 4: 0.6); the rate sums over three directions */
  double weno_eps;       /* WENO5 epsilon, 1e-6 */
  double mix_alpha;      /* small-cell mixing threshold, 0.5 */
  double ratio_threshold;/* time-step-ratio truncation threshold, 0.7 (Sec. 3.1) */
  int ext_iters;         /* extension Jacobi sweeps, 10 */
  int reinit_iters;      /* reinitialisation sweeps per level-set step, 2 */
  double band;           /* narrow-band half-width in cells, 6 */
  int flux_correction;   /* 1 = Eq. 8-9 correction on */
  int force_ratio_one;   /* test switch: multi-dt cycle with dt1 = dt2 */
  int tait[2];           /* 1 = Tait's equation (Eq. 4) for fluid k, as in sif_config */
  double tait_B[2], tait_rho0[2], tait_p0[2];
  void *cuda_stream;     /* cudaStream_t for all work; NULL = a private blocking stream */
  int device;            /* CUDA device ordinal */
  double sigma;          /* surface tension coefficient (Eq. 10), >= 0; 0 = none.  The
                            interface Riemann problem carries the jump p_N - p_P =
                            sigma kappa, kappa = div(grad phi / |grad phi|) by central
                            differences (2 / r for a sphere), and each fluid receives
                            the exchange flux of its own interface pressure */
  double mu[2];          /* dynamic viscosities of fluids N and P (Eq. 3, 5), >= 0; 0 =
                            inviscid.  Face viscous fluxes by central differences of the
                            stencil states times the apertures; with both fluids viscous
                            the traction of the velocity field that is continuous across
                            the interface (harmonic-mean viscosity) joins the exchange
                            flux; the explicit limit 2 nu (1/dx^2 + 1/dy^2 + 1/dz^2) joins
                            the CFL rate */
} sif3_config;

/* Create a context; allocates its device memory (about 110 planes of
 * (nx+6)(ny+6)(nz+6) doubles).  SIF_EINVAL for a bad configuration,
 * SIF_ECUDA when allocation fails (nothing leaked, *out = NULL). */
int sif3_create(const sif3_config *cfg, sif3_ctx **out);

/* Initial data: phi (one plane, a signed distance), prim_N / prim_P five
 * planes each (rho, u, v, w, p); the conservative states alpha_k U_k are
 * formed and small cells mixed (Sec. 2.2), t = 0. */
int sif3_init_fluids(sif3_ctx *ctx, const double *phi, const double *prim_N,
                     const double *prim_P, int mem_kind);

/* nsteps steps of the single-time-step method (the paper's original
 * method: both fluids and the level set advance with min_k dt_k), each
 * cut to end at t_end when t_end > 0.  SIF_ENONPHYS / SIF_ENOCONV as in
 * sif.h; info (may be NULL) describes the last step and counts the call's
 * finite-volume updates. */
int sif3_step_single_dt(sif3_ctx *ctx, int nsteps, double t_end, sif_cycle_info *info);

/* ncycles accelerated cycles (Sec. 3.1): fluid 1 (the larger stable step)
 * takes one RK2 step of dt1 = n dt2 while fluid 2 and the level set
 * sub-cycle, fluid 1 seen through Eq. 7, corrected by Eq. 8-9 at the end.
 * The sub-step loop stops with SIF_ETIMEOUT after 4096 sub-steps. */
int sif3_step_multi_dt(sif3_ctx *ctx, int ncycles, double t_end, sif_cycle_info *info);

/* State out / in: q_N, q_P five planes of alpha U each (mass, x-, y-,
 * z-momentum, energy), phi one plane; any may be NULL.  set_state
 * recomputes the geometry from phi and clears the error bits a failed step
 * left. */
int sif3_get_state(sif3_ctx *ctx, double *qN, double *qP, double *phi, int mem_kind);
int sif3_set_state(sif3_ctx *ctx, const double *qN, const double *qP, const double *phi,
                   int mem_kind);

/* out[10] (host): volume integrals of alpha U for fluid N then P, five
 * components each. */
int sif3_integrals(sif3_ctx *ctx, double *out);

/* Geometry of the current level set: alpha_P, the P-apertures of the lower
 * x, y and z faces of every cell and S (N to P); each one plane, any may be
 * NULL. */
int sif3_geometry(sif3_ctx *ctx, double *alpha, double *ax, double *ay, double *az,
                  double *sx, double *sy, double *sz, int mem_kind);

int sif3_get_time(const sif3_ctx *ctx, double *t);

/* Limits of the two bounded loops of a step, as sif_set_limits (no
 * counterpart in the paper): max_substeps, the fluid-2 sub-steps one
 * accelerated cycle may take (default 4096), and newton_iters, the Newton
 * iterations of each interface Riemann problem (default 50).  A cycle that
 * reaches max_substeps before its last sub-step stops with SIF_ETIMEOUT and
 * leaves the state undefined (restore it with sif3_set_state); a Riemann
 * problem not converged after newton_iters iterations makes the step return
 * SIF_ENOCONV.  A value <= 0 keeps that limit; SIF_EINVAL above 1000000
 * sub-steps or 10000 iterations. */
int sif3_set_limits(sif3_ctx *ctx, int max_substeps, int newton_iters);

/* Kernel timing of the finite-volume stages (the dominant kernel): while
 * enabled every launch is bracketed by events on the context's stream and
 * its duration summed; sif3_profile_read returns and clears the totals
 * (launches, milliseconds, computed and open (cell, fluid) stage updates). */
int sif3_profile_enable(sif3_ctx *ctx, int on);
int sif3_profile_read(sif3_ctx *ctx, sif_profile *out);

const char *sif3_last_error(const sif3_ctx *ctx);
int sif3_destroy(sif3_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
