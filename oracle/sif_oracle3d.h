/*
 * sif_oracle3d.h -- serial FP64 CPU oracle of the three-dimensional form of
 * the conservative sharp-interface method with multi-time-step sub-cycling
 * (Long, Cai & Pan, arXiv 1905.03917; the 3D rows of Tables 1, 3 and 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests and the CPU-baseline leg of
 * bench.py may load it.  It shares no code with the CUDA library.  It uses
 * the two-dimensional oracle's pointwise routines (WENO5, the two-material
 * Riemann problem, the square's area fraction), which are pinned there.
 *
 * Scope: stiffened-gas or Tait fluids (Eq. 1, 4) with or without surface
 * tension (Eq. 10) and viscosity (Eq. 3, 5), component-wise WENO5 on
 * Lax-Friedrichs split fluxes, TVD-RK2, the single-time-step step and the accelerated cycle of
 * Sec. 3.1 (Eq. 7-9).
 */
#ifndef SIF_ORACLE3D_H
#define SIF_ORACLE3D_H

#include "sif_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;
  double x0, y0, z0, dx, dy, dz;
  int bc[6];          /* ORC_BC_* for -x, +x, -y, +y, -z, +z */
  double gamma[2];    /* [0] fluid N (phi < 0), [1] fluid P */
  double pinf[2];
  double cfl;
  double weno_eps;
  double mix_alpha;
  double ratio_threshold;
  int ext_iters;
  int reinit_iters;
  double band;        /* narrow band half-width in cells */
  int flux_correction;
  int force_ratio_one;
  int tait[2];        /* Tait's equation for fluid k (Eq. 4) */
  double tait_B[2], tait_rho0[2], tait_p0[2];
  double sigma;       /* surface tension coefficient (Eq. 10); 0 = none */
  double mu[2];       /* dynamic viscosities of fluids N and P (Eq. 3, 5); 0 = inviscid */
} orc3_config;

typedef struct orc3_ctx orc3_ctx;

orc3_ctx *orc3_create(const orc3_config *cfg);
void orc3_destroy(orc3_ctx *o);
/* phi: nx*ny*nz, x fastest then y then z; prim_N / prim_P: 5 such planes
 * (rho, u, v, w, p). */
int orc3_init(orc3_ctx *o, const double *phi, const double *prim_N, const double *prim_P);
int orc3_step_single_dt(orc3_ctx *o, int nsteps, double t_end, orc_info *info);
int orc3_step_multi_dt(orc3_ctx *o, int ncycles, double t_end, orc_info *info);
/* q_N / q_P: 5 planes of (alpha U) per fluid; phi: one plane. Any may be NULL. */
int orc3_get_state(const orc3_ctx *o, double *qN, double *qP, double *phi);
int orc3_set_state(orc3_ctx *o, const double *qN, const double *qP, const double *phi);
/* out[10]: volume integrals of (alpha U)_k, k = N then P, 5 components each */
int orc3_integrals(const orc3_ctx *o, double *out);
/* geometry of the current level set: alpha_P, P-apertures of the lower x,
 * y and z faces of every cell, and the interface vector S (N to P); each
 * nx*ny*nz (the faces at the upper domain ends are not returned) */
int orc3_geometry(orc3_ctx *o, double *alpha, double *ax, double *ay, double *az,
                  double *sx, double *sy, double *sz);
/* volume fraction and interface vector of one unit cube from its eight
 * corner values c[i + 2 j + 4 k] (i, j, k in {0, 1} along x, y, z);
 * s[3] in unit-face areas; returns alpha_P */
double orc3_cell_alpha(const double *c, double *s);
/* curvature div(grad phi / |grad phi|) of the current level set at cell
 * (i, j, k), second-order central differences */
double orc3_curvature(orc3_ctx *o, int i, int j, int k);
double orc3_time(const orc3_ctx *o);
int orc3_status(const orc3_ctx *o);

#ifdef __cplusplus
}
#endif
#endif
