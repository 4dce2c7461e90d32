/*
 * sif_oracle.h -- serial FP64 CPU oracle of the conservative sharp-interface
 * method with multi-time-step sub-cycling (Long, Cai & Pan, arXiv 1905.03917).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA library: every formula here is
 * written out plainly, loop by loop, in the order the paper states it.
 *
 * Parity status per function is listed in the header comment of
 * sif_oracle.c.
 */
#ifndef SIF_ORACLE_H
#define SIF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary kinds for the four domain sides (-x, +x, -y, +y). */
#define ORC_BC_REFLECT 0
#define ORC_BC_ZEROGRAD 1
#define ORC_BC_PERIODIC 2

/* Sticky error bits reported by orc_status(). */
#define ORC_ERR_NONPHYS 1  /* rho <= 0 or p + p_inf <= 0 in a real cell */
#define ORC_ERR_NOCONV 2   /* interface Riemann Newton did not converge */
#define ORC_ERR_INVAL 4    /* unsupported configuration */

typedef struct {
  int dim;            /* 1 or 2; dim 1 requires ny == 1 */
  int nx, ny;
  double x0, y0, dx, dy;
  int bc[4];          /* ORC_BC_* for -x, +x, -y, +y */
  double gamma[2];    /* stiffened gas: [0] fluid N (phi < 0), [1] fluid P */
  double pinf[2];
  double cfl;         /* 0.6 */
  int rk_order;       /* 2 (paper) or 3 (SSP-RK3; its multi-dt cycle is cycle_rk3) */
  double weno_eps;    /* 1e-6 */
  double mix_alpha;   /* small-cell threshold, 0.5 */
  double ratio_threshold; /* n truncation threshold, 0.7 */
  int ext_iters;      /* extension Jacobi sweeps, 10 */
  int reinit_iters;   /* reinitialisation sweeps per level-set step, 2 */
  double band;        /* narrow band half-width in cells, 6 */
  int flux_correction;   /* 1 = interfacial flux correction on */
  int force_ratio_one;   /* test only: multi-dt cycle with dt1 = dt2 */
  int weno_char;         /* 1 = WENO5 on characteristic fields, 0 = component-wise */
  double sigma;          /* surface tension coefficient (Eq. 10); 0 = none */
  double mu[2];          /* dynamic viscosities of fluids N and P (Eq. 3, 5); 0 = inviscid */
  /* Tait's equation (Eq. 4) for fluid k when tait[k] = 1: p = B ((rho /
   * rho0)^gamma - 1) + p0, the pressure a function of the density alone
   * (the energy component is carried but does not enter it); pinf[k] is
   * then B - p0, which gives the sound speed c^2 = gamma (p + pinf) / rho */
  int tait[2];
  double tait_B[2], tait_rho0[2], tait_p0[2];
  /* face flux: 0 = WENO5 on Lax-Friedrichs split fluxes (the paper's),
   * 1 = HLLC (Toro's contact-restoring approximate Riemann solver) between
   * WENO5 reconstructions of the primitive state from either side
   * (requires weno_char 0) */
  int flux;
} orc_config;

typedef struct {
  double t, dt1, dt2, n_raw, n_used;
  int role_fluid1; /* index (0 = N, 1 = P) of the fluid with the larger step */
  int substeps;    /* fluid-2 sub-steps taken in the last cycle */
  int err;
  long long open_updates; /* (cell, fluid) finite-volume stage updates of the call
                             in cells with a face open to the fluid */
} orc_info;

typedef struct orc_ctx orc_ctx;

orc_ctx *orc_create(const orc_config *cfg);
void orc_destroy(orc_ctx *o);
/* phi: nx*ny; prim_N / prim_P: 4 planes (rho, u, v, p) of nx*ny, x fastest. */
int orc_init(orc_ctx *o, const double *phi, const double *prim_N, const double *prim_P);
int orc_step_single_dt(orc_ctx *o, int nsteps, double t_end, orc_info *info);
int orc_step_multi_dt(orc_ctx *o, int ncycles, double t_end, orc_info *info);
/* q_N / q_P: 4 planes of (alpha U) per fluid; phi: nx*ny. Any may be NULL. */
int orc_get_state(const orc_ctx *o, double *q_N, double *q_P, double *phi);
int orc_set_state(orc_ctx *o, const double *q_N, const double *q_P, const double *phi);
/* out[k*4+m] = sum over cells of (alpha U)_k,m dx dy. */
int orc_integrals(const orc_ctx *o, double *out);
double orc_time(const orc_ctx *o);
int orc_status(const orc_ctx *o);

/* HLLC flux through a face of direction d (0 = x, 1 = y) between the
 * primitive states WL and WR (rho, u, v, p) of one stiffened gas (gamma,
 * pinf): Davis's wave-speed bounds S_L = min(un_L - c_L, un_R - c_R),
 * S_R = max(un_L + c_L, un_R + c_R), the contact speed S* from the
 * momentum balance across the two outer waves, and the flux of the state
 * region the face lies in.  F = flux of (rho, rho u, rho v, E).  Returns
 * ORC_ERR_INVAL for a non-physical state. */
int orc_hllc(const double *WL, const double *WR, double gamma, double pinf, int d, double *F);

/* Geometry of the current level set: alpha_P, x-face and y-face P-apertures
 * (left/bottom face of each cell, nx+1 by ny and nx by ny+1 arrays), and
 * the interface vector S (N to P) per cell. Any output may be NULL. */
int orc_geometry(orc_ctx *o, double *alpha, double *ax, double *ay,
                 double *sx, double *sy);
/* Exact two-material Riemann problem with a pressure jump across the
 * contact: the left star pressure exceeds the right one by jump (surface
 * tension, Eq. 10).  L, R = (rho, u, p, gamma, pinf).  out = right star
 * pressure, star velocity, left and right star densities and sound
 * speeds, Newton iterations, left star pressure.  Returns ORC_ERR_NOCONV if
 * Newton does not converge in 50 iterations. */
int orc_riemann_jump(const double *L, const double *R, double jump, double *out);
/* The same with either side barotropic (baro_l, baro_r = 1: a fluid on the
 * curve p + pinf proportional to rho^gamma, Tait's equation): its shock
 * branch from mass and momentum alone, its star density on the curve. */
int orc_riemann_jump2(const double *L, const double *R, double jump, int baro_l, int baro_r,
                      double *out);
/* Curvature div(grad phi / |grad phi|) of the current level set at cell
 * (i, j) by central differences (0 in 1D or where grad phi = 0). */
double orc_curvature(orc_ctx *o, int i, int j);
/* Characteristic basis of the Euler flux Jacobian in direction d (0 = x,
 * 1 = y) at the primitive state (rho, u, v, p) of a stiffened gas (g, pinf):
 * R[m*4+f] = component m of the right eigenvector of field f (eigenvalues
 * un - c, un, un, un + c with un the velocity along d), L[f*4+m] = row f
 * of the inverse.  Returns ORC_ERR_INVAL for a non-physical state. */
int orc_char_basis(double g, double pinf, double rho, double u, double v, double p, int d,
                   double *L, double *R);
/* Right-hand side L_k of the cut-cell update (Eq. 2) for fluid k at the
 * current state, after the interaction step; out is 4 planes of nx*ny. */
int orc_rhs(orc_ctx *o, int k, double *out);
/* One reinitialisation pass (reinit_iters sweeps) on the current phi. */
int orc_reinit_only(orc_ctx *o);
/* Small-cell mixing of fluid k on the current state (in place). */
int orc_mix_only(orc_ctx *o, int k);
/* Extension: stencil states W_k (4 primitive planes) after extension. */
int orc_stencil_states(orc_ctx *o, int k, double *out);

/* Pointwise pieces for unit pins. */
double orc_weno5(const double *v, double eps);
double orc_edge_fraction(double a, double b);
double orc_cell_alpha(double c00, double c10, double c11, double c01);
/* Exact two-material stiffened-gas Riemann problem.
 * L/R: rho, u, p, gamma, pinf. out: p*, u*, rho*_L, rho*_R, c*_L, c*_R,
 * iterations. Returns 0, or ORC_ERR_NOCONV. */
int orc_riemann(const double *L, const double *R, double *out);

/* Discrete adjoint of the single-time-step RK2 step with its schedule
 * frozen (rk_order 2 only; ORC_ERR_INVAL otherwise).
 * orc_step_taped: one ordinary single-dt step that also returns its
 *   schedule: dt, the Lax-Friedrichs speeds lf[8] (index stage*4 + fluid*2
 *   + direction) and the level sets after stage 1 (phi1) and after the step
 *   (phi2), nx*ny each.
 * orc_replay_step: the same step from the current state with that schedule
 *   taken as given (the frozen map; bitwise equal to the taped step when
 *   started from the taped state).
 * orc_adjoint_step: lam_out = J^T lam_in for the frozen map J at the
 *   current state; lam_in / lam_out are 8 planes of nx*ny (fluid N
 *   components 0-3, then fluid P).  The context's state is unchanged. */
int orc_step_taped(orc_ctx *o, double *dt, double *lf, double *phi1, double *phi2);
int orc_replay_step(orc_ctx *o, double dt, const double *lf, const double *phi1,
                    const double *phi2);
int orc_adjoint_step(orc_ctx *o, double dt, const double *lf, const double *phi1,
                     const double *phi2, const double *lam_in, double *lam_out);
/* Stage-level pieces: both fluids' right-hand sides (8 planes) at the
 * current state with Lax-Friedrichs speeds lf[4] (fluid*2 + direction)
 * taken as given; the transpose of their Jacobian applied to mu (8
 * planes); the transpose of mixing fluid k (4 planes, in place). */
int orc_rhs_frozen(orc_ctx *o, const double *lf, double *out);
int orc_rhs_adjoint(orc_ctx *o, const double *lf, const double *mu, double *lq);
int orc_mix_adjoint(orc_ctx *o, int k, double *lam);
/* Transpose of orc_init with respect to the primitive fields, at the
 * current level set: lam_q (8 planes) -> lam_prim (8 planes, rho u v p of
 * fluid N then fluid P); prim_N / prim_P as given to orc_init. */
int orc_adjoint_init(orc_ctx *o, const double *prim_N, const double *prim_P,
                     const double *lam_q, double *lam_prim);
/* d weno5(v) / d v (5 values). */
void orc_weno5_grad(const double *v, double eps, double *g);
/* lam_p dp* + lam_u du* of the Riemann problem as a row vector over
 * (rho, u, p) of each side: gL[3], gR[3]. */
int orc_riemann_grad(const double *L, const double *R, double lam_p, double lam_u, double *gL,
                     double *gR);

#ifdef __cplusplus
}
#endif
#endif
