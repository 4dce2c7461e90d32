/*
 * sif_oracle.c -- plain, slow, serial FP64 oracle of the accelerated
 * conservative sharp-interface method (Long, Cai & Pan, arXiv 1905.03917).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and
 * the CPU-baseline leg of bench.py, never by the product path.  It shares
 * no code with the CUDA library.  Compile with -O2 -ffp-contract=off and no
 * fast-math so that every operation is rounded as written.
 *
 * What each part follows and what pins it (tests/test_oracle_*.py):
 *   edge fraction, cell volume fraction, apertures, interface vector
 *       -- Sec. 2.1 / Fig. 1 (cut cell with apertures and interface
 *          segment); pinned by exact half-plane areas and segment lengths
 *          and by circle areas.
 *   WENO5-JS reconstruction, Lax-Friedrichs splitting, TVD-RK2 / SSP-RK3
 *       -- Sec. 4 (WENO-LF, RK2, CFL 0.6); pinned by fifth-order
 *          convergence of the single-fluid operator and by the
 *          single-fluid reduction of Eq. 2.
 *   exact stiffened-gas Riemann problem (interface interaction)
 *       -- Sec. 2.1 (interface exchange flux X); pinned by textbook
 *          ideal-gas star states and by Rankine-Hugoniot / isentrope
 *          checks of the stiffened-gas solution.
 *   cut-cell update with X, mixing, extension -- Eq. 2, Sec. 2.1-2.3;
 *          pinned by the static-interface test, exact conservation and
 *          the 1D exact-solution convergence test.
 *   level-set advection (Eq. 6) and reinitialisation (Sec. 2.3) -- pinned
 *          by rigid translation of a circle and invariance of a planar
 *          signed distance under reinitialisation.
 *   multi-time-step cycle: time-step ratio and its truncation, fluid-1
 *          previous/future states, Eq. 7 interpolation, Eq. 8-9 correction
 *          quantities and the final correction -- Sec. 3.1 steps 1-5;
 *          pinned by exact conservation with the correction on (and its
 *          visible loss with it off) and by the bitwise ratio-one
 *          reduction to the single-step method.
 *   discrete adjoint of the frozen single-time-step RK2 step and of the
 *          initialisation (the transposes of every operation of the step
 *          with its schedule -- dt, Lax-Friedrichs speeds, level sets --
 *          taken as given) -- pinned by central differences of the
 *          pointwise pieces (WENO5 with its weights, the Riemann problem),
 *          a brute-force Jacobian of both right-hand sides on a 16 x 16
 *          bubble, exact transposition of the mixing, the conservation
 *          identities of the transposed step, and central differences of
 *          a wall-pressure functional over 20 replayed steps.
 * Parity unpinned (checked only against the GPU): the number of extension
 * and reinitialisation sweeps and the band width (the paper gives none).
 */
#include "sif_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define GH 3 /* ghost layers: the WENO5 stencil reaches three cells */
/* A cell counts as holding fluid k (its stencil state is (alpha U)/alpha
 * and it enters the CFL bound) only if alpha_k exceeds this; thinner
 * slivers, which round-off in the corner values creates, take extended
 * states like empty cells while their (alpha U) is still carried and
 * mixed. */
#define ALPHA_REAL 1e-6
/* (a cut cell whose content is not a physical state is treated the same
 * way: see is_real and prim) */

struct orc_ctx {
  orc_config c;
  int PX, PY, NP;
  double h; /* min(dx, dy) */
  double *q[2][4];  /* (alpha U)_k: mass, x-mom, y-mom, energy */
  double *w[2][4];  /* stencil states W_k: rho, u, v, p */
  double *phi;
  double *alpha, *ax, *ay, *sx, *sy; /* alpha_P, P-apertures, S (N to P) */
  double *xn[3];    /* interface exchange X as applied to fluid N */
  double *xp[3];    /* and to fluid P (-xn without surface tension) */
  double *ul[2];    /* level-set velocity */
  double smax[2];   /* CFL maxima per fluid (cells and star states) */
  double lf[2][2];  /* Lax-Friedrichs alpha per fluid and direction */
  double t;
  int err;
  /* (cell, fluid) pairs whose update had a face open to the fluid, summed
   * over the finite-volume stages: the work count of the throughput figure */
  long long open_updates;
  /* scratch */
  double *q0[2][4], *L[2][4], *old[4], *fx[4], *fy[4];
  double *prev[4], *fut[4], *qi[4], *xc[3];
  double *phi0, *lphi, *p0;
  /* RK3 cycle: the level set at the two sub-step boundaries around fluid
   * 1's third-stage time and at the end of the cycle */
  double *phia, *phib, *phie;
  unsigned char *band, *rext;
  /* per fluid: 1 where a small cell's content is not a physical state
   * (set by prim for the current stage) */
  unsigned char *nostate[2];
};

#define ID(o, i, j) ((i) + GH + ((j) + GH) * (o)->PX)

static double sq(double a) { return a * a; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* ------------------------------------------------------------------ */
/* ghost layers                                                        */

/* vel: 0 scalar, 1 x-velocity (odd at x walls), 2 y-velocity (odd at y
 * walls).  x ghosts are filled for interior rows, then y ghosts for every
 * column including the x ghosts. */
static void fill_ghost(orc_ctx *o, double *a, int vel) {
  int nx = o->c.nx, ny = o->c.ny;
  for (int j = 0; j < ny; j++) {
    for (int m = 0; m < GH; m++) {
      double sl = (vel == 1 && o->c.bc[0] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      double sr = (vel == 1 && o->c.bc[1] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      double vl, vr;
      switch (o->c.bc[0]) {
        case ORC_BC_REFLECT: vl = a[ID(o, m, j)]; break;
        case ORC_BC_PERIODIC: vl = a[ID(o, nx - 1 - m, j)]; break;
        default: vl = a[ID(o, 0, j)];
      }
      switch (o->c.bc[1]) {
        case ORC_BC_REFLECT: vr = a[ID(o, nx - 1 - m, j)]; break;
        case ORC_BC_PERIODIC: vr = a[ID(o, m, j)]; break;
        default: vr = a[ID(o, nx - 1, j)];
      }
      a[ID(o, -1 - m, j)] = sl < 0 ? -vl : vl;
      a[ID(o, nx + m, j)] = sr < 0 ? -vr : vr;
    }
  }
  for (int i = -GH; i < nx + GH; i++) {
    for (int m = 0; m < GH; m++) {
      double sb = (vel == 2 && o->c.bc[2] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      double st = (vel == 2 && o->c.bc[3] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      double vb, vt;
      switch (o->c.bc[2]) {
        case ORC_BC_REFLECT: vb = a[ID(o, i, m)]; break;
        case ORC_BC_PERIODIC: vb = a[ID(o, i, ny - 1 - m)]; break;
        default: vb = a[ID(o, i, 0)];
      }
      switch (o->c.bc[3]) {
        case ORC_BC_REFLECT: vt = a[ID(o, i, ny - 1 - m)]; break;
        case ORC_BC_PERIODIC: vt = a[ID(o, i, m)]; break;
        default: vt = a[ID(o, i, ny - 1)];
      }
      a[ID(o, i, -1 - m)] = sb < 0 ? -vb : vb;
      a[ID(o, i, ny + m)] = st < 0 ? -vt : vt;
    }
  }
}

/* ------------------------------------------------------------------ */
/* geometry from the level set (Sec. 2.1, Fig. 1)                      */

double orc_edge_fraction(double a, double b) {
  /* fraction of the straight edge from value a to value b with phi >= 0,
   * phi varying linearly along the edge */
  if (a >= 0.0 && b >= 0.0) return 1.0;
  if (a < 0.0 && b < 0.0) return 0.0;
  if (a >= 0.0) return a / (a - b);
  return b / (b - a);
}

double orc_cell_alpha(double c00, double c10, double c11, double c01) {
  /* area of {phi >= 0} in the unit cell, phi bilinear through the corner
   * values (counter-clockwise from the lower-left corner), approximated by
   * the polygon through the P corners and the edge crossings.  In the
   * saddle case the P corners are taken as disconnected triangles. */
  const double v[4] = {c00, c10, c11, c01};
  const double px[4] = {0.0, 1.0, 1.0, 0.0};
  const double py[4] = {0.0, 0.0, 1.0, 1.0};
  int npos = 0, changes = 0;
  for (int e = 0; e < 4; e++) {
    if (v[e] >= 0.0) npos++;
    if ((v[e] >= 0.0) != (v[(e + 1) & 3] >= 0.0)) changes++;
  }
  if (npos == 4) return 1.0;
  if (npos == 0) return 0.0;
  if (changes == 4) {
    double area = 0.0;
    for (int e = 0; e < 4; e++) {
      if (v[e] < 0.0) continue;
      int n = (e + 1) & 3, p = (e + 3) & 3;
      double l1 = v[e] / (v[e] - v[n]);
      double l2 = v[e] / (v[e] - v[p]);
      area += 0.5 * l1 * l2;
    }
    return area;
  }
  double X[8], Y[8];
  int m = 0;
  for (int e = 0; e < 4; e++) {
    int n = (e + 1) & 3;
    if (v[e] >= 0.0) {
      X[m] = px[e];
      Y[m] = py[e];
      m++;
    }
    if ((v[e] >= 0.0) != (v[n] >= 0.0)) {
      double s = v[e] / (v[e] - v[n]);
      X[m] = px[e] + s * (px[n] - px[e]);
      Y[m] = py[e] + s * (py[n] - py[e]);
      m++;
    }
  }
  double a2 = 0.0;
  for (int k = 0; k < m; k++) {
    int k1 = (k + 1) % m;
    a2 += X[k] * Y[k1] - X[k1] * Y[k];
  }
  return 0.5 * a2;
}

/* level set at the lower-left corner of cell (i, j): mean of the four
 * cells sharing that corner */
static double corner(const orc_ctx *o, const double *p, int i, int j) {
  return 0.25 * ((p[ID(o, i - 1, j - 1)] + p[ID(o, i, j - 1)]) +
                 (p[ID(o, i - 1, j)] + p[ID(o, i, j)]));
}

static void geometry(orc_ctx *o, double *p) {
  int nx = o->c.nx, ny = o->c.ny;
  fill_ghost(o, p, 0);
  for (int j = 0; j < ny; j++)
    for (int i = 0; i <= nx; i++)
      o->ax[ID(o, i, j)] =
          orc_edge_fraction(corner(o, p, i, j), corner(o, p, i, j + 1));
  for (int j = 0; j <= ny; j++)
    for (int i = 0; i < nx; i++)
      o->ay[ID(o, i, j)] =
          orc_edge_fraction(corner(o, p, i, j), corner(o, p, i + 1, j));
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      int c = ID(o, i, j);
      o->alpha[c] = orc_cell_alpha(corner(o, p, i, j), corner(o, p, i + 1, j),
                                   corner(o, p, i + 1, j + 1),
                                   corner(o, p, i, j + 1));
      /* the faces of the P region and its interface segment close:
       * S = sum over faces of A_P times the outward face normal length */
      o->sx[c] = (o->ax[ID(o, i + 1, j)] - o->ax[c]) * o->c.dy;
      o->sy[c] = (o->ay[ID(o, i, j + 1)] - o->ay[c]) * o->c.dx;
    }
}

static double vol(const orc_ctx *o, int k, int c) {
  return k == 1 ? o->alpha[c] : 1.0 - o->alpha[c];
}

/* unit normal grad(phi)/|grad(phi)| by central differences (points into P) */
static void normal(const orc_ctx *o, const double *p, int i, int j,
                   double *nxo, double *nyo) {
  double gx = (p[ID(o, i + 1, j)] - p[ID(o, i - 1, j)]) / (2.0 * o->c.dx);
  double gy = o->c.dim == 2
                  ? (p[ID(o, i, j + 1)] - p[ID(o, i, j - 1)]) / (2.0 * o->c.dy)
                  : 0.0;
  double m = sqrt(gx * gx + gy * gy);
  if (m > 0.0) {
    *nxo = gx / m;
    *nyo = gy / m;
  } else {
    *nxo = 0.0;
    *nyo = 0.0;
  }
}

static int inside(const orc_ctx *o, int i, int j) {
  return i >= 0 && i < o->c.nx && j >= 0 && j < o->c.ny;
}

/* ------------------------------------------------------------------ */
/* small-cell mixing (Sec. 2.2, last paragraph)                        */

/* targets of small cell (i, j) of fluid k: the normal-direction neighbours
 * that are not small cells themselves, weighted by the squared normal
 * components; when there is none, the largest of the eight neighbours if
 * it is not small; failing that, the normal-direction neighbours larger
 * than the source.  (Mixing a small cell into another small one lets
 * inconsistent content pile up in thin, under-resolved films.)  Returns
 * the number of targets, their cells and weights beta (summing to one). */
static int mix_targets(orc_ctx *o, int k, int i, int j, int tc[3], double beta[3]) {
  int c = ID(o, i, j);
  double as = vol(o, k, c);
  double nxv, nyv;
  normal(o, o->phi, i, j, &nxv, &nyv);
  if (k == 0) {
    nxv = -nxv;
    nyv = -nyv;
  }
  int sx = nxv >= 0.0 ? 1 : -1, sy = nyv >= 0.0 ? 1 : -1;
  int ti[3] = {i + sx, i, i + sx}, tj[3] = {j, j + sy, j + sy};
  double wt[3] = {nxv * nxv, nyv * nyv, fabs(nxv * nyv)};
  int nt = o->c.dim == 2 ? 3 : 1;
  int keep[3] = {0, 0, 0};
  double sum = 0.0;
  for (int t = 0; t < nt; t++) {
    if (!inside(o, ti[t], tj[t]) || !(wt[t] > 0.0)) continue;
    if (!(vol(o, k, ID(o, ti[t], tj[t])) >= o->c.mix_alpha)) continue;
    keep[t] = 1;
    sum += wt[t];
  }
  if (!(sum > 0.0)) {
    int best = -1;
    double ab = 0.0;
    for (int dj = -1; dj <= 1; dj++)
      for (int di = -1; di <= 1; di++) {
        if ((di == 0 && dj == 0) || (o->c.dim == 1 && dj != 0) || !inside(o, i + di, j + dj))
          continue;
        double at = vol(o, k, ID(o, i + di, j + dj));
        if (at > ab) {
          ab = at;
          best = ID(o, i + di, j + dj);
        }
      }
    if (best >= 0 && ab >= o->c.mix_alpha) {
      tc[0] = best;
      beta[0] = 1.0;
      return 1;
    }
    for (int t = 0; t < nt; t++) {
      if (!inside(o, ti[t], tj[t]) || !(wt[t] > 0.0)) continue;
      if (!(vol(o, k, ID(o, ti[t], tj[t])) > as)) continue;
      keep[t] = 1;
      sum += wt[t];
    }
  }
  if (!(sum > 0.0)) return 0;
  int n = 0;
  for (int t = 0; t < nt; t++) {
    if (!keep[t]) continue;
    tc[n] = ID(o, ti[t], tj[t]);
    beta[n] = wt[t] / sum;
    n++;
  }
  return n;
}

static void mix(orc_ctx *o, int k, double *const q[4]) {
  int nx = o->c.nx, ny = o->c.ny;
  for (int m = 0; m < 4; m++) memcpy(o->old[m], q[m], sizeof(double) * o->NP);
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      int c = ID(o, i, j);
      double as = vol(o, k, c);
      if (as >= o->c.mix_alpha) continue;
      if (as == 0.0 && o->old[0][c] == 0.0 && o->old[1][c] == 0.0 &&
          o->old[2][c] == 0.0 && o->old[3][c] == 0.0)
        continue;
      int tcs[3];
      double betas[3];
      int nt = mix_targets(o, k, i, j, tcs, betas);
      for (int t = 0; t < nt; t++) {
        int tc = tcs[t];
        double beta = betas[t];
        double at = vol(o, k, tc);
        double den = as * beta + at;
        for (int m = 0; m < 4; m++) {
          double M = beta * (o->old[m][tc] * as - o->old[m][c] * at) / den;
          q[m][c] += M;
          q[m][tc] -= M;
        }
      }
    }
}

/* ------------------------------------------------------------------ */
/* stencil states: real cells and extension (Sec. 2.3, last paragraph) */

/* a cell holds fluid k for stencil and CFL purposes if its volume
 * fraction exceeds the sliver threshold and, for a cut cell, its content
 * is a physical state */
static int is_real(const orc_ctx *o, int k, int c) {
  return vol(o, k, c) > ALPHA_REAL && !o->nostate[k][c];
}

/* Cut cells whose content is not a physical state -- a cell that has just
 * opened with no neighbour to mix from, or an under-resolved film whose
 * content ran away -- take extended states like slivers; their content is
 * carried, updated and mixed.  A full cell with such content is an error. */
static void prim(orc_ctx *o, int k, double *const q[4]) {
  double g = o->c.gamma[k], pi = o->c.pinf[k];
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      double a = vol(o, k, c);
      o->nostate[k][c] = 0;
      if (!(a > ALPHA_REAL)) continue;
      double rho = q[0][c] / a;
      double u = q[1][c] / q[0][c];
      double v = q[2][c] / q[0][c];
      double E = q[3][c] / a;
      double p;
      if (o->c.tait[k]) /* Tait's equation (Eq. 4): the density alone */
        p = o->c.tait_B[k] * (pow(rho / o->c.tait_rho0[k], g) - 1.0) + o->c.tait_p0[k];
      else
        p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v)) - g * pi;
      if (!(rho > 0.0) || !(p + pi > 0.0)) {
        if (a < 1.0) {
          o->nostate[k][c] = 1;
          continue;
        }
        o->err |= ORC_ERR_NONPHYS;
      }
      o->w[k][0][c] = rho;
      o->w[k][1][c] = u;
      o->w[k][2][c] = v;
      o->w[k][3][c] = p;
    }
}

/* Jacobi sweeps of the steady upwind discretisation of n_k . grad(q) = 0
 * (n_k the unit normal pointing into fluid k) for band cells that hold no
 * fluid k: each sweep sets a target to the upwind-weighted mean of its
 * upwind x and y neighbours (neighbours outside the domain drop out). */
static void extend(orc_ctx *o, int k, const double *p) {
  double bw = o->c.band * o->h;
  for (int it = 0; it < o->c.ext_iters; it++) {
    for (int m = 0; m < 4; m++) memcpy(o->old[m], o->w[k][m], sizeof(double) * o->NP);
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j);
        if (!(fabs(p[c]) < bw) || is_real(o, k, c)) continue;
        double nxv, nyv;
        normal(o, p, i, j, &nxv, &nyv);
        if (k == 0) {
          nxv = -nxv;
          nyv = -nyv;
        }
        int sx = nxv >= 0.0 ? 1 : -1, sy = nyv >= 0.0 ? 1 : -1;
        double wx = fabs(nxv) / o->c.dx;
        double wy = o->c.dim == 2 ? fabs(nyv) / o->c.dy : 0.0;
        if (!inside(o, i + sx, j)) wx = 0.0;
        if (!inside(o, i, j + sy)) wy = 0.0;
        double den = wx + wy;
        if (!(den > 0.0)) continue;
        for (int m = 0; m < 4; m++) {
          double num = 0.0;
          if (wx > 0.0) num += wx * o->old[m][ID(o, i + sx, j)];
          if (wy > 0.0) num += wy * o->old[m][ID(o, i, j + sy)];
          o->w[k][m][c] = num / den;
        }
      }
  }
}

/* Lax-Friedrichs alpha over every cell whose state can enter a stencil
 * (real or extended), and the CFL sum over real cells. */
static void wave_maxima(orc_ctx *o, int k, const double *p) {
  double g = o->c.gamma[k], pi = o->c.pinf[k];
  double bw = o->c.band * o->h;
  double lx = 0.0, ly = 0.0, sm = 0.0;
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      int real = is_real(o, k, c);
      if (!real && !(fabs(p[c]) < bw)) continue;
      double rho = o->w[k][0][c], u = o->w[k][1][c], v = o->w[k][2][c];
      double pr = o->w[k][3][c];
      double cs = sqrt(dmax(g * (pr + pi) / rho, 0.0));
      lx = dmax(lx, fabs(u) + cs);
      ly = dmax(ly, fabs(v) + cs);
      if (real) {
        double s = (fabs(u) + cs) / o->c.dx;
        if (o->c.dim == 2) s += (fabs(v) + cs) / o->c.dy;
        /* explicit viscous limit: 2 nu (1/dx^2 + 1/dy^2) added to the rate */
        if (o->c.mu[k] > 0.0) {
          double id2 = 1.0 / (o->c.dx * o->c.dx) + (o->c.dim == 2 ? 1.0 / (o->c.dy * o->c.dy) : 0.0);
          s += 2.0 * o->c.mu[k] / rho * id2;
        }
        sm = dmax(sm, s);
      }
    }
  o->lf[k][0] = lx;
  o->lf[k][1] = ly;
  o->smax[k] = sm;
}

/* ------------------------------------------------------------------ */
/* interface interaction: exact two-material Riemann problem           */

static void side_f(double p, double rho, double pk, double g, double pi,
                   double ck, int baro, double *f, double *df) {
  double P = pk + pi, Pp = p + pi;
  if (p > pk && baro) {
    /* barotropic shock (Tait): u jump^2 = (p - pk)(1/rho - 1/rho*), rho* =
     * rho r^(1/g), r = (p + pi)/(pk + pi); 1 - r^(-1/g) without
     * cancellation for r near 1 */
    double x = (p - pk) / P;
    double a = -expm1(-log1p(x) / g);        /* 1 - r^(-1/g) */
    double gsq = (p - pk) * a / rho;
    double dg = (a + (p - pk) * pow(1.0 + x, -1.0 / g - 1.0) / (g * P)) / rho;
    *f = sqrt(gsq);
    *df = dg / (2.0 * *f);
  } else if (p > pk) {
    double A = 2.0 / ((g + 1.0) * rho);
    double B = (g - 1.0) / (g + 1.0) * P;
    double qr = sqrt(A / (Pp + B));
    *f = (p - pk) * qr;
    *df = qr * (1.0 - 0.5 * (p - pk) / (Pp + B));
  } else {
    double r = Pp / P;
    *f = 2.0 * ck / (g - 1.0) * (pow(r, (g - 1.0) / (2.0 * g)) - 1.0);
    *df = 1.0 / (rho * ck) * pow(r, -(g + 1.0) / (2.0 * g));
  }
}

static double star_density(double p, double rho, double pk, double g, double pi, int baro) {
  double r = (p + pi) / (pk + pi);
  if (p > pk && !baro) {
    double qq = (g - 1.0) / (g + 1.0);
    return rho * (r + qq) / (qq * r + 1.0);
  }
  return rho * pow(r, 1.0 / g);
}

/* The star state satisfies u*_L = u*_R with p*_L = p*_R + jump: Newton on
 * the right star pressure p for f_L(p + jump) + f_R(p) + u_R - u_L = 0,
 * from the acoustic guess, each side's p + p_inf floored. */
int orc_riemann_jump2(const double *L, const double *R, double jump, int bl, int br,
                      double *out) {
  double rl = L[0], ul = L[1], pl = L[2], gl = L[3], pil = L[4];
  double rr = R[0], ur = R[1], pr = R[2], gr = R[3], pir = R[4];
  double cl = sqrt(gl * (pl + pil) / rl), cr = sqrt(gr * (pr + pir) / rr);
  double pscale = dmin(pl + pil, pr + pir);
  double pfloor = dmax(-pir, -pil - jump) + 1e-12 * pscale;
  double p = 0.5 * ((pl - jump) + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
  /* iterates stay above the floor without landing on it (where a
   * rarefaction's derivative diverges and a tiny step would pass for
   * convergence): a guess below it starts halfway to the larger pressure,
   * a step across it halves the distance to it instead */
  if (p < pfloor) p = pfloor + 0.5 * (dmax(pl - jump, pr) - pfloor);
  int it = 0, conv = 0, done = 0;
  double fl, dfl, fr, dfr;
  while (it < 50) {
    it++;
    side_f(p + jump, rl, pl, gl, pil, cl, bl, &fl, &dfl);
    side_f(p, rr, pr, gr, pir, cr, br, &fr, &dfr);
    double F = fl + fr + (ur - ul);
    double pn = p - F / (dfl + dfr);
    if (pn < pfloor) pn = pfloor + 0.5 * (p - pfloor);
    double dp = fabs(pn - p);
    p = pn;
    if (conv) {
      done = 1;
      break;
    }
    if (dp <= 1e-10 * (fabs(p) + pscale)) conv = 1;
  }
  double plst = p + jump;
  side_f(plst, rl, pl, gl, pil, cl, bl, &fl, &dfl);
  side_f(p, rr, pr, gr, pir, cr, br, &fr, &dfr);
  double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  double rsl = star_density(plst, rl, pl, gl, pil, bl);
  double rsr = star_density(p, rr, pr, gr, pir, br);
  out[0] = p;
  out[1] = us;
  out[2] = rsl;
  out[3] = rsr;
  out[4] = sqrt(gl * (plst + pil) / rsl);
  out[5] = sqrt(gr * (p + pir) / rsr);
  out[6] = (double)it;
  out[7] = plst;
  return (done || conv) ? 0 : ORC_ERR_NOCONV;
}

int orc_riemann_jump(const double *L, const double *R, double jump, double *out) {
  return orc_riemann_jump2(L, R, jump, 0, 0, out);
}

int orc_riemann(const double *L, const double *R, double *out) {
  double o8[8];
  int rc = orc_riemann_jump(L, R, 0.0, o8);
  for (int q = 0; q < 7; q++) out[q] = o8[q];
  return rc;
}

/* curvature of the level set: (phi_xx phi_y^2 - 2 phi_x phi_y phi_xy +
 * phi_yy phi_x^2) / |grad phi|^3, second-order central differences */
static double curvature(const orc_ctx *o, const double *p, int i, int j) {
  if (o->c.dim != 2) return 0.0;
  double dx = o->c.dx, dy = o->c.dy;
  double c0 = p[ID(o, i, j)];
  double px = (p[ID(o, i + 1, j)] - p[ID(o, i - 1, j)]) / (2.0 * dx);
  double py = (p[ID(o, i, j + 1)] - p[ID(o, i, j - 1)]) / (2.0 * dy);
  double pxx = (p[ID(o, i + 1, j)] - 2.0 * c0 + p[ID(o, i - 1, j)]) / (dx * dx);
  double pyy = (p[ID(o, i, j + 1)] - 2.0 * c0 + p[ID(o, i, j - 1)]) / (dy * dy);
  double pxy = (p[ID(o, i + 1, j + 1)] - p[ID(o, i + 1, j - 1)] - p[ID(o, i - 1, j + 1)] +
                p[ID(o, i - 1, j - 1)]) / (4.0 * dx * dy);
  double g2 = px * px + py * py;
  if (!(g2 > 0.0)) return 0.0;
  return (pxx * py * py - 2.0 * px * py * pxy + pyy * px * px) / (g2 * sqrt(g2));
}

static void visc_stress(double mu, double ux, double uy, double vx, double vy, double *txx,
                        double *txy, double *tyy);

/* velocity component m (1: u, 2: v) at cell (i, j) of the field that is
 * continuous across the interface: that of the fluid on whose side of the
 * interface the cell's centre lies (phi < 0: N) */
static double vel_across(const orc_ctx *o, const double *p, int m, int i, int j) {
  int c = ID(o, i, j);
  return o->w[p[c] < 0.0 ? 0 : 1][m][c];
}

/* X for every cut cell (|S| > 0): fluid N receives momentum -p_I,N S and
 * energy -p_I,N u_I |S|, fluid P momentum p_I,P S and energy p_I,P u_I |S|;
 * no mass crosses.  Without surface tension p_I,N = p_I,P; with it the
 * pressure jumps by sigma kappa from fluid P into fluid N (Eq. 10; kappa
 * > 0 where fluid N is convex, as inside a drop of fluid N). */
static void interface(orc_ctx *o, const double *p) {
  for (int m = 0; m < 3; m++) memset(o->xn[m], 0, sizeof(double) * o->NP);
  for (int m = 0; m < 3; m++) memset(o->xp[m], 0, sizeof(double) * o->NP);
  for (int m = 0; m < 2; m++) memset(o->ul[m], 0, sizeof(double) * o->NP);
  double fac = 1.0 / o->c.dx + (o->c.dim == 2 ? 1.0 / o->c.dy : 0.0);
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      double Sx = o->sx[c], Sy = o->sy[c];
      if (Sx == 0.0 && Sy == 0.0) continue;
      double Sm = sqrt(Sx * Sx + Sy * Sy);
      double nxv, nyv;
      normal(o, p, i, j, &nxv, &nyv);
      if (nxv == 0.0 && nyv == 0.0) {
        nxv = Sx / Sm;
        nyv = Sy / Sm;
      }
      double L[5] = {o->w[0][0][c], o->w[0][1][c] * nxv + o->w[0][2][c] * nyv,
                     o->w[0][3][c], o->c.gamma[0], o->c.pinf[0]};
      double R[5] = {o->w[1][0][c], o->w[1][1][c] * nxv + o->w[1][2][c] * nyv,
                     o->w[1][3][c], o->c.gamma[1], o->c.pinf[1]};
      double out[8];
      double jump = o->c.sigma != 0.0 ? o->c.sigma * curvature(o, p, i, j) : 0.0;
      if (orc_riemann_jump2(L, R, jump, o->c.tait[0], o->c.tait[1], out))
        o->err |= ORC_ERR_NOCONV;
      double psN = out[7], psP = out[0], us = out[1];
      o->xn[0][c] = -psN * Sx;
      o->xn[1][c] = -psN * Sy;
      o->xn[2][c] = -psN * us * Sm;
      o->xp[0][c] = psP * Sx;
      o->xp[1][c] = psP * Sy;
      o->xp[2][c] = psP * us * Sm;
      /* viscous traction across the interface (Eq. 5's interface term):
       * the stress of the velocity field that is continuous across it (at
       * every cell the velocity of the fluid on whose side of the
       * interface its centre lies), by central differences at the cut
       * cell, with the harmonic mean of the two viscosities; fluid N
       * receives it through S and fluid P the opposite, each with its work
       * at that field's velocity in the cut cell (momentum and energy leave
       * one fluid as they enter the other) */
      if (o->c.mu[0] > 0.0 && o->c.mu[1] > 0.0) {
        double muI = 2.0 * o->c.mu[0] * o->c.mu[1] / (o->c.mu[0] + o->c.mu[1]);
        double ux = (vel_across(o, p, 1, i + 1, j) - vel_across(o, p, 1, i - 1, j)) /
                    (2.0 * o->c.dx);
        double vx = (vel_across(o, p, 2, i + 1, j) - vel_across(o, p, 2, i - 1, j)) /
                    (2.0 * o->c.dx);
        double uy = 0.0, vy = 0.0;
        if (o->c.dim == 2) {
          uy = (vel_across(o, p, 1, i, j + 1) - vel_across(o, p, 1, i, j - 1)) / (2.0 * o->c.dy);
          vy = (vel_across(o, p, 2, i, j + 1) - vel_across(o, p, 2, i, j - 1)) / (2.0 * o->c.dy);
        }
        double txx, txy, tyy;
        visc_stress(muI, ux, uy, vx, vy, &txx, &txy, &tyy);
        double fx = txx * Sx + txy * Sy, fy = txy * Sx + tyy * Sy;
        double e = vel_across(o, p, 1, i, j) * fx + vel_across(o, p, 2, i, j) * fy;
        o->xn[0][c] = o->xn[0][c] + fx;
        o->xn[1][c] = o->xn[1][c] + fy;
        o->xn[2][c] = o->xn[2][c] + e;
        o->xp[0][c] = o->xp[0][c] - fx;
        o->xp[1][c] = o->xp[1][c] - fy;
        o->xp[2][c] = o->xp[2][c] - e;
      }
      o->ul[0][c] = us * nxv;
      o->ul[1][c] = us * nyv;
      o->smax[0] = dmax(o->smax[0], (fabs(us) + out[4]) * fac);
      o->smax[1] = dmax(o->smax[1], (fabs(us) + out[5]) * fac);
    }
}

/* level-set velocity: cut-cell values u_I n carried outward through the
 * band by the same upwind Jacobi sweeps, upwind meaning toward the
 * interface on either side */
static void extend_ls_velocity(orc_ctx *o, const double *p) {
  double bw = o->c.band * o->h;
  for (int it = 0; it < o->c.ext_iters; it++) {
    for (int m = 0; m < 2; m++) memcpy(o->old[m], o->ul[m], sizeof(double) * o->NP);
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j);
        if (!(fabs(p[c]) < bw)) continue;
        if (o->sx[c] != 0.0 || o->sy[c] != 0.0) continue;
        double nxv, nyv;
        normal(o, p, i, j, &nxv, &nyv);
        if (p[c] >= 0.0) {
          nxv = -nxv;
          nyv = -nyv;
        }
        int sx = nxv >= 0.0 ? 1 : -1, sy = nyv >= 0.0 ? 1 : -1;
        double wx = fabs(nxv) / o->c.dx;
        double wy = o->c.dim == 2 ? fabs(nyv) / o->c.dy : 0.0;
        if (!inside(o, i + sx, j)) wx = 0.0;
        if (!inside(o, i, j + sy)) wy = 0.0;
        double den = wx + wy;
        if (!(den > 0.0)) continue;
        for (int m = 0; m < 2; m++) {
          double num = 0.0;
          if (wx > 0.0) num += wx * o->old[m][ID(o, i + sx, j)];
          if (wy > 0.0) num += wy * o->old[m][ID(o, i, j + sy)];
          o->ul[m][c] = num / den;
        }
      }
  }
}

/* interaction step for the stage states qs and level set p */
static void eval(orc_ctx *o, double *const qs[2][4], double *p) {
  geometry(o, p);
  for (int k = 0; k < 2; k++) {
    prim(o, k, qs[k]);
    extend(o, k, p);
    wave_maxima(o, k, p);
  }
  interface(o, p);
  extend_ls_velocity(o, p);
}

/* ------------------------------------------------------------------ */
/* WENO5-LF fluxes and the cut-cell right-hand side (Eq. 2)            */

double orc_weno5(const double *v, double eps) {
  double v1 = v[0], v2 = v[1], v3 = v[2], v4 = v[3], v5 = v[4];
  double q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0;
  double q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0;
  double q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0;
  double b0 = 13.0 / 12.0 * sq(v1 - 2.0 * v2 + v3) + 0.25 * sq(v1 - 4.0 * v2 + 3.0 * v3);
  double b1 = 13.0 / 12.0 * sq(v2 - 2.0 * v3 + v4) + 0.25 * sq(v2 - v4);
  double b2 = 13.0 / 12.0 * sq(v3 - 2.0 * v4 + v5) + 0.25 * sq(3.0 * v3 - 4.0 * v4 + v5);
  double a0 = 0.1 / sq(eps + b0);
  double a1 = 0.6 / sq(eps + b1);
  double a2 = 0.3 / sq(eps + b2);
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* Lax-Friedrichs split fluxes of the stencil state of fluid k at cell c in
 * direction d (0 = x, 1 = y): fp = (F + a U)/2, fm = (F - a U)/2 */
static void split(const orc_ctx *o, int k, int c, int d, double a, double *fp,
                  double *fm) {
  double g = o->c.gamma[k], pi = o->c.pinf[k];
  double rho = o->w[k][0][c], u = o->w[k][1][c], v = o->w[k][2][c];
  double p = o->w[k][3][c];
  double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v);
  double U[4] = {rho, rho * u, rho * v, E};
  double F[4];
  if (d == 0) {
    F[0] = rho * u;
    F[1] = rho * u * u + p;
    F[2] = rho * u * v;
    F[3] = u * (E + p);
  } else {
    F[0] = rho * v;
    F[1] = rho * u * v;
    F[2] = rho * v * v + p;
    F[3] = v * (E + p);
  }
  for (int m = 0; m < 4; m++) {
    fp[m] = 0.5 * (F[m] + a * U[m]);
    fm[m] = 0.5 * (F[m] - a * U[m]);
  }
}

/* Eigenvectors of the flux Jacobian dF_d/dU of the 2D Euler equations.
 * With un the velocity along d, ut the one across it, q = (u^2+v^2)/2,
 * c^2 = g (p + pinf)/rho and H = (E + p)/rho = c^2/(g-1) + q (the
 * stiffened gas shifts p by a constant, so the ideal-gas structure holds
 * with this c), the fields are the acoustic waves un -+ c, the entropy wave
 * and the shear wave (both un).  Right eigenvectors, in (rho, rho un,
 * rho ut, E) order: (1, un - c, ut, H - un c), (1, un, ut, q), (0, 0, 1, ut),
 * (1, un + c, ut, H + un c); with b1 = (g-1)/c^2 and b2 = b1 q the left
 * ones are (b2 + un/c, -b1 un - 1/c, -b1 ut, b1)/2, (1 - b2, b1 un, b1 ut,
 * -b1), (-ut, 0, 1, 0), (b2 - un/c, -b1 un + 1/c, -b1 ut, b1)/2.  The x and y
 * momentum components are then placed in the grid's order. */
int orc_char_basis(double g, double pinf, double rho, double u, double v, double p, int d,
                   double *L, double *R) {
  if (!(rho > 0.0) || !(p + pinf > 0.0) || !(g > 1.0) || (d != 0 && d != 1))
    return ORC_ERR_INVAL;
  double un = d == 0 ? u : v, ut = d == 0 ? v : u;
  double c = sqrt(g * (p + pinf) / rho);
  double q = 0.5 * (u * u + v * v);
  double H = c * c / (g - 1.0) + q;
  double b1 = (g - 1.0) / (c * c), b2 = b1 * q;
  /* in (rho, rho un, rho ut, E) order */
  double Rn[4][4] = {{1.0, 1.0, 0.0, 1.0},
                     {un - c, un, 0.0, un + c},
                     {ut, ut, 1.0, ut},
                     {H - un * c, q, ut, H + un * c}};
  double Ln[4][4] = {{0.5 * (b2 + un / c), 0.5 * (-b1 * un - 1.0 / c), 0.5 * (-b1 * ut), 0.5 * b1},
                     {1.0 - b2, b1 * un, b1 * ut, -b1},
                     {-ut, 0.0, 1.0, 0.0},
                     {0.5 * (b2 - un / c), 0.5 * (-b1 * un + 1.0 / c), 0.5 * (-b1 * ut), 0.5 * b1}};
  /* grid component m of (rho, rho u, rho v, E) is component perm[m] of the
   * (rho, rho un, rho ut, E) ordering */
  int perm[4] = {0, d == 0 ? 1 : 2, d == 0 ? 2 : 1, 3};
  for (int m = 0; m < 4; m++)
    for (int f = 0; f < 4; f++) {
      R[m * 4 + f] = Rn[perm[m]][f];
      L[f * 4 + m] = Ln[f][perm[m]];
    }
  return 0;
}

/* physical flux of direction d and conserved state of a primitive state of
 * a stiffened gas */
static void euler_flux(const double *W, double g, double pi, int d, double *F, double *U) {
  double rho = W[0], u = W[1], v = W[2], p = W[3];
  double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v);
  double un = d == 0 ? u : v;
  U[0] = rho;
  U[1] = rho * u;
  U[2] = rho * v;
  U[3] = E;
  F[0] = rho * un;
  F[1] = rho * u * un;
  F[2] = rho * v * un;
  F[3] = un * (E + p);
  F[1 + d] += p;
}

/* HLLC (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics,
 * Sec. 10.4): the two outer waves S_L, S_R bound the fan, the contact
 * moves with S*, and the star states on either side of it are
 *   U*_K = rho_K (S_K - un_K) / (S_K - S*) (1, S* along d, ut_K across d,
 *          E_K / rho_K + (S* - un_K) (S* + p_K / (rho_K (S_K - un_K)))).
 * The flux is F_L, F_L + S_L (U*_L - U_L), F_R + S_R (U*_R - U_R) or F_R
 * as the face (x/t = 0) lies left of S_L, between S_L and S*, between S*
 * and S_R, or right of S_R. */
int orc_hllc(const double *WL, const double *WR, double g, double pi, int d, double *F) {
  if (!(WL[0] > 0.0) || !(WR[0] > 0.0) || !(WL[3] + pi > 0.0) || !(WR[3] + pi > 0.0) ||
      !(g > 1.0) || (d != 0 && d != 1))
    return ORC_ERR_INVAL;
  double FL[4], UL[4], FR[4], UR[4];
  euler_flux(WL, g, pi, d, FL, UL);
  euler_flux(WR, g, pi, d, FR, UR);
  double rl = WL[0], rr = WR[0], pl = WL[3], pr = WR[3];
  double ul = d == 0 ? WL[1] : WL[2], ur = d == 0 ? WR[1] : WR[2];
  double cl = sqrt(g * (pl + pi) / rl), cr = sqrt(g * (pr + pi) / rr);
  double SL = dmin(ul - cl, ur - cr), SR = dmax(ul + cl, ur + cr);
  if (SL >= 0.0) {
    for (int m = 0; m < 4; m++) F[m] = FL[m];
    return 0;
  }
  if (SR <= 0.0) {
    for (int m = 0; m < 4; m++) F[m] = FR[m];
    return 0;
  }
  double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
              (rl * (SL - ul) - rr * (SR - ur));
  const double *W = Ss >= 0.0 ? WL : WR;
  const double *FK = Ss >= 0.0 ? FL : FR;
  const double *UK = Ss >= 0.0 ? UL : UR;
  double SK = Ss >= 0.0 ? SL : SR, uK = Ss >= 0.0 ? ul : ur;
  double fac = W[0] * (SK - uK) / (SK - Ss);
  double Us[4];
  Us[0] = fac;
  Us[1] = fac * (d == 0 ? Ss : W[1]);
  Us[2] = fac * (d == 0 ? W[2] : Ss);
  Us[3] = fac * (UK[3] / W[0] + (Ss - uK) * (Ss + W[3] / (W[0] * (SK - uK))));
  for (int m = 0; m < 4; m++) F[m] = FK[m] + SK * (Us[m] - UK[m]);
  return 0;
}

/* HLLC face flux of fluid k between cells c - s and c: each primitive
 * component reconstructed by WENO5 from the left (cells c-3s .. c+s) and
 * from the right (cells c+2s .. c-2s); a reconstructed state that is not
 * physical (density or p + pinf not positive) is replaced by its cell's
 * own state (first order) */
static void face_flux_hllc(const orc_ctx *o, int k, int c, int s, int d, double *Fh) {
  double g = o->c.gamma[k], pi = o->c.pinf[k];
  double WL[4], WR[4];
  for (int m = 0; m < 4; m++) {
    const double *w = o->w[k][m];
    double vl[5], vr[5];
    for (int r = 0; r < 5; r++) {
      vl[r] = w[c + (r - 3) * s];
      vr[r] = w[c + (2 - r) * s];
    }
    WL[m] = orc_weno5(vl, o->c.weno_eps);
    WR[m] = orc_weno5(vr, o->c.weno_eps);
  }
  if (!(WL[0] > 0.0) || !(WL[3] + pi > 0.0))
    for (int m = 0; m < 4; m++) WL[m] = o->w[k][m][c - s];
  if (!(WR[0] > 0.0) || !(WR[3] + pi > 0.0))
    for (int m = 0; m < 4; m++) WR[m] = o->w[k][m][c];
  if (orc_hllc(WL, WR, g, pi, d, Fh) != 0)
    for (int m = 0; m < 4; m++) Fh[m] = NAN;  /* a non-physical stencil state */
}

/* numerical flux through the face between cells c - s and c, where s is
 * the index stride of direction d.  Component-wise: WENO5 of each
 * conserved component of the split fluxes.  Characteristic-wise: the split
 * fluxes of the stencil are projected on the left eigenvectors of the face
 * state (the mean of the two adjacent cells' stencil states), each field is
 * reconstructed by WENO5, and the fields are mapped back by the right
 * eigenvectors. */
static void face_flux(const orc_ctx *o, int k, int c, int s, int d, double *Fh) {
  if (o->c.flux == 1) {
    face_flux_hllc(o, k, c, s, d, Fh);
    return;
  }
  double a = o->lf[k][d];
  double fp[6][4], fm[6][4];
  for (int r = 0; r < 6; r++) split(o, k, c + (r - 3) * s, d, a, fp[r], fm[r]);
  if (!o->c.weno_char) {
    for (int m = 0; m < 4; m++) {
      double vp[5] = {fp[0][m], fp[1][m], fp[2][m], fp[3][m], fp[4][m]};
      double vm[5] = {fm[5][m], fm[4][m], fm[3][m], fm[2][m], fm[1][m]};
      Fh[m] = orc_weno5(vp, o->c.weno_eps) + orc_weno5(vm, o->c.weno_eps);
    }
    return;
  }
  int cl = c - s, cr = c;
  double rho = 0.5 * (o->w[k][0][cl] + o->w[k][0][cr]);
  double u = 0.5 * (o->w[k][1][cl] + o->w[k][1][cr]);
  double v = 0.5 * (o->w[k][2][cl] + o->w[k][2][cr]);
  double p = 0.5 * (o->w[k][3][cl] + o->w[k][3][cr]);
  double L[16], R[16], h[4];
  orc_char_basis(o->c.gamma[k], o->c.pinf[k], rho, u, v, p, d, L, R);
  for (int f = 0; f < 4; f++) {
    double vp[5], vm[5];
    for (int r = 0; r < 5; r++) {
      vp[r] = 0.0;
      vm[r] = 0.0;
      for (int m = 0; m < 4; m++) {
        vp[r] += L[f * 4 + m] * fp[r][m];
        vm[r] += L[f * 4 + m] * fm[5 - r][m];
      }
    }
    h[f] = orc_weno5(vp, o->c.weno_eps) + orc_weno5(vm, o->c.weno_eps);
  }
  for (int m = 0; m < 4; m++) {
    Fh[m] = 0.0;
    for (int f = 0; f < 4; f++) Fh[m] += R[m * 4 + f] * h[f];
  }
}

/* Viscous stress of fluid k (Stokes' hypothesis, no heat conduction):
 * tau_xx = mu (4/3 u_x - 2/3 v_y), tau_yy = mu (4/3 v_y - 2/3 u_x),
 * tau_xy = mu (u_y + v_x). */
static void visc_stress(double mu, double ux, double uy, double vx, double vy, double *txx,
                        double *txy, double *tyy) {
  *txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy);
  *tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux);
  *txy = mu * (uy + vx);
}

/* viscous flux through the face between cells c - s and c (direction d)
 * from the stencil states by central differences: the normal derivatives
 * across the face, the tangential ones averaged over the two cells */
static void viscous_face(const orc_ctx *o, int k, int c, int s, int d, double *Fv) {
  const double *u = o->w[k][1], *v = o->w[k][2];
  double dx = o->c.dx, dy = o->c.dy;
  int cl = c - s;
  double ux, uy, vx, vy;
  if (d == 0) {
    ux = (u[c] - u[cl]) / dx;
    vx = (v[c] - v[cl]) / dx;
    if (o->c.dim == 2) {
      int t = o->PX;
      uy = ((u[c + t] - u[c - t]) + (u[cl + t] - u[cl - t])) / (4.0 * dy);
      vy = ((v[c + t] - v[c - t]) + (v[cl + t] - v[cl - t])) / (4.0 * dy);
    } else {
      uy = vy = 0.0;
    }
  } else {
    uy = (u[c] - u[cl]) / dy;
    vy = (v[c] - v[cl]) / dy;
    ux = ((u[c + 1] - u[c - 1]) + (u[cl + 1] - u[cl - 1])) / (4.0 * dx);
    vx = ((v[c + 1] - v[c - 1]) + (v[cl + 1] - v[cl - 1])) / (4.0 * dx);
  }
  double txx, txy, tyy;
  visc_stress(o->c.mu[k], ux, uy, vx, vy, &txx, &txy, &tyy);
  double uf = 0.5 * (u[cl] + u[c]), vf = 0.5 * (v[cl] + v[c]);
  Fv[0] = 0.0;
  if (d == 0) {
    Fv[1] = txx;
    Fv[2] = txy;
    Fv[3] = uf * txx + vf * txy;
  } else {
    Fv[1] = txy;
    Fv[2] = tyy;
    Fv[3] = uf * txy + vf * tyy;
  }
}

static void fv_rhs(orc_ctx *o, int k, double *const L[4]) {
  int nx = o->c.nx, ny = o->c.ny;
  fill_ghost(o, o->w[k][0], 0);
  fill_ghost(o, o->w[k][1], 1);
  fill_ghost(o, o->w[k][2], 2);
  fill_ghost(o, o->w[k][3], 0);
  for (int m = 0; m < 4; m++) {
    memset(o->fx[m], 0, sizeof(double) * o->NP);
    memset(o->fy[m], 0, sizeof(double) * o->NP);
  }
  double Fh[4];
  for (int j = 0; j < ny; j++)
    for (int i = 0; i <= nx; i++) {
      int c = ID(o, i, j);
      double A = k == 1 ? o->ax[c] : 1.0 - o->ax[c];
      if (A == 0.0) continue;
      face_flux(o, k, c, 1, 0, Fh);
      if (o->c.mu[k] > 0.0) {
        double Fv[4];
        viscous_face(o, k, c, 1, 0, Fv);
        for (int m = 0; m < 4; m++) Fh[m] = Fh[m] - Fv[m];
      }
      for (int m = 0; m < 4; m++) o->fx[m][c] = A * Fh[m];
    }
  if (o->c.dim == 2)
    for (int j = 0; j <= ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j);
        double A = k == 1 ? o->ay[c] : 1.0 - o->ay[c];
        if (A == 0.0) continue;
        face_flux(o, k, c, o->PX, 1, Fh);
        if (o->c.mu[k] > 0.0) {
          double Fv[4];
          viscous_face(o, k, c, o->PX, 1, Fv);
          for (int m = 0; m < 4; m++) Fh[m] = Fh[m] - Fv[m];
        }
        for (int m = 0; m < 4; m++) o->fy[m][c] = A * Fh[m];
      }
  double dxdy = o->c.dx * o->c.dy;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      int c = ID(o, i, j);
      /* a cell counts as updated if one of its faces is open to fluid k */
      double Al = k == 1 ? o->ax[c] : 1.0 - o->ax[c];
      double Ar = k == 1 ? o->ax[ID(o, i + 1, j)] : 1.0 - o->ax[ID(o, i + 1, j)];
      int open = Al != 0.0 || Ar != 0.0;
      if (o->c.dim == 2) {
        double Ab = k == 1 ? o->ay[c] : 1.0 - o->ay[c];
        double At = k == 1 ? o->ay[ID(o, i, j + 1)] : 1.0 - o->ay[ID(o, i, j + 1)];
        open = open || Ab != 0.0 || At != 0.0;
      }
      o->open_updates += open;
      for (int m = 0; m < 4; m++) {
        double r = (o->fx[m][c] - o->fx[m][ID(o, i + 1, j)]) / o->c.dx;
        if (o->c.dim == 2) r += (o->fy[m][c] - o->fy[m][ID(o, i, j + 1)]) / o->c.dy;
        if (m > 0) r += (k == 0 ? o->xn : o->xp)[m - 1][c] / dxdy;
        L[m][c] = r;
      }
    }
}

/* ------------------------------------------------------------------ */
/* level set: advection (Eq. 6) and reinitialisation                   */

static void make_band(orc_ctx *o, const double *p) {
  double bw = o->c.band * o->h;
  memset(o->band, 0, o->NP);
  memset(o->rext, 0, o->NP);
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++)
      o->band[ID(o, i, j)] = fabs(p[ID(o, i, j)]) < bw;
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j), r = o->band[c];
      if (i > 0) r |= o->band[ID(o, i - 1, j)];
      if (i < o->c.nx - 1) r |= o->band[ID(o, i + 1, j)];
      if (o->c.dim == 2) {
        if (j > 0) r |= o->band[ID(o, i, j - 1)];
        if (j < o->c.ny - 1) r |= o->band[ID(o, i, j + 1)];
      }
      o->rext[c] = (unsigned char)r;
    }
}

/* upwind HJ-WENO5 derivative along stride s: backward-biased if up > 0 */
static double hj_deriv(const orc_ctx *o, const double *p, int c, int s, double h,
                       int backward) {
  double v[5];
  if (backward) {
    for (int r = 0; r < 5; r++) {
      int m = c + (r - 2) * s;
      v[r] = (p[m] - p[m - s]) / h;
    }
  } else {
    for (int r = 0; r < 5; r++) {
      int m = c + (2 - r) * s;
      v[r] = (p[m + s] - p[m]) / h;
    }
  }
  return orc_weno5(v, o->c.weno_eps);
}

static void ls_rhs(orc_ctx *o, double *p, double *L) {
  fill_ghost(o, p, 0);
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      if (!o->band[c]) {
        L[c] = 0.0;
        continue;
      }
      double u = o->ul[0][c], v = o->ul[1][c];
      double px = 0.0, py = 0.0;
      if (u != 0.0) px = hj_deriv(o, p, c, 1, o->c.dx, u > 0.0);
      if (o->c.dim == 2 && v != 0.0) py = hj_deriv(o, p, c, o->PX, o->c.dy, v > 0.0);
      L[c] = -(u * px + v * py);
    }
}

static double grad_est(const double *p, int c, int s, double h) {
  double dm = fabs(p[c] - p[c - s]), dp = fabs(p[c + s] - p[c]);
  double dc = 0.5 * fabs(p[c + s] - p[c - s]);
  return dmax(dmax(dc, dp), dm) / h;
}

/* sweeps of phi_tau + S(phi0)(|grad phi| - 1) = 0 (Godunov upwind with
 * WENO5 one-sided derivatives) with the subcell fix in cells where phi0
 * changes sign across a face, over the band and its face neighbours;
 * cells farther out keep their last values */
static void reinit(orc_ctx *o, double *p) {
  int nx = o->c.nx, ny = o->c.ny, d2 = o->c.dim == 2;
  double h = o->h;
  fill_ghost(o, p, 0);
  memcpy(o->p0, p, sizeof(double) * o->NP);
  for (int it = 0; it < o->c.reinit_iters; it++) {
    fill_ghost(o, p, 0);
    memcpy(o->old[0], p, sizeof(double) * o->NP);
    const double *q = o->old[0], *z = o->p0;
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j);
        if (!o->rext[c]) continue;
        double s0 = z[c];
        int pos = s0 >= 0.0;
        int cut = (z[c - 1] >= 0.0) != pos || (z[c + 1] >= 0.0) != pos;
        if (d2) cut = cut || (z[c - o->PX] >= 0.0) != pos || (z[c + o->PX] >= 0.0) != pos;
        if (cut) {
          /* subcell distance from phi0 and its central-difference gradient
           * (one-sided maxima where the central difference vanishes) */
          double gx = (z[c + 1] - z[c - 1]) / (2.0 * o->c.dx);
          double gy = d2 ? (z[c + o->PX] - z[c - o->PX]) / (2.0 * o->c.dy) : 0.0;
          double gm = sqrt(gx * gx + gy * gy);
          if (!(gm > 1e-8)) {
            gx = grad_est(z, c, 1, o->c.dx);
            gy = d2 ? grad_est(z, c, o->PX, o->c.dy) : 0.0;
            gm = sqrt(gx * gx + gy * gy);
          }
          /* the interface lies no farther than the linear crossing toward
           * any face neighbour of opposite sign */
          double dmin = INFINITY;
          const int nbs[4] = {-1, 1, -o->PX, o->PX};
          for (int e = 0; e < (d2 ? 4 : 2); e++) {
            double zn = z[c + nbs[e]];
            if ((zn >= 0.0) == pos) continue;
            double hh = e < 2 ? o->c.dx : o->c.dy;
            double dd = fabs(s0) / (fabs(s0) + fabs(zn)) * hh;
            if (dd < dmin) dmin = dd;
          }
          double D = fabs(s0) / gm;
          if (D > dmin) D = dmin;
          D = pos ? D : -D;
          double sg = pos ? 1.0 : -1.0;
          p[c] = q[c] - 0.5 * (sg * fabs(q[c]) - D);
        } else {
          double S = s0 / sqrt(s0 * s0 + h * h);
          /* one-sided HJ-WENO5 derivatives in the Godunov Hamiltonian */
          double a = hj_deriv(o, q, c, 1, o->c.dx, 1), b = hj_deriv(o, q, c, 1, o->c.dx, 0);
          double cc = 0.0, d = 0.0;
          if (d2) {
            cc = hj_deriv(o, q, c, o->PX, o->c.dy, 1);
            d = hj_deriv(o, q, c, o->PX, o->c.dy, 0);
          }
          double G;
          if (s0 > 0.0)
            G = dmax(sq(dmax(a, 0.0)), sq(dmin(b, 0.0))) +
                dmax(sq(dmax(cc, 0.0)), sq(dmin(d, 0.0)));
          else if (s0 < 0.0)
            G = dmax(sq(dmin(a, 0.0)), sq(dmax(b, 0.0))) +
                dmax(sq(dmin(cc, 0.0)), sq(dmax(d, 0.0)));
          else
            continue;
          double nv = q[c] - 0.5 * h * S * (sqrt(G) - 1.0);
          /* no new extremum: a positive value stays at or above its
           * smallest face neighbour, a negative one at or below its
           * largest (the WENO derivatives can overshoot at the kinks that
           * form where the moving band meets the level set outside it) */
          double lo = dmin(q[c - 1], q[c + 1]), hi = dmax(q[c - 1], q[c + 1]);
          if (d2) {
            lo = dmin(lo, dmin(q[c - o->PX], q[c + o->PX]));
            hi = dmax(hi, dmax(q[c - o->PX], q[c + o->PX]));
          }
          if (s0 > 0.0 && nv < lo) nv = lo;
          if (s0 < 0.0 && nv > hi) nv = hi;
          p[c] = nv;
        }
      }
  }
}

/* ------------------------------------------------------------------ */
/* time integration                                                    */

static const double RK2A[3] = {0.0, 0.0, 0.5}, RK2B[3] = {0.0, 1.0, 0.5};
static const double RK3A[4] = {0.0, 0.0, 0.75, 1.0 / 3.0};
static const double RK3B[4] = {0.0, 1.0, 0.25, 2.0 / 3.0};

/* dst = cur + dt L (stage 1), else dst = a base + b (cur + dt L) */
static void rk_plane(orc_ctx *o, int s, double *dst, const double *base,
                     const double *cur, const double *L, double dt,
                     const unsigned char *mask) {
  double a = o->c.rk_order == 3 ? RK3A[s] : RK2A[s];
  double b = o->c.rk_order == 3 ? RK3B[s] : RK2B[s];
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      if (mask && !mask[c]) continue;
      if (s == 1)
        dst[c] = cur[c] + dt * L[c];
      else
        dst[c] = a * base[c] + b * (cur[c] + dt * L[c]);
    }
}

static double dt_of(const orc_ctx *o, int k) {
  return o->smax[k] > 0.0 ? o->c.cfl / o->smax[k] : INFINITY;
}

static void copy_planes(orc_ctx *o, double *const dst[4], double *const src[4], int n) {
  for (int m = 0; m < n; m++) memcpy(dst[m], src[m], sizeof(double) * o->NP);
}

static void copy_out(const orc_ctx *o, const double *src, double *dst);

/* what a recorded step keeps of its schedule: the Lax-Friedrichs speeds of
 * each stage (stage, fluid, direction) and the level set after stage 1 */
typedef struct {
  double *lf;   /* 8 */
  double *phi1; /* nx*ny */
} step_record;

/* one RK step of both fluids and the level set with a common dt, the
 * first interaction step having been evaluated already */
static void single_step_after_eval(orc_ctx *o, double dt, step_record *rec) {
  int S = o->c.rk_order;
  for (int k = 0; k < 2; k++) copy_planes(o, o->q0[k], o->q[k], 4);
  memcpy(o->phi0, o->phi, sizeof(double) * o->NP);
  make_band(o, o->phi0);
  for (int s = 1; s <= S; s++) {
    if (s > 1) eval(o, o->q, o->phi);
    if (rec && s <= 2)
      for (int k = 0; k < 2; k++)
        for (int d = 0; d < 2; d++) rec->lf[(s - 1) * 4 + k * 2 + d] = o->lf[k][d];
    for (int k = 0; k < 2; k++) fv_rhs(o, k, o->L[k]);
    ls_rhs(o, o->phi, o->lphi);
    for (int k = 0; k < 2; k++)
      for (int m = 0; m < 4; m++)
        rk_plane(o, s, o->q[k][m], o->q0[k][m], o->q[k][m], o->L[k][m], dt, NULL);
    rk_plane(o, s, o->phi, o->phi0, o->phi, o->lphi, dt, o->band);
    if (rec && s == 1) copy_out(o, o->phi, rec->phi1);
    if (s == S) reinit(o, o->phi);
    geometry(o, o->phi);
    mix(o, 0, o->q[0]);
    mix(o, 1, o->q[1]);
  }
  o->t += dt;
}

int orc_step_single_dt(orc_ctx *o, int nsteps, double t_end, orc_info *info) {
  long long open0 = o->open_updates;
  for (int n = 0; n < nsteps; n++) {
    if (t_end > 0.0 && o->t >= t_end) break;
    eval(o, o->q, o->phi);
    double dt = dmin(dt_of(o, 0), dt_of(o, 1));
    if (t_end > 0.0 && o->t + dt > t_end) dt = t_end - o->t;
    single_step_after_eval(o, dt, NULL);
    if (info) {
      info->t = o->t;
      info->dt1 = dt;
      info->dt2 = dt;
      info->n_raw = 1.0;
      info->n_used = 1.0;
      info->role_fluid1 = -1;
      info->substeps = 1;
    }
  }
  if (info) {
    info->err = o->err;
    info->open_updates = o->open_updates - open0;
  }
  return o->err;
}

/* Eq. 8 (shared evaluation) or Eq. 9 (fluid-2-only evaluation): update of
 * the correction quantities with the exchange flux as applied to fluid 1 */
static void record(orc_ctx *o, int f1, int shared, double dt1, double dt2) {
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      for (int m = 0; m < 3; m++) {
        double x1 = (f1 == 0 ? o->xn : o->xp)[m][c];
        if (shared) o->xc[m][c] = o->xc[m][c] + (-0.5 * x1) * dt1;
        o->xc[m][c] = o->xc[m][c] + (0.5 * x1) * dt2;
      }
    }
}

/* Eq. 7: fluid-1 state at fluid-2 time t2 inside the cycle */
static void interpolate(orc_ctx *o, double th) {
  for (int m = 0; m < 4; m++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j);
        o->qi[m][c] = (1.0 - th) * o->prev[m][c] + th * o->fut[m][c];
      }
}

static void cycle_rk3(orc_ctx *o, int f1, double dt1, double dt2, orc_info *info);

/* one cycle of the accelerated method (Sec. 3.1, steps 1-5) */
static void cycle(orc_ctx *o, double t_end, orc_info *info) {
  eval(o, o->q, o->phi);
  double dtk[2] = {dt_of(o, 0), dt_of(o, 1)};
  for (int k = 0; k < 2; k++)
    if (t_end > 0.0 && o->t + dtk[k] > t_end) dtk[k] = t_end - o->t;
  int f1 = dtk[1] > dtk[0] ? 1 : 0, f2 = 1 - f1;
  double dt1 = dtk[f1], dt2 = dtk[f2];
  double nraw = dt1 / dt2;
  if (info) {
    info->n_raw = nraw;
    info->role_fluid1 = f1;
    info->dt2 = dt2;
  }
  if (o->c.force_ratio_one) {
    dt1 = dt2;
  } else {
    if (isfinite(dt1)) {
      double fl = floor(nraw);
      if (nraw - fl < o->c.ratio_threshold) dt1 = fl * dt2;
    }
    if (!isfinite(dt1) || dt1 <= dt2) {
      single_step_after_eval(o, dt2, NULL);
      if (info) {
        info->dt1 = dt2;
        info->n_used = 1.0;
        info->substeps = 1;
        info->t = o->t;
      }
      return;
    }
  }
  if (info) {
    info->dt1 = dt1;
    info->n_used = dt1 / dt2;
  }
  if (o->c.rk_order == 3) {
    cycle_rk3(o, f1, dt1, dt2, info);
    return;
  }
  for (int m = 0; m < 3; m++) memset(o->xc[m], 0, sizeof(double) * o->NP);
  /* step 2: fluid-1 first RK stage with dt1; keep previous and future */
  fv_rhs(o, f1, o->L[f1]);
  copy_planes(o, o->prev, o->q[f1], 4);
  for (int m = 0; m < 4; m++)
    rk_plane(o, 1, o->fut[m], o->prev[m], o->prev[m], o->L[f1][m], dt1, NULL);
  double t2 = 0.0;
  int sub = 0;
  double *qs[2][4];
  for (;;) {
    sub++;
    if (sub > 1) {
      interpolate(o, t2 / dt1);
      geometry(o, o->phi);
      mix(o, f1, o->qi);
      for (int m = 0; m < 4; m++) {
        qs[f1][m] = o->qi[m];
        qs[f2][m] = o->q[f2][m];
      }
      eval(o, qs, o->phi);
      dt2 = dt_of(o, f2);
    }
    int last = (dt1 - t2) <= dt2 * (1.0 + 1e-12);
    if (last) dt2 = dt1 - t2;
    record(o, f1, sub == 1, dt1, dt2);
    /* step 3: fluid-2 and level-set first RK stage with dt2 */
    copy_planes(o, o->q0[f2], o->q[f2], 4);
    memcpy(o->phi0, o->phi, sizeof(double) * o->NP);
    make_band(o, o->phi0);
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    for (int m = 0; m < 4; m++)
      rk_plane(o, 1, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 1, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    geometry(o, o->phi);
    mix(o, f2, o->q[f2]);
    if (last) {
      mix(o, f1, o->fut);
      for (int m = 0; m < 4; m++) qs[f1][m] = o->fut[m];
    } else {
      interpolate(o, (t2 + dt2) / dt1);
      mix(o, f1, o->qi);
      for (int m = 0; m < 4; m++) qs[f1][m] = o->qi[m];
    }
    for (int m = 0; m < 4; m++) qs[f2][m] = o->q[f2][m];
    eval(o, qs, o->phi);
    record(o, f1, last, dt1, dt2);
    /* step 4 (and 5 on the last sub-step): second RK stage */
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    if (last) fv_rhs(o, f1, o->L[f1]);
    for (int m = 0; m < 4; m++)
      rk_plane(o, 2, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 2, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    if (last)
      for (int m = 0; m < 4; m++)
        rk_plane(o, 2, o->q[f1][m], o->prev[m], o->fut[m], o->L[f1][m], dt1, NULL);
    reinit(o, o->phi);
    if (last) {
      if (o->c.flux_correction) {
        double dxdy = o->c.dx * o->c.dy;
        for (int j = 0; j < o->c.ny; j++)
          for (int i = 0; i < o->c.nx; i++) {
            int c = ID(o, i, j);
            for (int m = 0; m < 3; m++) o->q[f1][m + 1][c] += o->xc[m][c] / dxdy;
          }
      }
      geometry(o, o->phi);
      mix(o, f1, o->q[f1]);
      mix(o, f2, o->q[f2]);
      break;
    }
    t2 += dt2;
    geometry(o, o->phi);
    mix(o, f2, o->q[f2]);
  }
  o->t += dt1;
  if (info) {
    info->substeps = sub;
    info->t = o->t;
  }
}

/* Eq. 8-9 with the weight b of the evaluation's Runge-Kutta stage: a
 * fluid-2 evaluation adds b dt2 X_1; one that fluid 1 uses too (shared)
 * also removes b dt1 X_1; a fluid-1-only evaluation (dt2 = 0, shared)
 * only removes b dt1 X_1. */
static void record_b(orc_ctx *o, int f1, int shared, double b, double dt1, double dt2) {
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      for (int m = 0; m < 3; m++) {
        double x1 = (f1 == 0 ? o->xn : o->xp)[m][c];
        if (shared) o->xc[m][c] = o->xc[m][c] + (-b * x1) * dt1;
        if (dt2 > 0.0) o->xc[m][c] = o->xc[m][c] + (b * x1) * dt2;
      }
    }
}

/* linear interpolation in time between two snapshots a (weight 1 - th)
 * and b (weight th); where they agree the value is kept as it is */
static void interp2(const orc_ctx *o, double *dst, const double *a, const double *b, double th) {
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      dst[c] = a[c] == b[c] ? a[c] : (1.0 - th) * a[c] + th * b[c];
    }
}

/* The evaluation of fluid 1's third RK3 stage inside a cycle: fluid 1's
 * stencil states on the current geometry (recovered, extended) and its
 * wave speeds, and no exchange flux -- the correction quantities would
 * remove that evaluation's exchange from fluid 1's result exactly, so it
 * is left out (fluid 1 ends with the exchange fluid 2 received, Eq. 8-9).
 * Fluid 2's stencil states are extended on the same geometry from where
 * they are, as warm start of the next interaction step. */
static void eval_third(orc_ctx *o, int f1, double *p) {
  prim(o, f1, o->q[f1]);
  for (int k = 0; k < 2; k++) extend(o, k, p);
  for (int k = 0; k < 2; k++) wave_maxima(o, k, p);
  for (int m = 0; m < 3; m++) {
    memset(o->xn[m], 0, sizeof(double) * o->NP);
    memset(o->xp[m], 0, sizeof(double) * o->NP);
  }
}

/* One accelerated cycle with SSP-RK3 (stage weights b = 1/6, 1/6, 2/3 at
 * the stage times t^n, t^n + dt, t^n + dt/2): the generalisation of Sec.
 * 3.1 steps 1-5, whose scheme is written for RK2.  Fluid 1 (the larger
 * step dt1) takes its first stage at t^n, sharing the cycle's first
 * interaction step with fluid 2's first sub-step; fluid 2 sub-cycles with
 * dt2, every one of its stage evaluations seeing fluid 1 by Eq. 7 between
 * its states at t^n and after its first stage; fluid 1's second stage
 * shares the last sub-step's second evaluation (both at t1 = t^n + dt1);
 * fluid 1's third stage is evaluated at t^n + dt1/2 on the level set
 * interpolated linearly between the two sub-step boundaries around that
 * time (with a single sub-step, dt1 = dt2, it shares fluid 2's third
 * evaluation instead, which makes that cycle the single-step method).  The
 * correction quantities collect b dt2 X_1 of every fluid-2 evaluation and
 * -b dt1 X_1 of every fluid-1 one (Eq. 8-9 with RK3's weights) and are
 * applied to fluid 1 at the end, before its mixing.  That would remove
 * the exchange flux of fluid 1's own third evaluation from its result
 * exactly (the flux enters only that last update), so that evaluation
 * carries none (eval_third). */
static void cycle_rk3(orc_ctx *o, int f1, double dt1, double dt2, orc_info *info) {
  const int f2 = 1 - f1;
  const double b12 = 1.0 / 6.0, b3 = 2.0 / 3.0;
  const double th = 0.5 * dt1;  /* fluid 1's third-stage time, from t^n */
  for (int m = 0; m < 3; m++) memset(o->xc[m], 0, sizeof(double) * o->NP);
  /* fluid-1 first stage with dt1; previous and future states */
  fv_rhs(o, f1, o->L[f1]);
  copy_planes(o, o->prev, o->q[f1], 4);
  for (int m = 0; m < 4; m++)
    rk_plane(o, 1, o->fut[m], o->prev[m], o->prev[m], o->L[f1][m], dt1, NULL);
  double t2 = 0.0, ta = 0.0, tb = 0.0;
  int sub = 0, have_a = 0, have_b = 0;
  double *qs[2][4];
  for (;;) {
    sub++;
    if (sub > 1) {
      interpolate(o, t2 / dt1);
      geometry(o, o->phi);
      mix(o, f1, o->qi);
      for (int m = 0; m < 4; m++) {
        qs[f1][m] = o->qi[m];
        qs[f2][m] = o->q[f2][m];
      }
      eval(o, qs, o->phi);
      dt2 = dt_of(o, f2);
    }
    int last = (dt1 - t2) <= dt2 * (1.0 + 1e-12);
    if (last) dt2 = dt1 - t2;
    const int single = sub == 1 && last;  /* dt1 = dt2: all shared */
    record_b(o, f1, sub == 1, b12, dt1, dt2);
    /* the sub-step that reaches fluid 1's third-stage time starts here */
    if (!have_a && (th < t2 + dt2 || last)) {
      memcpy(o->phia, o->phi, sizeof(double) * o->NP);
      ta = t2;
      have_a = 1;
    }
    /* stage 1 of fluid 2 and the level set */
    copy_planes(o, o->q0[f2], o->q[f2], 4);
    memcpy(o->phi0, o->phi, sizeof(double) * o->NP);
    make_band(o, o->phi0);
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    for (int m = 0; m < 4; m++)
      rk_plane(o, 1, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 1, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    geometry(o, o->phi);
    mix(o, f2, o->q[f2]);
    /* stage 2 at t2 + dt2: fluid 1 by Eq. 7, at t1 its future state */
    if (last) {
      mix(o, f1, o->fut);
      for (int m = 0; m < 4; m++) qs[f1][m] = o->fut[m];
    } else {
      interpolate(o, (t2 + dt2) / dt1);
      mix(o, f1, o->qi);
      for (int m = 0; m < 4; m++) qs[f1][m] = o->qi[m];
    }
    for (int m = 0; m < 4; m++) qs[f2][m] = o->q[f2][m];
    eval(o, qs, o->phi);
    record_b(o, f1, last, b12, dt1, dt2);
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    if (last) fv_rhs(o, f1, o->L[f1]);
    for (int m = 0; m < 4; m++)
      rk_plane(o, 2, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 2, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    if (last)
      for (int m = 0; m < 4; m++)
        rk_plane(o, 2, o->q[f1][m], o->prev[m], o->fut[m], o->L[f1][m], dt1, NULL);
    geometry(o, o->phi);
    mix(o, f2, o->q[f2]);
    /* (with more sub-steps fluid 1's second-stage state is mixed with the
     * geometry of its third stage, after the loop) */
    if (single) mix(o, f1, o->q[f1]);
    /* stage 3 at t2 + dt2/2: fluid 1 by Eq. 7 (with one sub-step its own
     * second-stage state, the evaluation being shared) */
    if (single) {
      for (int m = 0; m < 4; m++) qs[f1][m] = o->q[f1][m];
    } else {
      interpolate(o, (t2 + 0.5 * dt2) / dt1);
      mix(o, f1, o->qi);
      for (int m = 0; m < 4; m++) qs[f1][m] = o->qi[m];
    }
    for (int m = 0; m < 4; m++) qs[f2][m] = o->q[f2][m];
    eval(o, qs, o->phi);
    record_b(o, f1, single, b3, dt1, dt2);
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    if (single) fv_rhs(o, f1, o->L[f1]);
    for (int m = 0; m < 4; m++)
      rk_plane(o, 3, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 3, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    if (single)
      for (int m = 0; m < 4; m++)
        rk_plane(o, 3, o->q[f1][m], o->prev[m], o->q[f1][m], o->L[f1][m], dt1, NULL);
    reinit(o, o->phi);
    geometry(o, o->phi);
    mix(o, f2, o->q[f2]);
    /* the sub-step that reached fluid 1's third-stage time ends here */
    if (have_a && !have_b) {
      memcpy(o->phib, o->phi, sizeof(double) * o->NP);
      tb = t2 + dt2;
      have_b = 1;
    }
    if (last) break;
    t2 += dt2;
  }
  if (sub > 1) {
    /* fluid 1's third stage at t^n + dt1/2 on the level set interpolated
     * between the bracketing sub-step boundaries (a fluid-1-only
     * evaluation; fluid 1's second-stage state is mixed with its geometry) */
    double w = (th - ta) / (tb - ta);
    memcpy(o->phie, o->phi, sizeof(double) * o->NP);
    interp2(o, o->phi, o->phia, o->phib, w);
    geometry(o, o->phi);
    mix(o, f1, o->q[f1]);
    eval_third(o, f1, o->phi);
    fv_rhs(o, f1, o->L[f1]);
    for (int m = 0; m < 4; m++)
      rk_plane(o, 3, o->q[f1][m], o->prev[m], o->q[f1][m], o->L[f1][m], dt1, NULL);
    memcpy(o->phi, o->phie, sizeof(double) * o->NP);
    geometry(o, o->phi);
  }
  if (o->c.flux_correction) {
    double dxdy = o->c.dx * o->c.dy;
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j);
        for (int m = 0; m < 3; m++) o->q[f1][m + 1][c] += o->xc[m][c] / dxdy;
      }
  }
  mix(o, f1, o->q[f1]);
  o->t += dt1;
  if (info) {
    info->substeps = sub;
    info->t = o->t;
  }
}

int orc_step_multi_dt(orc_ctx *o, int ncycles, double t_end, orc_info *info) {
  long long open0 = o->open_updates;
  for (int n = 0; n < ncycles; n++) {
    if (t_end > 0.0 && o->t >= t_end) break;
    cycle(o, t_end, info);
  }
  if (info) {
    info->err = o->err;
    info->open_updates = o->open_updates - open0;
  }
  return o->err;
}

/* ------------------------------------------------------------------ */
/* context                                                             */

static double *plane(orc_ctx *o) { return (double *)calloc((size_t)o->NP, sizeof(double)); }

orc_ctx *orc_create(const orc_config *cfg) {
  if (cfg->nx < GH || (cfg->dim == 2 && cfg->ny < GH) || (cfg->dim == 1 && cfg->ny != 1))
    return NULL;
  if (cfg->rk_order != 2 && cfg->rk_order != 3) return NULL;
  if (cfg->weno_char != 0 && cfg->weno_char != 1) return NULL;
  if (cfg->flux != 0 && cfg->flux != 1) return NULL;
  if (cfg->flux == 1 && cfg->weno_char) return NULL;
  if (!(cfg->sigma >= 0.0) || !isfinite(cfg->sigma)) return NULL;
  for (int k = 0; k < 2; k++)
    if (!(cfg->mu[k] >= 0.0) || !isfinite(cfg->mu[k])) return NULL;
  for (int k = 0; k < 2; k++) {
    if (cfg->tait[k] != 0 && cfg->tait[k] != 1) return NULL;
    if (cfg->tait[k] && (!(cfg->tait_B[k] > 0.0) || !(cfg->tait_rho0[k] > 0.0) ||
                         !isfinite(cfg->tait_p0[k]) || !isfinite(cfg->tait_B[k])))
      return NULL;
  }
  orc_ctx *o = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  o->c = *cfg;
  /* a Tait fluid's sound speed is the stiffened gas's with pinf = B - p0 */
  for (int k = 0; k < 2; k++)
    if (o->c.tait[k]) o->c.pinf[k] = o->c.tait_B[k] - o->c.tait_p0[k];
  if (o->c.dim == 1) o->c.bc[2] = o->c.bc[3] = ORC_BC_ZEROGRAD;
  o->PX = cfg->nx + 2 * GH;
  o->PY = cfg->ny + 2 * GH;
  o->NP = o->PX * o->PY;
  o->h = cfg->dim == 2 ? dmin(cfg->dx, cfg->dy) : cfg->dx;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      o->q[k][m] = plane(o);
      o->w[k][m] = plane(o);
      o->q0[k][m] = plane(o);
      o->L[k][m] = plane(o);
    }
  for (int m = 0; m < 4; m++) {
    o->old[m] = plane(o);
    o->fx[m] = plane(o);
    o->fy[m] = plane(o);
    o->prev[m] = plane(o);
    o->fut[m] = plane(o);
    o->qi[m] = plane(o);
  }
  o->phia = plane(o);
  o->phib = plane(o);
  o->phie = plane(o);
  for (int m = 0; m < 3; m++) {
    o->xn[m] = plane(o);
    o->xp[m] = plane(o);
    o->xc[m] = plane(o);
  }
  o->ul[0] = plane(o);
  o->ul[1] = plane(o);
  o->phi = plane(o);
  o->alpha = plane(o);
  o->ax = plane(o);
  o->ay = plane(o);
  o->sx = plane(o);
  o->sy = plane(o);
  o->phi0 = plane(o);
  o->lphi = plane(o);
  o->p0 = plane(o);
  o->band = (unsigned char *)calloc((size_t)o->NP, 1);
  o->rext = (unsigned char *)calloc((size_t)o->NP, 1);
  o->nostate[0] = (unsigned char *)calloc((size_t)o->NP, 1);
  o->nostate[1] = (unsigned char *)calloc((size_t)o->NP, 1);
  return o;
}

void orc_destroy(orc_ctx *o) {
  if (!o) return;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      free(o->q[k][m]);
      free(o->w[k][m]);
      free(o->q0[k][m]);
      free(o->L[k][m]);
    }
  for (int m = 0; m < 4; m++) {
    free(o->old[m]);
    free(o->fx[m]);
    free(o->fy[m]);
    free(o->prev[m]);
    free(o->fut[m]);
    free(o->qi[m]);
  }
  free(o->phia);
  free(o->phib);
  free(o->phie);
  for (int m = 0; m < 3; m++) {
    free(o->xn[m]);
    free(o->xp[m]);
    free(o->xc[m]);
  }
  free(o->ul[0]);
  free(o->ul[1]);
  free(o->phi);
  free(o->alpha);
  free(o->ax);
  free(o->ay);
  free(o->sx);
  free(o->sy);
  free(o->phi0);
  free(o->lphi);
  free(o->p0);
  free(o->band);
  free(o->rext);
  free(o->nostate[0]);
  free(o->nostate[1]);
  free(o);
}

int orc_init(orc_ctx *o, const double *phi, const double *pN, const double *pP) {
  int nx = o->c.nx, ny = o->c.ny, n = nx * ny;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) o->phi[ID(o, i, j)] = phi[i + j * nx];
  geometry(o, o->phi);
  for (int k = 0; k < 2; k++) {
    const double *pr = k == 0 ? pN : pP;
    double g = o->c.gamma[k], pi = o->c.pinf[k];
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j), s = i + j * nx;
        double rho = pr[s], u = pr[n + s], v = pr[2 * n + s], p = pr[3 * n + s];
        o->w[k][0][c] = rho;
        o->w[k][1][c] = u;
        o->w[k][2][c] = v;
        o->w[k][3][c] = p;
        double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v);
        double a = vol(o, k, c);
        o->q[k][0][c] = a * rho;
        o->q[k][1][c] = a * (rho * u);
        o->q[k][2][c] = a * (rho * v);
        o->q[k][3][c] = a * E;
      }
  }
  mix(o, 0, o->q[0]);
  mix(o, 1, o->q[1]);
  o->t = 0.0;
  o->err = 0;
  return 0;
}

static void copy_out(const orc_ctx *o, const double *src, double *dst) {
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) dst[i + j * o->c.nx] = src[ID(o, i, j)];
}

static void copy_in(orc_ctx *o, const double *src, double *dst) {
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) dst[ID(o, i, j)] = src[i + j * o->c.nx];
}

int orc_get_state(const orc_ctx *o, double *qN, double *qP, double *phi) {
  int n = o->c.nx * o->c.ny;
  for (int m = 0; m < 4; m++) {
    if (qN) copy_out(o, o->q[0][m], qN + m * n);
    if (qP) copy_out(o, o->q[1][m], qP + m * n);
  }
  if (phi) copy_out(o, o->phi, phi);
  return 0;
}

int orc_set_state(orc_ctx *o, const double *qN, const double *qP, const double *phi) {
  int n = o->c.nx * o->c.ny;
  for (int m = 0; m < 4; m++) {
    if (qN) copy_in(o, qN + m * n, o->q[0][m]);
    if (qP) copy_in(o, qP + m * n, o->q[1][m]);
  }
  if (phi) copy_in(o, phi, o->phi);
  geometry(o, o->phi);
  return 0;
}

int orc_integrals(const orc_ctx *o, double *out) {
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) {
      double s = 0.0;
      for (int j = 0; j < o->c.ny; j++)
        for (int i = 0; i < o->c.nx; i++) s += o->q[k][m][ID(o, i, j)];
      out[k * 4 + m] = s * (o->c.dx * o->c.dy);
    }
  return 0;
}

double orc_curvature(orc_ctx *o, int i, int j) {
  fill_ghost(o, o->phi, 0);
  return curvature(o, o->phi, i, j);
}

double orc_time(const orc_ctx *o) { return o->t; }
int orc_status(const orc_ctx *o) { return o->err; }

int orc_geometry(orc_ctx *o, double *alpha, double *ax, double *ay, double *sx,
                 double *sy) {
  int nx = o->c.nx, ny = o->c.ny;
  geometry(o, o->phi);
  if (alpha) copy_out(o, o->alpha, alpha);
  if (sx) copy_out(o, o->sx, sx);
  if (sy) copy_out(o, o->sy, sy);
  if (ax)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i <= nx; i++) ax[i + j * (nx + 1)] = o->ax[ID(o, i, j)];
  if (ay)
    for (int j = 0; j <= ny; j++)
      for (int i = 0; i < nx; i++) ay[i + j * nx] = o->ay[ID(o, i, j)];
  return 0;
}

int orc_rhs(orc_ctx *o, int k, double *out) {
  int n = o->c.nx * o->c.ny;
  eval(o, o->q, o->phi);
  fv_rhs(o, k, o->L[k]);
  for (int m = 0; m < 4; m++) copy_out(o, o->L[k][m], out + m * n);
  return o->err;
}

int orc_stencil_states(orc_ctx *o, int k, double *out) {
  int n = o->c.nx * o->c.ny;
  eval(o, o->q, o->phi);
  for (int m = 0; m < 4; m++) copy_out(o, o->w[k][m], out + m * n);
  return o->err;
}

int orc_reinit_only(orc_ctx *o) {
  make_band(o, o->phi);
  reinit(o, o->phi);
  return 0;
}

int orc_mix_only(orc_ctx *o, int k) {
  geometry(o, o->phi);
  mix(o, k, o->q[k]);
  return 0;
}

/* ------------------------------------------------------------------ */
/* discrete adjoint of the single-time-step RK2 step with its schedule  */
/* frozen                                                               */
/*                                                                      */
/* The frozen step takes the step size, the Lax-Friedrichs speeds of    */
/* both stages and the level sets after stage 1 and after the step as   */
/* given, so every geometric decision (volume fractions, apertures,     */
/* interface vectors, extension and mixing targets and weights, which   */
/* cells are real) is fixed; what remains is a differentiable map of    */
/* the conserved states (alpha U)_k: primitive recovery, extension      */
/* (linear), the interface Riemann problem (implicit function of its    */
/* two side states), WENO5 with its nonlinear weights, the LF split     */
/* fluxes, the aperture-weighted divergence of Eq. 2, the RK2           */
/* combination and the mixing (linear).  The adjoint below is the       */
/* transpose of that map's Jacobian, written operation by operation in  */
/* reverse order.  Pins: central finite differences of the replayed     */
/* step (orc_replay_step), exact conservation identities of the         */
/* transposed step, and finite differences of the pointwise pieces.     */

int orc_step_taped(orc_ctx *o, double *dt_out, double *lf, double *phi1, double *phi2) {
  if (o->c.rk_order != 2) {
    o->err |= ORC_ERR_INVAL;
    return o->err;
  }
  eval(o, o->q, o->phi);
  double dt = dmin(dt_of(o, 0), dt_of(o, 1));
  step_record rec = {lf, phi1};
  single_step_after_eval(o, dt, &rec);
  *dt_out = dt;
  copy_out(o, o->phi, phi2);
  return o->err;
}

/* interaction step with the stage's Lax-Friedrichs speeds given */
static void eval_frozen(orc_ctx *o, double *const qs[2][4], const double *lf) {
  eval(o, qs, o->phi);
  for (int k = 0; k < 2; k++)
    for (int d = 0; d < 2; d++) o->lf[k][d] = lf[k * 2 + d];
}

/* stage s of the frozen step, ending with the level set phi_after in
 * place (geometry refreshed) and the mixing done */
static void frozen_stage(orc_ctx *o, int s, double dt, const double *lf, const double *phi_after) {
  eval_frozen(o, o->q, lf);
  for (int k = 0; k < 2; k++) fv_rhs(o, k, o->L[k]);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      rk_plane(o, s, o->q[k][m], o->q0[k][m], o->q[k][m], o->L[k][m], dt, NULL);
  copy_in(o, phi_after, o->phi);
  geometry(o, o->phi);
  mix(o, 0, o->q[0]);
  mix(o, 1, o->q[1]);
}

int orc_replay_step(orc_ctx *o, double dt, const double *lf, const double *phi1,
                    const double *phi2) {
  if (o->c.rk_order != 2) {
    o->err |= ORC_ERR_INVAL;
    return o->err;
  }
  for (int k = 0; k < 2; k++) copy_planes(o, o->q0[k], o->q[k], 4);
  frozen_stage(o, 1, dt, lf, phi1);
  frozen_stage(o, 2, dt, lf + 4, phi2);
  o->t += dt;
  return o->err;
}

/* d weno5 / d v, the nonlinear weights included */
void orc_weno5_grad(const double *v, double eps, double *g) {
  double v1 = v[0], v2 = v[1], v3 = v[2], v4 = v[3], v5 = v[4];
  double q[3] = {(2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0, (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0,
                 (2.0 * v3 + 5.0 * v4 - v5) / 6.0};
  static const double dq[3][5] = {{2.0 / 6.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0},
                                  {0.0, -1.0 / 6.0, 5.0 / 6.0, 2.0 / 6.0, 0.0},
                                  {0.0, 0.0, 2.0 / 6.0, 5.0 / 6.0, -1.0 / 6.0}};
  /* beta_i = 13/12 s_i^2 + 1/4 t_i^2 with s_i, t_i linear in v */
  static const double ds[3][5] = {{1, -2, 1, 0, 0}, {0, 1, -2, 1, 0}, {0, 0, 1, -2, 1}};
  static const double dt_[3][5] = {{1, -4, 3, 0, 0}, {0, 1, 0, -1, 0}, {0, 0, 3, -4, 1}};
  static const double d[3] = {0.1, 0.6, 0.3};
  double b[3], db[3][5], a[3], S = 0.0;
  for (int i = 0; i < 3; i++) {
    double si = 0.0, ti = 0.0;
    for (int r = 0; r < 5; r++) {
      si += ds[i][r] * v[r];
      ti += dt_[i][r] * v[r];
    }
    b[i] = 13.0 / 12.0 * si * si + 0.25 * ti * ti;
    for (int r = 0; r < 5; r++) db[i][r] = 13.0 / 6.0 * si * ds[i][r] + 0.5 * ti * dt_[i][r];
    a[i] = d[i] / sq(eps + b[i]);
    S += a[i];
  }
  double res = (a[0] * q[0] + a[1] * q[1] + a[2] * q[2]) / S;
  for (int r = 0; r < 5; r++) {
    double acc = 0.0;
    for (int i = 0; i < 3; i++) {
      double dai = -2.0 * a[i] / (eps + b[i]) * db[i][r];
      acc += a[i] * dq[i][r] + (q[i] - res) * dai;
    }
    g[r] = acc / S;
  }
}

/* side function of the Riemann problem and its partial derivatives with
 * respect to p, the side density and the side pressure */
static void side_grad(double p, double rho, double pk, double g, double pi, double *f,
                      double *fp, double *fr, double *fk) {
  double P = pk + pi, Pp = p + pi;
  double ck = sqrt(g * P / rho);
  if (p > pk) {
    double A = 2.0 / ((g + 1.0) * rho);
    double B = (g - 1.0) / (g + 1.0) * P;
    double qr = sqrt(A / (Pp + B));
    *f = (p - pk) * qr;
    *fp = qr * (1.0 - 0.5 * (p - pk) / (Pp + B));
    *fk = -qr - 0.5 * (p - pk) * qr / (Pp + B) * (g - 1.0) / (g + 1.0);
  } else {
    double r = Pp / P, e = (g - 1.0) / (2.0 * g);
    double re = pow(r, e);
    *f = 2.0 * ck / (g - 1.0) * (re - 1.0);
    *fp = 1.0 / (rho * ck) * pow(r, -(g + 1.0) / (2.0 * g));
    *fk = *f / (2.0 * P) - ck * re / (g * P);
  }
  *fr = -*f / (2.0 * rho);
}

/* vector-Jacobian product of (p*, u*) of the exact Riemann problem with
 * respect to (rho, u, p) of each side, by the implicit-function theorem
 * on f_L(p) + f_R(p) + u_R - u_L = 0 at the converged p*. */
int orc_riemann_grad(const double *L, const double *R, double lam_p, double lam_u, double *gL,
                     double *gR) {
  double out[7];
  int rc = orc_riemann(L, R, out);
  double p = out[0];
  double fL, fpL, frL, fkL, fR, fpR, frR, fkR;
  side_grad(p, L[0], L[2], L[3], L[4], &fL, &fpL, &frL, &fkL);
  side_grad(p, R[0], R[2], R[3], R[4], &fR, &fpR, &frR, &fkR);
  /* u* = (uL + uR)/2 + (fR - fL)/2 depends on p* as well */
  double lp = lam_p + lam_u * 0.5 * (fpR - fpL);
  double kappa = lp / (fpL + fpR);
  gL[0] = -0.5 * lam_u * frL - kappa * frL;
  gL[1] = 0.5 * lam_u + kappa;
  gL[2] = -0.5 * lam_u * fkL - kappa * fkL;
  gR[0] = 0.5 * lam_u * frR - kappa * frR;
  gR[1] = 0.5 * lam_u - kappa;
  gR[2] = 0.5 * lam_u * fkR - kappa * fkR;
  return rc;
}

/* transpose of the split flux: lam_fp, lam_fm at one cell into the
 * primitive adjoint lw of that cell (direction d, LF speed a) */
static void split_T(const orc_ctx *o, int k, const double *const W[4], int c, int d, double a,
                    const double *lfp, const double *lfm, double *const lw[4]) {
  double g = o->c.gamma[k], pi = o->c.pinf[k];
  double rho = W[0][c], u = W[1][c], v = W[2][c], p = W[3][c];
  double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v);
  double lF[4], lU[4];
  for (int m = 0; m < 4; m++) {
    lF[m] = 0.5 * (lfp[m] + lfm[m]);
    lU[m] = 0.5 * a * (lfp[m] - lfm[m]);
  }
  double ke = 0.5 * (u * u + v * v);
  /* U = (rho, rho u, rho v, E) */
  double gr = lU[0] + lU[1] * u + lU[2] * v + lU[3] * ke;
  double gu = lU[1] * rho + lU[3] * rho * u;
  double gv = lU[2] * rho + lU[3] * rho * v;
  double gp = lU[3] / (g - 1.0);
  if (d == 0) {
    /* F = (rho u, rho u^2 + p, rho u v, u (E + p)) */
    gr += lF[0] * u + lF[1] * u * u + lF[2] * u * v + lF[3] * u * ke;
    gu += lF[0] * rho + lF[1] * 2.0 * rho * u + lF[2] * rho * v + lF[3] * (E + p + rho * u * u);
    gv += lF[2] * rho * u + lF[3] * rho * u * v;
    gp += lF[1] + lF[3] * u * (1.0 / (g - 1.0) + 1.0);
  } else {
    /* F = (rho v, rho u v, rho v^2 + p, v (E + p)) */
    gr += lF[0] * v + lF[1] * u * v + lF[2] * v * v + lF[3] * v * ke;
    gu += lF[1] * rho * v + lF[3] * rho * u * v;
    gv += lF[0] * rho + lF[1] * rho * u + lF[2] * 2.0 * rho * v + lF[3] * (E + p + rho * v * v);
    gp += lF[2] + lF[3] * v * (1.0 / (g - 1.0) + 1.0);
  }
  lw[0][c] += gr;
  lw[1][c] += gu;
  lw[2][c] += gv;
  lw[3][c] += gp;
}

/* transpose of the face flux of direction d (stride s, spacing hd) at the
 * face between cells c - s and c, weighted by lam_F (4 components) */
static void face_flux_T(const orc_ctx *o, int k, const double *const W[4], int c, int s, int d,
                        double a, const double *lamF, double *const lw[4]) {
  double g = o->c.gamma[k], pi = o->c.pinf[k];
  double fp[6][4], fm[6][4];
  for (int r = 0; r < 6; r++) {
    int cc = c + (r - 3) * s;
    double rho = W[0][cc], u = W[1][cc], v = W[2][cc], p = W[3][cc];
    double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v);
    double U[4] = {rho, rho * u, rho * v, E}, F[4];
    if (d == 0) {
      F[0] = rho * u;
      F[1] = rho * u * u + p;
      F[2] = rho * u * v;
      F[3] = u * (E + p);
    } else {
      F[0] = rho * v;
      F[1] = rho * u * v;
      F[2] = rho * v * v + p;
      F[3] = v * (E + p);
    }
    for (int m = 0; m < 4; m++) {
      fp[r][m] = 0.5 * (F[m] + a * U[m]);
      fm[r][m] = 0.5 * (F[m] - a * U[m]);
    }
  }
  double lfp[6][4] = {{0}}, lfm[6][4] = {{0}};
  for (int m = 0; m < 4; m++) {
    double vp[5] = {fp[0][m], fp[1][m], fp[2][m], fp[3][m], fp[4][m]};
    double vm[5] = {fm[5][m], fm[4][m], fm[3][m], fm[2][m], fm[1][m]};
    double gp[5], gm[5];
    orc_weno5_grad(vp, o->c.weno_eps, gp);
    orc_weno5_grad(vm, o->c.weno_eps, gm);
    for (int r = 0; r < 5; r++) {
      lfp[r][m] += lamF[m] * gp[r];
      lfm[5 - r][m] += lamF[m] * gm[r];
    }
  }
  for (int r = 0; r < 6; r++) split_T(o, k, W, c + (r - 3) * s, d, a, lfp[r], lfm[r], lw);
}

/* transpose of the aperture-weighted flux divergence of Eq. 2 for fluid k:
 * mu (4 planes) is the adjoint of L_k; accumulates into lw (4 padded
 * planes, ghost cells included) */
static void fluxdiv_T(orc_ctx *o, int k, const double *const W[4], const double *lf,
                      double *const mu[4], double *const lw[4]) {
  int nx = o->c.nx, ny = o->c.ny;
  double lamF[4];
  for (int j = 0; j < ny; j++)
    for (int i = 0; i <= nx; i++) {
      int c = ID(o, i, j);
      double A = k == 1 ? o->ax[c] : 1.0 - o->ax[c];
      if (A == 0.0) continue;
      for (int m = 0; m < 4; m++) {
        double r = i < nx ? mu[m][c] : 0.0, l = i > 0 ? mu[m][c - 1] : 0.0;
        lamF[m] = A * (r - l) / o->c.dx;
      }
      face_flux_T(o, k, W, c, 1, 0, lf[0], lamF, lw);
    }
  if (o->c.dim == 2)
    for (int j = 0; j <= ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j);
        double A = k == 1 ? o->ay[c] : 1.0 - o->ay[c];
        if (A == 0.0) continue;
        for (int m = 0; m < 4; m++) {
          double r = j < ny ? mu[m][c] : 0.0, l = j > 0 ? mu[m][c - o->PX] : 0.0;
          lamF[m] = A * (r - l) / o->c.dy;
        }
        face_flux_T(o, k, W, c, o->PX, 1, lf[1], lamF, lw);
      }
}

/* transpose of fill_ghost: ghost adjoints move back to the interior cells
 * they were copied from (the y pass first, as it ran last) */
static void ghost_T(orc_ctx *o, double *a, int vel) {
  int nx = o->c.nx, ny = o->c.ny;
  for (int i = -GH; i < nx + GH; i++)
    for (int m = 0; m < GH; m++) {
      double sb = (vel == 2 && o->c.bc[2] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      double st = (vel == 2 && o->c.bc[3] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      int jb, jt;
      switch (o->c.bc[2]) {
        case ORC_BC_REFLECT: jb = m; break;
        case ORC_BC_PERIODIC: jb = ny - 1 - m; break;
        default: jb = 0;
      }
      switch (o->c.bc[3]) {
        case ORC_BC_REFLECT: jt = ny - 1 - m; break;
        case ORC_BC_PERIODIC: jt = m; break;
        default: jt = ny - 1;
      }
      double gb = a[ID(o, i, -1 - m)], gt = a[ID(o, i, ny + m)];
      a[ID(o, i, -1 - m)] = 0.0;
      a[ID(o, i, ny + m)] = 0.0;
      a[ID(o, i, jb)] += sb * gb;
      a[ID(o, i, jt)] += st * gt;
    }
  for (int j = 0; j < ny; j++)
    for (int m = 0; m < GH; m++) {
      double sl = (vel == 1 && o->c.bc[0] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      double sr = (vel == 1 && o->c.bc[1] == ORC_BC_REFLECT) ? -1.0 : 1.0;
      int il, ir;
      switch (o->c.bc[0]) {
        case ORC_BC_REFLECT: il = m; break;
        case ORC_BC_PERIODIC: il = nx - 1 - m; break;
        default: il = 0;
      }
      switch (o->c.bc[1]) {
        case ORC_BC_REFLECT: ir = nx - 1 - m; break;
        case ORC_BC_PERIODIC: ir = m; break;
        default: ir = nx - 1;
      }
      double gl = a[ID(o, -1 - m, j)], gr = a[ID(o, nx + m, j)];
      a[ID(o, -1 - m, j)] = 0.0;
      a[ID(o, nx + m, j)] = 0.0;
      a[ID(o, il, j)] += sl * gl;
      a[ID(o, ir, j)] += sr * gr;
    }
}

/* transpose of the interface exchange: mu_N, mu_P are the adjoints of the
 * right-hand sides; the Riemann problem's side states are the stencil
 * states of both fluids at each cut cell */
static void interface_T(orc_ctx *o, double *const W[2][4], double *const mu[2][4],
                        double *const lw[2][4]) {
  double dxdy = o->c.dx * o->c.dy;
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      double Sx = o->sx[c], Sy = o->sy[c];
      if (Sx == 0.0 && Sy == 0.0) continue;
      double Sm = sqrt(Sx * Sx + Sy * Sy);
      double nxv, nyv;
      normal(o, o->phi, i, j, &nxv, &nyv);
      if (nxv == 0.0 && nyv == 0.0) {
        nxv = Sx / Sm;
        nyv = Sy / Sm;
      }
      double L[5] = {W[0][0][c], W[0][1][c] * nxv + W[0][2][c] * nyv, W[0][3][c],
                     o->c.gamma[0], o->c.pinf[0]};
      double R[5] = {W[1][0][c], W[1][1][c] * nxv + W[1][2][c] * nyv, W[1][3][c],
                     o->c.gamma[1], o->c.pinf[1]};
      double out[7];
      orc_riemann(L, R, out);
      double ps = out[0], us = out[1];
      /* X as applied to fluid N enters L_N with +1/dxdy and L_P with -1/dxdy */
      double lx0 = (mu[0][1][c] - mu[1][1][c]) / dxdy;
      double lx1 = (mu[0][2][c] - mu[1][2][c]) / dxdy;
      double lx2 = (mu[0][3][c] - mu[1][3][c]) / dxdy;
      double lam_p = -Sx * lx0 - Sy * lx1 - us * Sm * lx2;
      double lam_u = -ps * Sm * lx2;
      double gL[3], gR[3];
      orc_riemann_grad(L, R, lam_p, lam_u, gL, gR);
      lw[0][0][c] += gL[0];
      lw[0][1][c] += gL[1] * nxv;
      lw[0][2][c] += gL[1] * nyv;
      lw[0][3][c] += gL[2];
      lw[1][0][c] += gR[0];
      lw[1][1][c] += gR[1] * nxv;
      lw[1][2][c] += gR[1] * nyv;
      lw[1][3][c] += gR[2];
    }
}

/* transpose of the extension sweeps of fluid k (each sweep is the same
 * linear map: targets take the upwind-weighted mean of their upwind
 * neighbours, every other cell keeps its value) */
static void extend_T(orc_ctx *o, int k, double *const lw[4]) {
  double bw = o->c.band * o->h;
  const double *p = o->phi;
  for (int it = 0; it < o->c.ext_iters; it++) {
    for (int m = 0; m < 4; m++) memcpy(o->old[m], lw[m], sizeof(double) * o->NP);
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j);
        if (!(fabs(p[c]) < bw) || is_real(o, k, c)) continue;
        double nxv, nyv;
        normal(o, p, i, j, &nxv, &nyv);
        if (k == 0) {
          nxv = -nxv;
          nyv = -nyv;
        }
        int sx = nxv >= 0.0 ? 1 : -1, sy = nyv >= 0.0 ? 1 : -1;
        double wx = fabs(nxv) / o->c.dx;
        double wy = o->c.dim == 2 ? fabs(nyv) / o->c.dy : 0.0;
        if (!inside(o, i + sx, j)) wx = 0.0;
        if (!inside(o, i, j + sy)) wy = 0.0;
        double den = wx + wy;
        if (!(den > 0.0)) continue;
        /* the target's own value is overwritten: its adjoint moves to the
         * neighbours it was computed from */
        for (int m = 0; m < 4; m++) lw[m][c] -= o->old[m][c];
        for (int m = 0; m < 4; m++) {
          if (wx > 0.0) lw[m][ID(o, i + sx, j)] += wx / den * o->old[m][c];
          if (wy > 0.0) lw[m][ID(o, i, j + sy)] += wy / den * o->old[m][c];
        }
      }
  }
}

/* transpose of the primitive recovery of fluid k at its real cells; the
 * stencil states of other cells are extension or carried values, whose
 * adjoint ends here */
static void prim_T(orc_ctx *o, int k, const double *const W[4], double *const lw[4],
                   double *const lq[4]) {
  double g = o->c.gamma[k];
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      double a = vol(o, k, c);
      for (int m = 0; m < 4; m++) lq[m][c] = 0.0;
      if (!is_real(o, k, c)) continue;
      double rho = W[0][c], u = W[1][c], v = W[2][c];
      double lr = lw[0][c], lu = lw[1][c], lv = lw[2][c], lp = lw[3][c];
      double m0 = a * rho;
      lq[0][c] = lr / a - (lu * u + lv * v) / m0 + lp * (g - 1.0) * 0.5 * (u * u + v * v) / a;
      lq[1][c] = lu / m0 - lp * (g - 1.0) * u / a;
      lq[2][c] = lv / m0 - lp * (g - 1.0) * v / a;
      lq[3][c] = lp * (g - 1.0) / a;
    }
}

/* transpose of mixing fluid k (its incoming adjoint lam, in place); the
 * mixing is linear in the state, and a small cell with no fluid and no
 * content would mix as any other once it had content, so it is included */
static void mix_T(orc_ctx *o, int k, double *const lam[4]) {
  for (int m = 0; m < 4; m++) memcpy(o->old[m], lam[m], sizeof(double) * o->NP);
  for (int j = 0; j < o->c.ny; j++)
    for (int i = 0; i < o->c.nx; i++) {
      int c = ID(o, i, j);
      double as = vol(o, k, c);
      if (as >= o->c.mix_alpha) continue;
      int tcs[3];
      double betas[3];
      int nt = mix_targets(o, k, i, j, tcs, betas);
      for (int t = 0; t < nt; t++) {
        int tc = tcs[t];
        double beta = betas[t];
        double at = vol(o, k, tc);
        double den = as * beta + at;
        for (int m = 0; m < 4; m++) {
          /* M = beta (q_t as - q_s at) / den adds to the source and
           * subtracts at the target */
          double dM = o->old[m][c] - o->old[m][tc];
          lam[m][tc] += dM * beta * as / den;
          lam[m][c] -= dM * beta * at / den;
        }
      }
    }
}

/* adjoint of the right-hand sides of both fluids at the stage whose
 * stencil states are W (ghosts filled) and whose geometry is in place:
 * mu (adjoint of L, both fluids) -> lq (adjoint of the stage state) */
static void rhs_T(orc_ctx *o, double *const W[2][4], const double *lf, double *const mu[2][4],
                  double *const lw[2][4], double *const lq[2][4]) {
  static const int vel[4] = {0, 1, 2, 0};
  for (int k = 0; k < 2; k++) {
    for (int m = 0; m < 4; m++) memset(lw[k][m], 0, sizeof(double) * o->NP);
    fluxdiv_T(o, k, (const double *const *)W[k], lf + 2 * k, mu[k], lw[k]);
    for (int m = 0; m < 4; m++) ghost_T(o, lw[k][m], vel[m]);
  }
  interface_T(o, W, mu, lw);
  for (int k = 0; k < 2; k++) {
    extend_T(o, k, lw[k]);
    prim_T(o, k, (const double *const *)W[k], lw[k], lq[k]);
  }
}

int orc_adjoint_step(orc_ctx *o, double dt, const double *lf, const double *phi1,
                     const double *phi2, const double *lam_in, double *lam_out) {
  /* the adjoint is written for the component-wise reconstruction without
   * surface tension */
  if (o->c.rk_order != 2 || o->c.weno_char || o->c.flux || o->c.sigma != 0.0 ||
      o->c.mu[0] != 0.0 || o->c.mu[1] != 0.0) {
    o->err |= ORC_ERR_INVAL;
    return o->err;
  }
  int n = o->c.nx * o->c.ny;
  double *Qn[2][4], *W1[2][4], *W2[2][4], *lam[2][4], *ls[2][4], *mu[2][4], *lw[2][4],
      *lq[2][4], *lnew[2][4];
  double **all[9] = {&Qn[0][0], &W1[0][0], &W2[0][0], &lam[0][0], &ls[0][0],
                     &mu[0][0], &lw[0][0], &lq[0][0], &lnew[0][0]};
  for (int a = 0; a < 9; a++)
    for (int x = 0; x < 8; x++) all[a][x] = plane(o);
  double *phin = plane(o);
  unsigned char *ns1[2], *ns2[2];
  for (int k = 0; k < 2; k++) {
    ns1[k] = (unsigned char *)malloc((size_t)o->NP);
    ns2[k] = (unsigned char *)malloc((size_t)o->NP);
  }
  double t0 = o->t;
  for (int k = 0; k < 2; k++) copy_planes(o, Qn[k], o->q[k], 4);
  memcpy(phin, o->phi, sizeof(double) * o->NP);

  /* forward, keeping the stencil states of both stages */
  for (int k = 0; k < 2; k++) copy_planes(o, o->q0[k], o->q[k], 4);
  eval_frozen(o, o->q, lf);
  for (int k = 0; k < 2; k++) fv_rhs(o, k, o->L[k]);
  for (int k = 0; k < 2; k++) copy_planes(o, W1[k], o->w[k], 4);
  for (int k = 0; k < 2; k++) memcpy(ns1[k], o->nostate[k], (size_t)o->NP);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      rk_plane(o, 1, o->q[k][m], o->q0[k][m], o->q[k][m], o->L[k][m], dt, NULL);
  copy_in(o, phi1, o->phi);
  geometry(o, o->phi);
  mix(o, 0, o->q[0]);
  mix(o, 1, o->q[1]);
  eval_frozen(o, o->q, lf + 4);
  for (int k = 0; k < 2; k++) fv_rhs(o, k, o->L[k]);
  for (int k = 0; k < 2; k++) copy_planes(o, W2[k], o->w[k], 4);
  for (int k = 0; k < 2; k++) memcpy(ns2[k], o->nostate[k], (size_t)o->NP);

  /* reverse */
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) copy_in(o, lam_in + (k * 4 + m) * n, lam[k][m]);
  /* Q^{n+1} = mix_2(Q**) */
  copy_in(o, phi2, o->phi);
  geometry(o, o->phi);
  mix_T(o, 0, lam[0]);
  mix_T(o, 1, lam[1]);
  /* Q** = Q^n / 2 + (Q1 + dt L(Q1)) / 2 */
  copy_in(o, phi1, o->phi);
  geometry(o, o->phi);
  for (int k = 0; k < 2; k++) memcpy(o->nostate[k], ns2[k], (size_t)o->NP);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      for (int c = 0; c < o->NP; c++) mu[k][m][c] = 0.5 * dt * lam[k][m][c];
  rhs_T(o, W2, lf + 4, mu, lw, lq);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      for (int c = 0; c < o->NP; c++) ls[k][m][c] = 0.5 * lam[k][m][c] + lq[k][m][c];
  /* Q1 = mix_1(Q*) */
  mix_T(o, 0, ls[0]);
  mix_T(o, 1, ls[1]);
  /* Q* = Q^n + dt L(Q^n) */
  memcpy(o->phi, phin, sizeof(double) * o->NP);
  geometry(o, o->phi);
  for (int k = 0; k < 2; k++) memcpy(o->nostate[k], ns1[k], (size_t)o->NP);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      for (int c = 0; c < o->NP; c++) mu[k][m][c] = dt * ls[k][m][c];
  rhs_T(o, W1, lf, mu, lw, lq);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      for (int c = 0; c < o->NP; c++)
        lnew[k][m][c] = 0.5 * lam[k][m][c] + ls[k][m][c] + lq[k][m][c];
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) copy_out(o, lnew[k][m], lam_out + (k * 4 + m) * n);

  /* the context's state is left as it was */
  for (int k = 0; k < 2; k++) copy_planes(o, o->q[k], Qn[k], 4);
  memcpy(o->phi, phin, sizeof(double) * o->NP);
  geometry(o, o->phi);
  o->t = t0;
  for (int a = 0; a < 9; a++)
    for (int x = 0; x < 8; x++) free(all[a][x]);
  free(phin);
  for (int k = 0; k < 2; k++) {
    free(ns1[k]);
    free(ns2[k]);
  }
  return o->err;
}

/* right-hand sides of both fluids at the current state with the
 * Lax-Friedrichs speeds lf[4] (fluid*2 + direction) given, and the
 * transpose of their Jacobian: the stage-level pieces of the adjoint */
int orc_rhs_frozen(orc_ctx *o, const double *lf, double *out) {
  int n = o->c.nx * o->c.ny;
  eval_frozen(o, o->q, lf);
  for (int k = 0; k < 2; k++) {
    fv_rhs(o, k, o->L[k]);
    for (int m = 0; m < 4; m++) copy_out(o, o->L[k][m], out + (k * 4 + m) * n);
  }
  return o->err;
}

int orc_rhs_adjoint(orc_ctx *o, const double *lf, const double *mu_in, double *lq_out) {
  if (o->c.weno_char || o->c.flux || o->c.sigma != 0.0 || o->c.mu[0] != 0.0 ||
      o->c.mu[1] != 0.0) {
    o->err |= ORC_ERR_INVAL;
    return o->err;
  }
  int n = o->c.nx * o->c.ny;
  double *W[2][4], *mu[2][4], *lw[2][4], *lq[2][4];
  double **all[4] = {&W[0][0], &mu[0][0], &lw[0][0], &lq[0][0]};
  for (int a = 0; a < 4; a++)
    for (int x = 0; x < 8; x++) all[a][x] = plane(o);
  eval_frozen(o, o->q, lf);
  for (int k = 0; k < 2; k++) fv_rhs(o, k, o->L[k]);
  for (int k = 0; k < 2; k++) copy_planes(o, W[k], o->w[k], 4);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) copy_in(o, mu_in + (k * 4 + m) * n, mu[k][m]);
  rhs_T(o, W, lf, mu, lw, lq);
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) copy_out(o, lq[k][m], lq_out + (k * 4 + m) * n);
  for (int a = 0; a < 4; a++)
    for (int x = 0; x < 8; x++) free(all[a][x]);
  return o->err;
}

/* transpose of mixing fluid k with the current geometry: lam (4 planes of
 * nx*ny) in place */
int orc_mix_adjoint(orc_ctx *o, int k, double *lam) {
  int n = o->c.nx * o->c.ny;
  double *l[4];
  for (int m = 0; m < 4; m++) {
    l[m] = plane(o);
    copy_in(o, lam + m * n, l[m]);
  }
  geometry(o, o->phi);
  mix_T(o, k, l);
  for (int m = 0; m < 4; m++) {
    copy_out(o, l[m], lam + m * n);
    free(l[m]);
  }
  return 0;
}

/* transpose of the initialisation (alpha U from primitive fields, then
 * mixing) with the current level set: lam_q (8 planes) -> lam_prim (8
 * planes: rho, u, v, p of fluid N, then of fluid P) */
int orc_adjoint_init(orc_ctx *o, const double *pN, const double *pP, const double *lam_q,
                     double *lam_prim) {
  int nx = o->c.nx, ny = o->c.ny, n = nx * ny;
  double *l[2][4];
  geometry(o, o->phi);
  for (int k = 0; k < 2; k++) {
    for (int m = 0; m < 4; m++) {
      l[k][m] = plane(o);
      copy_in(o, lam_q + (k * 4 + m) * n, l[k][m]);
    }
    mix_T(o, k, l[k]);
  }
  for (int k = 0; k < 2; k++) {
    const double *pr = k == 0 ? pN : pP;
    double g = o->c.gamma[k];
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j), s = i + j * nx;
        double rho = pr[s], u = pr[n + s], v = pr[2 * n + s];
        double a = vol(o, k, c);
        double l0 = l[k][0][c], l1 = l[k][1][c], l2 = l[k][2][c], l3 = l[k][3][c];
        double *out = lam_prim + k * 4 * n;
        out[s] = a * (l0 + l1 * u + l2 * v + l3 * 0.5 * (u * u + v * v));
        out[n + s] = a * (l1 * rho + l3 * rho * u);
        out[2 * n + s] = a * (l2 * rho + l3 * rho * v);
        out[3 * n + s] = a * l3 / (g - 1.0);
      }
    for (int m = 0; m < 4; m++) free(l[k][m]);
  }
  return 0;
}
