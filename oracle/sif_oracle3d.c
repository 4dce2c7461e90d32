/*
 * sif_oracle3d.c -- plain, slow, serial FP64 oracle of the method in three
 * dimensions (Long, Cai & Pan, arXiv 1905.03917: Eq. 2 with a third pair of
 * faces, the level set of Eq. 6 in 3D, the accelerated cycle of Sec. 3.1;
 * the paper's 3D cases are the rows "Uniform grid - 3D" of Tables 1, 3, 4).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests and the CPU-baseline leg of
 * bench.py, never by the product path.  Compile with -O2 -ffp-contract=off.
 *
 * The paper runs its 3D cases with the same method and gives no formula of
 * its own for the third direction; every step here is the two-dimensional
 * oracle's with a z index added, except where a reading is needed:
 *   corner values -- the mean of the eight cells sharing the corner;
 *   face apertures -- the square's polygon area fraction of the 2D oracle
 *       over each face's four corner values;
 *   interface vector S -- the closure of the P region's faces, S_d = (A_d+
 *       - A_d-) times the face area (N to P, as in 2D);
 *   volume fraction -- the divergence theorem over the P region of the unit
 *       cell, alpha = (A_x+ + A_y+ + A_z+ - xi_m . s) / 3, with the interface
 *       patch taken as planar through the mean xi_m of its edge crossings
 *       (exact for a planar interface, equal to the 2D polygon area for a
 *       level set that does not vary along z);
 *   surface tension -- Eq. 10's jump sigma kappa with kappa the mean
 *       curvature div(grad phi / |grad phi|) by central differences, as in
 *       2D with the third axis's terms;
 *   viscosity -- the 2D oracle's face fluxes, interface traction and time
 *       step limit with the third velocity component and direction;
 *   mixing targets -- the seven neighbours toward the fluid along n_k (x, y,
 *       z, the three face diagonals and the cube diagonal) with weights
 *       n_x^2, n_y^2, n_z^2, |n_x n_y|, |n_x n_z|, |n_y n_z|, |n_x n_y
 *       n_z|^(2/3), which reduce to the 2D weights where n_z = 0; the
 *       fallbacks are the 2D ones over the 26 neighbours.
 * Pins (tests/test_oracle3d.py): exact half-space volumes and cut areas of
 * random planes, the 2D reduction of a z-invariant level set, sphere volume
 * and area convergence, the z-invariant reduction of a whole step to the 2D
 * oracle's step, the planar tube along each axis against the 1D oracle,
 * the permuted result of a case with permuted axes, exact conservation with
 * the correction (and its loss without it), the bitwise ratio-one reduction
 * of the accelerated cycle, and each fluid's mean velocity in uniform flow
 * past the droplet.
 * Parity unpinned beyond those: the weights of the mixing targets off the
 * coordinate planes (n_z != 0), a reading that only conservation and the
 * permutation test constrain.
 */
#include "sif_oracle3d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define GH 3
#define ALPHA_REAL 1e-6
#define NC 5 /* components: mass, x-, y-, z-momentum, energy */

struct orc3_ctx {
  orc3_config c;
  int PX, PY, PZ, NP;
  double h; /* min(dx, dy, dz) */
  double *q[2][NC];
  double *w[2][NC];  /* stencil states: rho, u, v, w, p */
  double *phi;
  double *alpha, *ax, *ay, *az, *sx, *sy, *sz;
  double *xn[4], *xp[4]; /* exchange X applied to fluid N / P */
  double *ul[3];
  double smax[2], lf[2][3];
  double t;
  int err;
  long long open_updates;
  double *q0[2][NC], *L[2][NC], *old[NC], *fl[3][NC];
  double *prev[NC], *fut[NC], *qi[NC], *xc[4];
  double *phi0, *lphi, *p0;
  unsigned char *band, *rext, *nostate[2];
};

#define ID(o, i, j, k) (((i) + GH) + (o)->PX * (((j) + GH) + (o)->PY * ((k) + GH)))

static double sq(double a) { return a * a; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* ------------------------------------------------------------------ */
/* ghost layers: x ghosts of interior (y, z) lines, then y ghosts of every
 * x including its ghosts, then z ghosts of every (x, y) including ghosts.
 * vel = d + 1 marks the velocity component odd at walls normal to d. */

static double ghost_src(const orc3_ctx *o, const double *a, int d, int side, int m, int i,
                        int j, int k, double *sgn, int vel) {
  int n = d == 0 ? o->c.nx : d == 1 ? o->c.ny : o->c.nz;
  int bc = o->c.bc[2 * d + side];
  int s;
  if (bc == ORC_BC_REFLECT)
    s = side == 0 ? m : n - 1 - m;
  else if (bc == ORC_BC_PERIODIC)
    s = side == 0 ? n - 1 - m : m;
  else
    s = side == 0 ? 0 : n - 1;
  *sgn = (vel == d + 1 && bc == ORC_BC_REFLECT) ? -1.0 : 1.0;
  if (d == 0) return a[ID(o, s, j, k)];
  if (d == 1) return a[ID(o, i, s, k)];
  return a[ID(o, i, j, s)];
}

static void fill_ghost(orc3_ctx *o, double *a, int vel) {
  int nx = o->c.nx, ny = o->c.ny, nz = o->c.nz;
  double sg, v;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int m = 0; m < GH; m++) {
        v = ghost_src(o, a, 0, 0, m, 0, j, k, &sg, vel);
        a[ID(o, -1 - m, j, k)] = sg < 0 ? -v : v;
        v = ghost_src(o, a, 0, 1, m, 0, j, k, &sg, vel);
        a[ID(o, nx + m, j, k)] = sg < 0 ? -v : v;
      }
  for (int k = 0; k < nz; k++)
    for (int i = -GH; i < nx + GH; i++)
      for (int m = 0; m < GH; m++) {
        v = ghost_src(o, a, 1, 0, m, i, 0, k, &sg, vel);
        a[ID(o, i, -1 - m, k)] = sg < 0 ? -v : v;
        v = ghost_src(o, a, 1, 1, m, i, 0, k, &sg, vel);
        a[ID(o, i, ny + m, k)] = sg < 0 ? -v : v;
      }
  for (int j = -GH; j < ny + GH; j++)
    for (int i = -GH; i < nx + GH; i++)
      for (int m = 0; m < GH; m++) {
        v = ghost_src(o, a, 2, 0, m, i, j, 0, &sg, vel);
        a[ID(o, i, j, -1 - m)] = sg < 0 ? -v : v;
        v = ghost_src(o, a, 2, 1, m, i, j, 0, &sg, vel);
        a[ID(o, i, j, nz + m)] = sg < 0 ? -v : v;
      }
}

/* ------------------------------------------------------------------ */
/* geometry (Sec. 2.1, Fig. 1, with a third pair of faces)              */

double orc3_cell_alpha(const double *c, double *s) {
  /* face apertures of the unit cube, each the square's area fraction over
   * its four corners counter-clockwise in the face's own (a, b) axes */
#define C(i, j, k) c[(i) + 2 * (j) + 4 * (k)]
  double axm = orc_cell_alpha(C(0, 0, 0), C(0, 1, 0), C(0, 1, 1), C(0, 0, 1));
  double axp = orc_cell_alpha(C(1, 0, 0), C(1, 1, 0), C(1, 1, 1), C(1, 0, 1));
  double aym = orc_cell_alpha(C(0, 0, 0), C(1, 0, 0), C(1, 0, 1), C(0, 0, 1));
  double ayp = orc_cell_alpha(C(0, 1, 0), C(1, 1, 0), C(1, 1, 1), C(0, 1, 1));
  double azm = orc_cell_alpha(C(0, 0, 0), C(1, 0, 0), C(1, 1, 0), C(0, 1, 0));
  double azp = orc_cell_alpha(C(0, 0, 1), C(1, 0, 1), C(1, 1, 1), C(0, 1, 1));
  s[0] = axp - axm;
  s[1] = ayp - aym;
  s[2] = azp - azm;
  int npos = 0;
  for (int v = 0; v < 8; v++) npos += c[v] >= 0.0;
  if (npos == 8) return 1.0;
  if (npos == 0) return 0.0;
  /* mean of the crossings on the twelve edges (phi linear along an edge) */
  double m[3] = {0.0, 0.0, 0.0};
  int nc = 0;
  for (int d = 0; d < 3; d++)
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        int lo[3], hi[3];
        /* the edge along d with the other two coordinates a, b */
        int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
        lo[d] = 0;
        hi[d] = 1;
        lo[e1] = hi[e1] = a;
        lo[e2] = hi[e2] = b;
        double va = C(lo[0], lo[1], lo[2]), vb = C(hi[0], hi[1], hi[2]);
        if ((va >= 0.0) == (vb >= 0.0)) continue;
        double t = va / (va - vb);
        double xi[3];
        xi[d] = t;
        xi[e1] = a;
        xi[e2] = b;
        for (int q = 0; q < 3; q++) m[q] += xi[q];
        nc++;
      }
#undef C
  for (int q = 0; q < 3; q++) m[q] /= nc;
  double al = (axp + ayp + azp - (m[0] * s[0] + m[1] * s[1] + m[2] * s[2])) / 3.0;
  if (al < 0.0) al = 0.0;
  if (al > 1.0) al = 1.0;
  return al;
}

static double corner(const orc3_ctx *o, const double *p, int i, int j, int k) {
  return 0.125 * (((p[ID(o, i - 1, j - 1, k - 1)] + p[ID(o, i, j - 1, k - 1)]) +
                   (p[ID(o, i - 1, j, k - 1)] + p[ID(o, i, j, k - 1)])) +
                  ((p[ID(o, i - 1, j - 1, k)] + p[ID(o, i, j - 1, k)]) +
                   (p[ID(o, i - 1, j, k)] + p[ID(o, i, j, k)])));
}

static void geometry(orc3_ctx *o, double *p) {
  int nx = o->c.nx, ny = o->c.ny, nz = o->c.nz;
  fill_ghost(o, p, 0);
  /* apertures of the lower faces of cells 0..n (the upper domain face is
   * the lower face of cell n) */
  for (int k = 0; k <= nz; k++)
    for (int j = 0; j <= ny; j++)
      for (int i = 0; i <= nx; i++) {
        int c = ID(o, i, j, k);
        double c000 = corner(o, p, i, j, k);
        if (j < ny && k < nz)
          o->ax[c] = orc_cell_alpha(c000, corner(o, p, i, j + 1, k),
                                    corner(o, p, i, j + 1, k + 1), corner(o, p, i, j, k + 1));
        if (i < nx && k < nz)
          o->ay[c] = orc_cell_alpha(c000, corner(o, p, i + 1, j, k),
                                    corner(o, p, i + 1, j, k + 1), corner(o, p, i, j, k + 1));
        if (i < nx && j < ny)
          o->az[c] = orc_cell_alpha(c000, corner(o, p, i + 1, j, k),
                                    corner(o, p, i + 1, j + 1, k), corner(o, p, i, j + 1, k));
      }
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j, k);
        double cv[8], s[3];
        for (int v = 0; v < 8; v++)
          cv[v] = corner(o, p, i + (v & 1), j + ((v >> 1) & 1), k + (v >> 2));
        o->alpha[c] = orc3_cell_alpha(cv, s);
        o->sx[c] = (o->ax[ID(o, i + 1, j, k)] - o->ax[c]) * (o->c.dy * o->c.dz);
        o->sy[c] = (o->ay[ID(o, i, j + 1, k)] - o->ay[c]) * (o->c.dx * o->c.dz);
        o->sz[c] = (o->az[ID(o, i, j, k + 1)] - o->az[c]) * (o->c.dx * o->c.dy);
      }
}

static double vol(const orc3_ctx *o, int k, int c) {
  return k == 1 ? o->alpha[c] : 1.0 - o->alpha[c];
}

static void normal(const orc3_ctx *o, const double *p, int i, int j, int k, double n[3]) {
  double g[3];
  g[0] = (p[ID(o, i + 1, j, k)] - p[ID(o, i - 1, j, k)]) / (2.0 * o->c.dx);
  g[1] = (p[ID(o, i, j + 1, k)] - p[ID(o, i, j - 1, k)]) / (2.0 * o->c.dy);
  g[2] = (p[ID(o, i, j, k + 1)] - p[ID(o, i, j, k - 1)]) / (2.0 * o->c.dz);
  double m = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  for (int d = 0; d < 3; d++) n[d] = m > 0.0 ? g[d] / m : 0.0;
}

static int inside(const orc3_ctx *o, int i, int j, int k) {
  return i >= 0 && i < o->c.nx && j >= 0 && j < o->c.ny && k >= 0 && k < o->c.nz;
}

/* ------------------------------------------------------------------ */
/* small-cell mixing (Sec. 2.2, last paragraph)                        */

/* Targets of small cell (i, j, k) of fluid k: the seven neighbours toward
 * the fluid along n_k that are not small, weighted as the file header
 * says; failing those, the largest of the 26 neighbours if it is not
 * small (searched plane by plane from the cell's own z, so that ties keep
 * the 2D choice); failing that, the seven neighbours larger than the
 * source. */
static int mix_targets(orc3_ctx *o, int kf, int i, int j, int k, int tc[7], double beta[7]) {
  int c = ID(o, i, j, k);
  double as = vol(o, kf, c);
  double n[3];
  normal(o, o->phi, i, j, k, n);
  if (kf == 0)
    for (int d = 0; d < 3; d++) n[d] = -n[d];
  int s0 = n[0] >= 0.0 ? 1 : -1, s1 = n[1] >= 0.0 ? 1 : -1, s2 = n[2] >= 0.0 ? 1 : -1;
  const int ti[7] = {i + s0, i, i, i + s0, i + s0, i, i + s0};
  const int tj[7] = {j, j + s1, j, j + s1, j, j + s1, j + s1};
  const int tk[7] = {k, k, k + s2, k, k + s2, k + s2, k + s2};
  double wt[7] = {n[0] * n[0], n[1] * n[1], n[2] * n[2], fabs(n[0] * n[1]),
                  fabs(n[0] * n[2]), fabs(n[1] * n[2]), 0.0};
  double triple = fabs(n[0] * n[1] * n[2]);
  wt[6] = triple > 0.0 ? pow(triple, 2.0 / 3.0) : 0.0;
  int keep[7] = {0, 0, 0, 0, 0, 0, 0};
  double sum = 0.0;
  for (int t = 0; t < 7; t++) {
    if (!inside(o, ti[t], tj[t], tk[t]) || !(wt[t] > 0.0)) continue;
    if (!(vol(o, kf, ID(o, ti[t], tj[t], tk[t])) >= o->c.mix_alpha)) continue;
    keep[t] = 1;
    sum += wt[t];
  }
  if (!(sum > 0.0)) {
    int best = -1;
    double ab = 0.0;
    const int dzs[3] = {0, -1, 1};
    for (int zz = 0; zz < 3; zz++)
      for (int dj = -1; dj <= 1; dj++)
        for (int di = -1; di <= 1; di++) {
          int dz = dzs[zz];
          if ((di == 0 && dj == 0 && dz == 0) || !inside(o, i + di, j + dj, k + dz)) continue;
          double at = vol(o, kf, ID(o, i + di, j + dj, k + dz));
          if (at > ab) {
            ab = at;
            best = ID(o, i + di, j + dj, k + dz);
          }
        }
    if (best >= 0 && ab >= o->c.mix_alpha) {
      tc[0] = best;
      beta[0] = 1.0;
      return 1;
    }
    for (int t = 0; t < 7; t++) {
      if (!inside(o, ti[t], tj[t], tk[t]) || !(wt[t] > 0.0)) continue;
      if (!(vol(o, kf, ID(o, ti[t], tj[t], tk[t])) > as)) continue;
      keep[t] = 1;
      sum += wt[t];
    }
  }
  if (!(sum > 0.0)) return 0;
  int nt = 0;
  for (int t = 0; t < 7; t++) {
    if (!keep[t]) continue;
    tc[nt] = ID(o, ti[t], tj[t], tk[t]);
    beta[nt] = wt[t] / sum;
    nt++;
  }
  return nt;
}

static void mix(orc3_ctx *o, int kf, double *const q[NC]) {
  for (int m = 0; m < NC; m++) memcpy(o->old[m], q[m], sizeof(double) * o->NP);
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        double as = vol(o, kf, c);
        if (as >= o->c.mix_alpha) continue;
        int empty = as == 0.0;
        for (int m = 0; m < NC; m++) empty = empty && o->old[m][c] == 0.0;
        if (empty) continue;
        int tcs[7];
        double betas[7];
        int nt = mix_targets(o, kf, i, j, k, tcs, betas);
        for (int t = 0; t < nt; t++) {
          int tc = tcs[t];
          double beta = betas[t];
          double at = vol(o, kf, tc);
          double den = as * beta + at;
          for (int m = 0; m < NC; m++) {
            double M = beta * (o->old[m][tc] * as - o->old[m][c] * at) / den;
            q[m][c] += M;
            q[m][tc] -= M;
          }
        }
      }
}

/* ------------------------------------------------------------------ */
/* stencil states (Sec. 2.3): real cells and extension                 */

static int is_real(const orc3_ctx *o, int kf, int c) {
  return vol(o, kf, c) > ALPHA_REAL && !o->nostate[kf][c];
}

static void prim(orc3_ctx *o, int kf, double *const q[NC]) {
  double g = o->c.gamma[kf], pi = o->c.pinf[kf];
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        double a = vol(o, kf, c);
        o->nostate[kf][c] = 0;
        if (!(a > ALPHA_REAL)) continue;
        double rho = q[0][c] / a;
        double u = q[1][c] / q[0][c];
        double v = q[2][c] / q[0][c];
        double w = q[3][c] / q[0][c];
        double E = q[4][c] / a;
        double p;
        if (o->c.tait[kf])
          p = o->c.tait_B[kf] * (pow(rho / o->c.tait_rho0[kf], g) - 1.0) + o->c.tait_p0[kf];
        else
          p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w)) - g * pi;
        if (!(rho > 0.0) || !(p + pi > 0.0)) {
          if (a < 1.0) {
            o->nostate[kf][c] = 1;
            continue;
          }
          o->err |= ORC_ERR_NONPHYS;
        }
        o->w[kf][0][c] = rho;
        o->w[kf][1][c] = u;
        o->w[kf][2][c] = v;
        o->w[kf][3][c] = w;
        o->w[kf][4][c] = p;
      }
}

/* one Jacobi sweep's value at a target: the upwind-weighted mean of its
 * upwind x, y and z neighbours of src (neighbours outside the domain drop
 * out); returns 0 where no neighbour is upwind */
static int upwind_mean(const orc3_ctx *o, int i, int j, int k, const double n[3],
                       double *const src[], int nf, double *out) {
  int s0 = n[0] >= 0.0 ? 1 : -1, s1 = n[1] >= 0.0 ? 1 : -1, s2 = n[2] >= 0.0 ? 1 : -1;
  double wx = fabs(n[0]) / o->c.dx, wy = fabs(n[1]) / o->c.dy, wz = fabs(n[2]) / o->c.dz;
  if (!inside(o, i + s0, j, k)) wx = 0.0;
  if (!inside(o, i, j + s1, k)) wy = 0.0;
  if (!inside(o, i, j, k + s2)) wz = 0.0;
  double den = wx + wy + wz;
  if (!(den > 0.0)) return 0;
  for (int m = 0; m < nf; m++) {
    double num = 0.0;
    if (wx > 0.0) num += wx * src[m][ID(o, i + s0, j, k)];
    if (wy > 0.0) num += wy * src[m][ID(o, i, j + s1, k)];
    if (wz > 0.0) num += wz * src[m][ID(o, i, j, k + s2)];
    out[m] = num / den;
  }
  return 1;
}

static void extend(orc3_ctx *o, int kf, const double *p) {
  double bw = o->c.band * o->h;
  for (int it = 0; it < o->c.ext_iters; it++) {
    for (int m = 0; m < NC; m++) memcpy(o->old[m], o->w[kf][m], sizeof(double) * o->NP);
    for (int k = 0; k < o->c.nz; k++)
      for (int j = 0; j < o->c.ny; j++)
        for (int i = 0; i < o->c.nx; i++) {
          int c = ID(o, i, j, k);
          if (!(fabs(p[c]) < bw) || is_real(o, kf, c)) continue;
          double n[3], out[NC];
          normal(o, p, i, j, k, n);
          if (kf == 0)
            for (int d = 0; d < 3; d++) n[d] = -n[d];
          if (!upwind_mean(o, i, j, k, n, o->old, NC, out)) continue;
          for (int m = 0; m < NC; m++) o->w[kf][m][c] = out[m];
        }
  }
}

static void wave_maxima(orc3_ctx *o, int kf, const double *p) {
  double g = o->c.gamma[kf], pi = o->c.pinf[kf];
  double bw = o->c.band * o->h;
  double l[3] = {0.0, 0.0, 0.0}, sm = 0.0;
  const double hd[3] = {o->c.dx, o->c.dy, o->c.dz};
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        int real = is_real(o, kf, c);
        if (!real && !(fabs(p[c]) < bw)) continue;
        double rho = o->w[kf][0][c], pr = o->w[kf][4][c];
        double cs = sqrt(dmax(g * (pr + pi) / rho, 0.0));
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
          double a = fabs(o->w[kf][1 + d][c]) + cs;
          l[d] = dmax(l[d], a);
          s += a / hd[d];
        }
        /* explicit viscous limit 2 nu (1/dx^2 + 1/dy^2 + 1/dz^2) */
        if (real && o->c.mu[kf] > 0.0)
          s += 2.0 * o->c.mu[kf] / rho *
               (1.0 / (hd[0] * hd[0]) + 1.0 / (hd[1] * hd[1]) + 1.0 / (hd[2] * hd[2]));
        if (real) sm = dmax(sm, s);
      }
  for (int d = 0; d < 3; d++) o->lf[kf][d] = l[d];
  o->smax[kf] = sm;
}

/* ------------------------------------------------------------------ */
/* interface interaction: the two-material Riemann problem along n      */

/* mean curvature of the level set, kappa = div(grad phi / |grad phi|), by
 * second-order central differences: (sum over the axes a of phi_aa times
 * the squared gradient across a, minus twice the sum over axis pairs of
 * phi_a phi_b phi_ab) / |grad phi|^3; 2 / r for phi = r - R */
static double curvature3(const orc3_ctx *o, const double *p, int i, int j, int k) {
  const double h[3] = {o->c.dx, o->c.dy, o->c.dz};
  const int st[3] = {1, o->PX, o->PX * o->PY};
  int c = ID(o, i, j, k);
  double g[3], gg[3][3];
  for (int a = 0; a < 3; a++) {
    g[a] = (p[c + st[a]] - p[c - st[a]]) / (2.0 * h[a]);
    gg[a][a] = (p[c + st[a]] - 2.0 * p[c] + p[c - st[a]]) / (h[a] * h[a]);
  }
  for (int a = 0; a < 3; a++)
    for (int b = a + 1; b < 3; b++) {
      int sa = st[a], sb = st[b];
      gg[a][b] = (p[c + sa + sb] - p[c + sa - sb] - p[c - sa + sb] + p[c - sa - sb]) /
                 (4.0 * h[a] * h[b]);
    }
  double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  if (!(g2 > 0.0)) return 0.0;
  double num = gg[0][0] * (g[1] * g[1] + g[2] * g[2]) + gg[1][1] * (g[0] * g[0] + g[2] * g[2]) +
               gg[2][2] * (g[0] * g[0] + g[1] * g[1]) -
               2.0 * (g[0] * g[1] * gg[0][1] + g[0] * g[2] * gg[0][2] + g[1] * g[2] * gg[1][2]);
  return num / (g2 * sqrt(g2));
}

/* Viscous stress (Stokes' hypothesis, no heat conduction) from the
 * velocity gradient G[a][b] = d u_b / d x_a: tau_aa = mu (4/3 G_aa - 2/3
 * (the other two diagonal terms)), tau_ab = mu (G_ab + G_ba). */
static void visc_stress3(double mu, const double G[3][3], double tau[3][3]) {
  tau[0][0] = mu * (4.0 / 3.0 * G[0][0] - 2.0 / 3.0 * G[1][1] - 2.0 / 3.0 * G[2][2]);
  tau[1][1] = mu * (4.0 / 3.0 * G[1][1] - 2.0 / 3.0 * G[0][0] - 2.0 / 3.0 * G[2][2]);
  tau[2][2] = mu * (4.0 / 3.0 * G[2][2] - 2.0 / 3.0 * G[0][0] - 2.0 / 3.0 * G[1][1]);
  tau[0][1] = tau[1][0] = mu * (G[1][0] + G[0][1]);
  tau[0][2] = tau[2][0] = mu * (G[2][0] + G[0][2]);
  tau[1][2] = tau[2][1] = mu * (G[2][1] + G[1][2]);
}

/* velocity component b (0..2) at cell c of the field that is continuous
 * across the interface: that of the fluid on whose side of the interface
 * the cell's centre lies (phi < 0: N) */
static double vel_across(const orc3_ctx *o, const double *p, int b, int c) {
  return o->w[p[c] < 0.0 ? 0 : 1][1 + b][c];
}

/* For every cut cell (S != 0): fluid N receives momentum -p_I,N S and
 * energy -p_I,N u_I |S|, fluid P momentum p_I,P S and energy p_I,P u_I |S|,
 * no mass; with surface tension the pressure jumps by sigma kappa from
 * fluid P into fluid N (Eq. 10), kappa > 0 where fluid N is convex; the
 * level-set velocity of the cell is u_I n; the star states' speeds enter
 * each fluid's CFL rate as (|u_I| + c*_k)(1/dx + 1/dy + 1/dz). */
static void interface(orc3_ctx *o, const double *p) {
  for (int m = 0; m < 4; m++) memset(o->xn[m], 0, sizeof(double) * o->NP);
  for (int m = 0; m < 4; m++) memset(o->xp[m], 0, sizeof(double) * o->NP);
  for (int m = 0; m < 3; m++) memset(o->ul[m], 0, sizeof(double) * o->NP);
  double fac = 1.0 / o->c.dx + 1.0 / o->c.dy + 1.0 / o->c.dz;
  /* the traction's central differences reach the ghost layers: the
   * velocities of both fluids' stencil states get the boundary conditions'
   * ghost values first */
  if (o->c.mu[0] > 0.0 && o->c.mu[1] > 0.0)
    for (int kf = 0; kf < 2; kf++)
      for (int b = 0; b < 3; b++) fill_ghost(o, o->w[kf][1 + b], 1 + b);
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        double S[3] = {o->sx[c], o->sy[c], o->sz[c]};
        if (S[0] == 0.0 && S[1] == 0.0 && S[2] == 0.0) continue;
        double Sm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        double n[3];
        normal(o, p, i, j, k, n);
        if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0)
          for (int d = 0; d < 3; d++) n[d] = S[d] / Sm;
        double un[2];
        for (int f = 0; f < 2; f++)
          un[f] = o->w[f][1][c] * n[0] + o->w[f][2][c] * n[1] + o->w[f][3][c] * n[2];
        double L[5] = {o->w[0][0][c], un[0], o->w[0][4][c], o->c.gamma[0], o->c.pinf[0]};
        double R[5] = {o->w[1][0][c], un[1], o->w[1][4][c], o->c.gamma[1], o->c.pinf[1]};
        double out[8];
        double jump = o->c.sigma != 0.0 ? o->c.sigma * curvature3(o, p, i, j, k) : 0.0;
        if (orc_riemann_jump2(L, R, jump, o->c.tait[0], o->c.tait[1], out))
          o->err |= ORC_ERR_NOCONV;
        double psN = out[7], psP = out[0], us = out[1];
        for (int d = 0; d < 3; d++) {
          o->xn[d][c] = -psN * S[d];
          o->xp[d][c] = psP * S[d];
          o->ul[d][c] = us * n[d];
        }
        o->xn[3][c] = -psN * us * Sm;
        o->xp[3][c] = psP * us * Sm;
        /* viscous traction across the interface (Eq. 5's interface term):
         * the stress of the velocity field that is continuous across it,
         * central differences at the cut cell, the harmonic mean of the two
         * viscosities; fluid N receives tau S and fluid P the opposite,
         * each with its work at that field's velocity in the cut cell */
        if (o->c.mu[0] > 0.0 && o->c.mu[1] > 0.0) {
          double muI = 2.0 * o->c.mu[0] * o->c.mu[1] / (o->c.mu[0] + o->c.mu[1]);
          const int st[3] = {1, o->PX, o->PX * o->PY};
          const double hd[3] = {o->c.dx, o->c.dy, o->c.dz};
          double G[3][3], tau[3][3];
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
              G[a][b] = (vel_across(o, p, b, c + st[a]) - vel_across(o, p, b, c - st[a])) /
                        (2.0 * hd[a]);
          visc_stress3(muI, G, tau);
          double f[3], e = 0.0;
          for (int a = 0; a < 3; a++) f[a] = tau[a][0] * S[0] + tau[a][1] * S[1] + tau[a][2] * S[2];
          for (int a = 0; a < 3; a++) e += vel_across(o, p, a, c) * f[a];
          for (int a = 0; a < 3; a++) {
            o->xn[a][c] = o->xn[a][c] + f[a];
            o->xp[a][c] = o->xp[a][c] - f[a];
          }
          o->xn[3][c] = o->xn[3][c] + e;
          o->xp[3][c] = o->xp[3][c] - e;
        }
        o->smax[0] = dmax(o->smax[0], (fabs(us) + out[4]) * fac);
        o->smax[1] = dmax(o->smax[1], (fabs(us) + out[5]) * fac);
      }
}

/* level-set velocity: the cut cells' u_I n carried outward through the
 * band by the same upwind sweeps, upwind meaning toward the interface */
static void extend_ls_velocity(orc3_ctx *o, const double *p) {
  double bw = o->c.band * o->h;
  for (int it = 0; it < o->c.ext_iters; it++) {
    for (int m = 0; m < 3; m++) memcpy(o->old[m], o->ul[m], sizeof(double) * o->NP);
    for (int k = 0; k < o->c.nz; k++)
      for (int j = 0; j < o->c.ny; j++)
        for (int i = 0; i < o->c.nx; i++) {
          int c = ID(o, i, j, k);
          if (!(fabs(p[c]) < bw)) continue;
          if (o->sx[c] != 0.0 || o->sy[c] != 0.0 || o->sz[c] != 0.0) continue;
          double n[3], out[3];
          normal(o, p, i, j, k, n);
          if (p[c] >= 0.0)
            for (int d = 0; d < 3; d++) n[d] = -n[d];
          if (!upwind_mean(o, i, j, k, n, o->old, 3, out)) continue;
          for (int m = 0; m < 3; m++) o->ul[m][c] = out[m];
        }
  }
}

static void eval(orc3_ctx *o, double *const qs[2][NC], double *p) {
  geometry(o, p);
  for (int kf = 0; kf < 2; kf++) {
    prim(o, kf, qs[kf]);
    extend(o, kf, p);
    wave_maxima(o, kf, p);
  }
  interface(o, p);
  extend_ls_velocity(o, p);
}

/* ------------------------------------------------------------------ */
/* WENO5-LF face fluxes and the cut-cell right-hand side (Eq. 2 in 3D)  */

static void split(const orc3_ctx *o, int kf, int c, int d, double a, double *fp, double *fm) {
  double g = o->c.gamma[kf], pi = o->c.pinf[kf];
  double rho = o->w[kf][0][c], p = o->w[kf][4][c];
  double vel[3] = {o->w[kf][1][c], o->w[kf][2][c], o->w[kf][3][c]};
  double E = (p + g * pi) / (g - 1.0) +
             0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
  double U[NC] = {rho, rho * vel[0], rho * vel[1], rho * vel[2], E};
  double un = vel[d];
  double F[NC];
  F[0] = rho * un;
  for (int e = 0; e < 3; e++) F[1 + e] = rho * vel[e] * un;
  F[1 + d] += p;
  F[4] = un * (E + p);
  for (int m = 0; m < NC; m++) {
    fp[m] = 0.5 * (F[m] + a * U[m]);
    fm[m] = 0.5 * (F[m] - a * U[m]);
  }
}

/* WENO5 of the split fluxes at the lower d-face of cell c (stride s) */
static void face_flux(const orc3_ctx *o, int kf, int c, int s, int d, double *Fh) {
  double a = o->lf[kf][d];
  double fp[6][NC], fm[6][NC];
  for (int r = 0; r < 6; r++) split(o, kf, c + (r - 3) * s, d, a, fp[r], fm[r]);
  for (int m = 0; m < NC; m++) {
    double vp[5] = {fp[0][m], fp[1][m], fp[2][m], fp[3][m], fp[4][m]};
    double vm[5] = {fm[5][m], fm[4][m], fm[3][m], fm[2][m], fm[1][m]};
    Fh[m] = orc_weno5(vp, o->c.weno_eps) + orc_weno5(vm, o->c.weno_eps);
  }
}

/* viscous flux through the lower d-face of cell c (stride s) from the
 * stencil states by central differences: the normal derivatives across the
 * face, the tangential ones the mean of the two cells' central differences */
static void viscous_face(const orc3_ctx *o, int kf, int c, int s, int d, double *Fv) {
  const double hd[3] = {o->c.dx, o->c.dy, o->c.dz};
  const int st[3] = {1, o->PX, o->PX * o->PY};
  int cl = c - s;
  double G[3][3], tau[3][3];
  for (int b = 0; b < 3; b++) {
    const double *u = o->w[kf][1 + b];
    for (int a = 0; a < 3; a++) {
      if (a == d)
        G[a][b] = (u[c] - u[cl]) / hd[a];
      else
        G[a][b] = ((u[c + st[a]] - u[c - st[a]]) + (u[cl + st[a]] - u[cl - st[a]])) /
                  (4.0 * hd[a]);
    }
  }
  visc_stress3(o->c.mu[kf], G, tau);
  Fv[0] = 0.0;
  double e = 0.0;
  for (int b = 0; b < 3; b++) {
    double uf = 0.5 * (o->w[kf][1 + b][cl] + o->w[kf][1 + b][c]);
    Fv[1 + b] = tau[d][b];
    e += uf * tau[d][b];
  }
  Fv[4] = e;
}

static double aperture(const orc3_ctx *o, int kf, int d, int c) {
  const double *A = d == 0 ? o->ax : d == 1 ? o->ay : o->az;
  return kf == 1 ? A[c] : 1.0 - A[c];
}

static void fv_rhs(orc3_ctx *o, int kf, double *const L[NC]) {
  int nx = o->c.nx, ny = o->c.ny, nz = o->c.nz;
  fill_ghost(o, o->w[kf][0], 0);
  fill_ghost(o, o->w[kf][1], 1);
  fill_ghost(o, o->w[kf][2], 2);
  fill_ghost(o, o->w[kf][3], 3);
  fill_ghost(o, o->w[kf][4], 0);
  const int st[3] = {1, o->PX, o->PX * o->PY};
  for (int d = 0; d < 3; d++) {
    for (int m = 0; m < NC; m++) memset(o->fl[d][m], 0, sizeof(double) * o->NP);
    for (int k = 0; k < nz + (d == 2); k++)
      for (int j = 0; j < ny + (d == 1); j++)
        for (int i = 0; i < nx + (d == 0); i++) {
          int c = ID(o, i, j, k);
          double A = aperture(o, kf, d, c);
          if (A == 0.0) continue;
          double Fh[NC];
          face_flux(o, kf, c, st[d], d, Fh);
          if (o->c.mu[kf] > 0.0) {
            double Fv[NC];
            viscous_face(o, kf, c, st[d], d, Fv);
            for (int m = 0; m < NC; m++) Fh[m] = Fh[m] - Fv[m];
          }
          for (int m = 0; m < NC; m++) o->fl[d][m][c] = A * Fh[m];
        }
  }
  const double hd[3] = {o->c.dx, o->c.dy, o->c.dz};
  double dv = o->c.dx * o->c.dy * o->c.dz;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = ID(o, i, j, k);
        int open = 0;
        for (int d = 0; d < 3; d++)
          open = open || aperture(o, kf, d, c) != 0.0 || aperture(o, kf, d, c + st[d]) != 0.0;
        o->open_updates += open;
        for (int m = 0; m < NC; m++) {
          double r = 0.0;
          for (int d = 0; d < 3; d++) r += (o->fl[d][m][c] - o->fl[d][m][c + st[d]]) / hd[d];
          if (m > 0) r += (kf == 0 ? o->xn : o->xp)[m - 1][c] / dv;
          L[m][c] = r;
        }
      }
}

/* ------------------------------------------------------------------ */
/* level set: advection (Eq. 6) and reinitialisation                   */

static void make_band(orc3_ctx *o, const double *p) {
  double bw = o->c.band * o->h;
  memset(o->band, 0, o->NP);
  memset(o->rext, 0, o->NP);
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) o->band[ID(o, i, j, k)] = fabs(p[ID(o, i, j, k)]) < bw;
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k), r = o->band[c];
        if (i > 0) r |= o->band[ID(o, i - 1, j, k)];
        if (i < o->c.nx - 1) r |= o->band[ID(o, i + 1, j, k)];
        if (j > 0) r |= o->band[ID(o, i, j - 1, k)];
        if (j < o->c.ny - 1) r |= o->band[ID(o, i, j + 1, k)];
        if (k > 0) r |= o->band[ID(o, i, j, k - 1)];
        if (k < o->c.nz - 1) r |= o->band[ID(o, i, j, k + 1)];
        o->rext[c] = (unsigned char)r;
      }
}

static double hj_deriv(const orc3_ctx *o, const double *p, int c, int s, double h, int backward) {
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

static void ls_rhs(orc3_ctx *o, double *p, double *L) {
  fill_ghost(o, p, 0);
  const int st[3] = {1, o->PX, o->PX * o->PY};
  const double hd[3] = {o->c.dx, o->c.dy, o->c.dz};
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        if (!o->band[c]) {
          L[c] = 0.0;
          continue;
        }
        double r = 0.0;
        for (int d = 0; d < 3; d++) {
          double u = o->ul[d][c];
          if (u != 0.0) r += u * hj_deriv(o, p, c, st[d], hd[d], u > 0.0);
        }
        L[c] = -r;
      }
}

static double grad_est(const double *p, int c, int s, double h) {
  double dm = fabs(p[c] - p[c - s]), dp = fabs(p[c + s] - p[c]);
  double dc = 0.5 * fabs(p[c + s] - p[c - s]);
  return dmax(dmax(dc, dp), dm) / h;
}

/* sweeps of phi_tau + S(phi0)(|grad phi| - 1) = 0: Godunov's Hamiltonian
 * with one-sided HJ-WENO5 derivatives, the subcell fix in cells where phi0
 * changes sign across a face, no new extremum among the face neighbours;
 * over the band and its face neighbours */
static void reinit(orc3_ctx *o, double *p) {
  double h = o->h;
  const int st[3] = {1, o->PX, o->PX * o->PY};
  const double hd[3] = {o->c.dx, o->c.dy, o->c.dz};
  fill_ghost(o, p, 0);
  memcpy(o->p0, p, sizeof(double) * o->NP);
  for (int it = 0; it < o->c.reinit_iters; it++) {
    fill_ghost(o, p, 0);
    memcpy(o->old[0], p, sizeof(double) * o->NP);
    const double *q = o->old[0], *z = o->p0;
    for (int k = 0; k < o->c.nz; k++)
      for (int j = 0; j < o->c.ny; j++)
        for (int i = 0; i < o->c.nx; i++) {
          int c = ID(o, i, j, k);
          if (!o->rext[c]) continue;
          double s0 = z[c];
          int pos = s0 >= 0.0;
          int cut = 0;
          for (int d = 0; d < 3; d++)
            cut = cut || (z[c - st[d]] >= 0.0) != pos || (z[c + st[d]] >= 0.0) != pos;
          if (cut) {
            double g[3], gm = 0.0;
            for (int d = 0; d < 3; d++) {
              g[d] = (z[c + st[d]] - z[c - st[d]]) / (2.0 * hd[d]);
              gm += g[d] * g[d];
            }
            gm = sqrt(gm);
            if (!(gm > 1e-8)) {
              gm = 0.0;
              for (int d = 0; d < 3; d++) {
                g[d] = grad_est(z, c, st[d], hd[d]);
                gm += g[d] * g[d];
              }
              gm = sqrt(gm);
            }
            double dmn = INFINITY;
            for (int d = 0; d < 3; d++)
              for (int sd = -1; sd <= 1; sd += 2) {
                double zn = z[c + sd * st[d]];
                if ((zn >= 0.0) == pos) continue;
                double dd = fabs(s0) / (fabs(s0) + fabs(zn)) * hd[d];
                if (dd < dmn) dmn = dd;
              }
            double D = fabs(s0) / gm;
            if (D > dmn) D = dmn;
            D = pos ? D : -D;
            double sg = pos ? 1.0 : -1.0;
            p[c] = q[c] - 0.5 * (sg * fabs(q[c]) - D);
          } else {
            if (s0 == 0.0) continue;
            double S = s0 / sqrt(s0 * s0 + h * h);
            double G = 0.0;
            for (int d = 0; d < 3; d++) {
              double a = hj_deriv(o, q, c, st[d], hd[d], 1);
              double b = hj_deriv(o, q, c, st[d], hd[d], 0);
              if (s0 > 0.0)
                G += dmax(sq(dmax(a, 0.0)), sq(dmin(b, 0.0)));
              else
                G += dmax(sq(dmin(a, 0.0)), sq(dmax(b, 0.0)));
            }
            double nv = q[c] - 0.5 * h * S * (sqrt(G) - 1.0);
            double lo = q[c - 1], hi = q[c - 1];
            for (int d = 0; d < 3; d++)
              for (int sd = -1; sd <= 1; sd += 2) {
                lo = dmin(lo, q[c + sd * st[d]]);
                hi = dmax(hi, q[c + sd * st[d]]);
              }
            if (s0 > 0.0 && nv < lo) nv = lo;
            if (s0 < 0.0 && nv > hi) nv = hi;
            p[c] = nv;
          }
        }
  }
}

/* ------------------------------------------------------------------ */
/* time integration: TVD-RK2 and the accelerated cycle (Sec. 3.1)       */

/* dst = cur + dt L (stage 1), else dst = (base + (cur + dt L)) / 2 */
static void rk_plane(orc3_ctx *o, int s, double *dst, const double *base, const double *cur,
                     const double *L, double dt, const unsigned char *mask) {
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        if (mask && !mask[c]) continue;
        if (s == 1)
          dst[c] = cur[c] + dt * L[c];
        else
          dst[c] = 0.5 * base[c] + 0.5 * (cur[c] + dt * L[c]);
      }
}

static double dt_of(const orc3_ctx *o, int kf) {
  return o->smax[kf] > 0.0 ? o->c.cfl / o->smax[kf] : INFINITY;
}

static void copy_planes(orc3_ctx *o, double *const dst[], double *const src[], int n) {
  for (int m = 0; m < n; m++) memcpy(dst[m], src[m], sizeof(double) * o->NP);
}

/* one RK2 step of both fluids and the level set with a common dt, the
 * first interaction step having been evaluated */
static void single_step_after_eval(orc3_ctx *o, double dt) {
  for (int kf = 0; kf < 2; kf++) copy_planes(o, o->q0[kf], o->q[kf], NC);
  memcpy(o->phi0, o->phi, sizeof(double) * o->NP);
  make_band(o, o->phi0);
  for (int s = 1; s <= 2; s++) {
    if (s > 1) eval(o, o->q, o->phi);
    for (int kf = 0; kf < 2; kf++) fv_rhs(o, kf, o->L[kf]);
    ls_rhs(o, o->phi, o->lphi);
    for (int kf = 0; kf < 2; kf++)
      for (int m = 0; m < NC; m++)
        rk_plane(o, s, o->q[kf][m], o->q0[kf][m], o->q[kf][m], o->L[kf][m], dt, NULL);
    rk_plane(o, s, o->phi, o->phi0, o->phi, o->lphi, dt, o->band);
    if (s == 2) reinit(o, o->phi);
    geometry(o, o->phi);
    mix(o, 0, o->q[0]);
    mix(o, 1, o->q[1]);
  }
  o->t += dt;
}

int orc3_step_single_dt(orc3_ctx *o, int nsteps, double t_end, orc_info *info) {
  long long open0 = o->open_updates;
  for (int n = 0; n < nsteps; n++) {
    if (t_end > 0.0 && o->t >= t_end) break;
    eval(o, o->q, o->phi);
    double dt = dmin(dt_of(o, 0), dt_of(o, 1));
    if (t_end > 0.0 && o->t + dt > t_end) dt = t_end - o->t;
    single_step_after_eval(o, dt);
    if (info) {
      info->t = o->t;
      info->dt1 = info->dt2 = dt;
      info->n_raw = info->n_used = 1.0;
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

/* Eq. 8 (an evaluation fluid 1 shares) and Eq. 9 (fluid 2 only) */
static void record(orc3_ctx *o, int f1, int shared, double dt1, double dt2) {
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++) {
        int c = ID(o, i, j, k);
        for (int m = 0; m < 4; m++) {
          double x1 = (f1 == 0 ? o->xn : o->xp)[m][c];
          if (shared) o->xc[m][c] = o->xc[m][c] + (-0.5 * x1) * dt1;
          o->xc[m][c] = o->xc[m][c] + (0.5 * x1) * dt2;
        }
      }
}

/* Eq. 7: fluid 1 at fluid-2 time theta dt1 inside the cycle */
static void interpolate(orc3_ctx *o, double th) {
  for (int m = 0; m < NC; m++)
    for (int k = 0; k < o->c.nz; k++)
      for (int j = 0; j < o->c.ny; j++)
        for (int i = 0; i < o->c.nx; i++) {
          int c = ID(o, i, j, k);
          o->qi[m][c] = (1.0 - th) * o->prev[m][c] + th * o->fut[m][c];
        }
}

/* one accelerated cycle (Sec. 3.1, steps 1-5) */
static void cycle(orc3_ctx *o, double t_end, orc_info *info) {
  eval(o, o->q, o->phi);
  double dtk[2] = {dt_of(o, 0), dt_of(o, 1)};
  for (int kf = 0; kf < 2; kf++)
    if (t_end > 0.0 && o->t + dtk[kf] > t_end) dtk[kf] = t_end - o->t;
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
      single_step_after_eval(o, dt2);
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
  for (int m = 0; m < 4; m++) memset(o->xc[m], 0, sizeof(double) * o->NP);
  /* step 2: fluid 1's first stage with dt1; previous and future states */
  fv_rhs(o, f1, o->L[f1]);
  copy_planes(o, o->prev, o->q[f1], NC);
  for (int m = 0; m < NC; m++)
    rk_plane(o, 1, o->fut[m], o->prev[m], o->prev[m], o->L[f1][m], dt1, NULL);
  double t2 = 0.0;
  int sub = 0;
  double *qs[2][NC];
  for (;;) {
    sub++;
    if (sub > 1) {
      interpolate(o, t2 / dt1);
      geometry(o, o->phi);
      mix(o, f1, o->qi);
      for (int m = 0; m < NC; m++) {
        qs[f1][m] = o->qi[m];
        qs[f2][m] = o->q[f2][m];
      }
      eval(o, qs, o->phi);
      dt2 = dt_of(o, f2);
    }
    int last = (dt1 - t2) <= dt2 * (1.0 + 1e-12);
    if (last) dt2 = dt1 - t2;
    record(o, f1, sub == 1, dt1, dt2);
    /* step 3: fluid 2 and the level set, first stage with dt2 */
    copy_planes(o, o->q0[f2], o->q[f2], NC);
    memcpy(o->phi0, o->phi, sizeof(double) * o->NP);
    make_band(o, o->phi0);
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    for (int m = 0; m < NC; m++)
      rk_plane(o, 1, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 1, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    geometry(o, o->phi);
    mix(o, f2, o->q[f2]);
    if (last) {
      mix(o, f1, o->fut);
      for (int m = 0; m < NC; m++) qs[f1][m] = o->fut[m];
    } else {
      interpolate(o, (t2 + dt2) / dt1);
      mix(o, f1, o->qi);
      for (int m = 0; m < NC; m++) qs[f1][m] = o->qi[m];
    }
    for (int m = 0; m < NC; m++) qs[f2][m] = o->q[f2][m];
    eval(o, qs, o->phi);
    record(o, f1, last, dt1, dt2);
    /* step 4 (and 5 on the last sub-step): second stage */
    fv_rhs(o, f2, o->L[f2]);
    ls_rhs(o, o->phi, o->lphi);
    if (last) fv_rhs(o, f1, o->L[f1]);
    for (int m = 0; m < NC; m++)
      rk_plane(o, 2, o->q[f2][m], o->q0[f2][m], o->q[f2][m], o->L[f2][m], dt2, NULL);
    rk_plane(o, 2, o->phi, o->phi0, o->phi, o->lphi, dt2, o->band);
    if (last)
      for (int m = 0; m < NC; m++)
        rk_plane(o, 2, o->q[f1][m], o->prev[m], o->fut[m], o->L[f1][m], dt1, NULL);
    reinit(o, o->phi);
    if (last) {
      if (o->c.flux_correction) {
        double dv = o->c.dx * o->c.dy * o->c.dz;
        for (int k = 0; k < o->c.nz; k++)
          for (int j = 0; j < o->c.ny; j++)
            for (int i = 0; i < o->c.nx; i++) {
              int c = ID(o, i, j, k);
              for (int m = 0; m < 4; m++) o->q[f1][m + 1][c] += o->xc[m][c] / dv;
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

int orc3_step_multi_dt(orc3_ctx *o, int ncycles, double t_end, orc_info *info) {
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

static double *plane(orc3_ctx *o) { return (double *)calloc((size_t)o->NP, sizeof(double)); }

#define FOR_PLANES(X)                                                   \
  for (int kf = 0; kf < 2; kf++)                                        \
    for (int m = 0; m < NC; m++) {                                      \
      X(o->q[kf][m]); X(o->w[kf][m]); X(o->q0[kf][m]); X(o->L[kf][m]);  \
    }                                                                   \
  for (int m = 0; m < NC; m++) {                                        \
    X(o->old[m]); X(o->prev[m]); X(o->fut[m]); X(o->qi[m]);             \
    for (int d = 0; d < 3; d++) X(o->fl[d][m]);                         \
  }                                                                     \
  for (int m = 0; m < 4; m++) {                                         \
    X(o->xn[m]); X(o->xp[m]); X(o->xc[m]);                              \
  }                                                                     \
  for (int d = 0; d < 3; d++) X(o->ul[d]);                              \
  X(o->phi); X(o->alpha); X(o->ax); X(o->ay); X(o->az);                 \
  X(o->sx); X(o->sy); X(o->sz); X(o->phi0); X(o->lphi); X(o->p0);

orc3_ctx *orc3_create(const orc3_config *cfg) {
  if (cfg->nx < GH || cfg->ny < GH || cfg->nz < GH) return NULL;
  if (!(cfg->dx > 0.0) || !(cfg->dy > 0.0) || !(cfg->dz > 0.0)) return NULL;
  if (!(cfg->sigma >= 0.0) || !isfinite(cfg->sigma)) return NULL;
  for (int k = 0; k < 2; k++)
    if (!(cfg->mu[k] >= 0.0) || !isfinite(cfg->mu[k])) return NULL;
  for (int k = 0; k < 2; k++) {
    if (cfg->tait[k] != 0 && cfg->tait[k] != 1) return NULL;
    if (cfg->tait[k] && (!(cfg->tait_B[k] > 0.0) || !(cfg->tait_rho0[k] > 0.0) ||
                         !isfinite(cfg->tait_p0[k]) || !isfinite(cfg->tait_B[k])))
      return NULL;
  }
  orc3_ctx *o = (orc3_ctx *)calloc(1, sizeof(orc3_ctx));
  o->c = *cfg;
  for (int k = 0; k < 2; k++)
    if (o->c.tait[k]) o->c.pinf[k] = o->c.tait_B[k] - o->c.tait_p0[k];
  o->PX = cfg->nx + 2 * GH;
  o->PY = cfg->ny + 2 * GH;
  o->PZ = cfg->nz + 2 * GH;
  o->NP = o->PX * o->PY * o->PZ;
  o->h = dmin(dmin(cfg->dx, cfg->dy), cfg->dz);
#define ALLOC(p) p = plane(o)
  FOR_PLANES(ALLOC)
#undef ALLOC
  o->band = (unsigned char *)calloc((size_t)o->NP, 1);
  o->rext = (unsigned char *)calloc((size_t)o->NP, 1);
  o->nostate[0] = (unsigned char *)calloc((size_t)o->NP, 1);
  o->nostate[1] = (unsigned char *)calloc((size_t)o->NP, 1);
  return o;
}

void orc3_destroy(orc3_ctx *o) {
  if (!o) return;
#define FREE(p) free(p)
  FOR_PLANES(FREE)
#undef FREE
  free(o->band);
  free(o->rext);
  free(o->nostate[0]);
  free(o->nostate[1]);
  free(o);
}

static void copy_out(const orc3_ctx *o, const double *src, double *dst) {
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++)
        dst[i + o->c.nx * (j + o->c.ny * k)] = src[ID(o, i, j, k)];
}

static void copy_in(orc3_ctx *o, const double *src, double *dst) {
  for (int k = 0; k < o->c.nz; k++)
    for (int j = 0; j < o->c.ny; j++)
      for (int i = 0; i < o->c.nx; i++)
        dst[ID(o, i, j, k)] = src[i + o->c.nx * (j + o->c.ny * k)];
}

int orc3_init(orc3_ctx *o, const double *phi, const double *pN, const double *pP) {
  int n = o->c.nx * o->c.ny * o->c.nz;
  copy_in(o, phi, o->phi);
  geometry(o, o->phi);
  for (int kf = 0; kf < 2; kf++) {
    const double *pr = kf == 0 ? pN : pP;
    double g = o->c.gamma[kf], pi = o->c.pinf[kf];
    for (int k = 0; k < o->c.nz; k++)
      for (int j = 0; j < o->c.ny; j++)
        for (int i = 0; i < o->c.nx; i++) {
          int c = ID(o, i, j, k), s = i + o->c.nx * (j + o->c.ny * k);
          double rho = pr[s], u = pr[n + s], v = pr[2 * n + s], w = pr[3 * n + s];
          double p = pr[4 * n + s];
          o->w[kf][0][c] = rho;
          o->w[kf][1][c] = u;
          o->w[kf][2][c] = v;
          o->w[kf][3][c] = w;
          o->w[kf][4][c] = p;
          double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
          double a = vol(o, kf, c);
          o->q[kf][0][c] = a * rho;
          o->q[kf][1][c] = a * (rho * u);
          o->q[kf][2][c] = a * (rho * v);
          o->q[kf][3][c] = a * (rho * w);
          o->q[kf][4][c] = a * E;
        }
  }
  mix(o, 0, o->q[0]);
  mix(o, 1, o->q[1]);
  o->t = 0.0;
  o->err = 0;
  return 0;
}

int orc3_get_state(const orc3_ctx *o, double *qN, double *qP, double *phi) {
  int n = o->c.nx * o->c.ny * o->c.nz;
  for (int m = 0; m < NC; m++) {
    if (qN) copy_out(o, o->q[0][m], qN + m * n);
    if (qP) copy_out(o, o->q[1][m], qP + m * n);
  }
  if (phi) copy_out(o, o->phi, phi);
  return 0;
}

int orc3_set_state(orc3_ctx *o, const double *qN, const double *qP, const double *phi) {
  int n = o->c.nx * o->c.ny * o->c.nz;
  for (int m = 0; m < NC; m++) {
    if (qN) copy_in(o, qN + m * n, o->q[0][m]);
    if (qP) copy_in(o, qP + m * n, o->q[1][m]);
  }
  if (phi) copy_in(o, phi, o->phi);
  geometry(o, o->phi);
  return 0;
}

int orc3_integrals(const orc3_ctx *o, double *out) {
  double dv = o->c.dx * o->c.dy * o->c.dz;
  for (int kf = 0; kf < 2; kf++)
    for (int m = 0; m < NC; m++) {
      double s = 0.0;
      for (int k = 0; k < o->c.nz; k++)
        for (int j = 0; j < o->c.ny; j++)
          for (int i = 0; i < o->c.nx; i++) s += o->q[kf][m][ID(o, i, j, k)];
      out[kf * NC + m] = s * dv;
    }
  return 0;
}

int orc3_geometry(orc3_ctx *o, double *alpha, double *ax, double *ay, double *az, double *sx,
                  double *sy, double *sz) {
  geometry(o, o->phi);
  if (alpha) copy_out(o, o->alpha, alpha);
  if (ax) copy_out(o, o->ax, ax);
  if (ay) copy_out(o, o->ay, ay);
  if (az) copy_out(o, o->az, az);
  if (sx) copy_out(o, o->sx, sx);
  if (sy) copy_out(o, o->sy, sy);
  if (sz) copy_out(o, o->sz, sz);
  return 0;
}

double orc3_curvature(orc3_ctx *o, int i, int j, int k) {
  fill_ghost(o, o->phi, 0);
  return curvature3(o, o->phi, i, j, k);
}

double orc3_time(const orc3_ctx *o) { return o->t; }
int orc3_status(const orc3_ctx *o) { return o->err; }
