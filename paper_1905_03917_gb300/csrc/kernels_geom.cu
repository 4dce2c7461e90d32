// kernels_geom.cu -- ghost layers, cut-cell geometry from the level set
// (Sec. 2.1, Fig. 1), narrow-band / cut-cell / active-tile lists compacted
// with warp ballots, small-cell mixing (Sec. 2.2) and initial data.
//
// Compiled without FMA contraction: these kernels take the branch
// decisions of the method (signs of corner values, small-cell and
// real-cell thresholds), so they round exactly like the CPU reference.
#include "sif_internal.cuh"

// ---------------------------------------------------------------------
// ghost layers in one pass: a ghost cell takes the value of the interior
// cell its x and y images map to (reflect / zero-gradient / periodic),
// negated once per reflecting wall for the matching velocity component --
// the same values as filling the x ghosts of the interior rows first and
// then the y ghosts of every column from them

__global__ void k_ghost(Grid g, GhostSet s) {
  SIF_TICK();
  int W = g.nx + 2 * SIF_GH;
  // ghost cells: the top and bottom strips (full width) and the left and
  // right strips of the interior rows
  int strip_y = W * SIF_GH, strip_x = SIF_GH * g.ny;
  int per = 2 * strip_y + 2 * strip_x;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * s.n) return;
  int pl = t / per, r = t % per, i, j;
  if (r < 2 * strip_y) {
    int q = r % strip_y;
    i = q % W - SIF_GH;
    j = r < strip_y ? -1 - q / W : g.ny + q / W;
  } else {
    r -= 2 * strip_y;
    int q = r % strip_x;
    j = q / SIF_GH;
    i = r < strip_x ? -1 - q % SIF_GH : g.nx + q % SIF_GH;
  }
  bool fx, fy;
  int si = ghost_image(i, g.nx, g.bc[0], g.bc[1], fx);
  int sj = ghost_image(j, g.ny, g.bc[2], g.bc[3], fy);
  // the plane and its velocity flag by select (a runtime index into the
  // parameter block would copy it to local memory)
  double *a = s.p[0];
  int vel = s.vel[0];
#pragma unroll
  for (int q = 1; q < 8; q++)
    if (pl == q) {
      a = s.p[q];
      vel = s.vel[q];
    }
  double v = a[gidx(g, si, sj)];
  bool neg = (vel == 1 && fx) || (vel == 2 && fy);
  a[gidx(g, i, j)] = neg ? -v : v;
}

void launch_fill_ghost(const Grid &g, const GhostSet &s, cudaStream_t st) {
  int n = (2 * (g.nx + 2 * SIF_GH) * SIF_GH + 2 * SIF_GH * g.ny) * s.n;
  launch_k(k_ghost, (n + 255) / 256, 256, 0, st, g, s);
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// warp-ballot compaction: one atomic per warp

__device__ inline void append_ballot(bool pred, int value, int *list, int *count) {
  unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (!mask) return;
  int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(mask) - 1) base = atomicAdd(count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
  if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

// ---------------------------------------------------------------------
// apertures, volume fraction and interface vector; cut-cell list

// geometry of grid point (i, j): the left x-face and bottom y-face of cell
// (i, j) and, for a cell inside the domain, its volume fraction and
// interface vector; returns whether the cell is cut
__device__ inline bool geom_point(const Grid &g, const double *__restrict__ p, int i, int j,
                                  double *alpha, double *ax, double *ay, double *sx,
                                  double *sy) {
  int c = gidx(g, i, j);
  // away from the interface all nine cells around the four corners share
  // a sign: every corner has it too, so the cell is full or empty
  int npos = 0;
#pragma unroll
  for (int dj = -1; dj <= 1; dj++)
#pragma unroll
    for (int di = -1; di <= 1; di++) npos += p[gidx(g, i + di, j + dj)] >= 0.0;
  if (npos == 9 || npos == 0) {
    double v = npos == 9 ? 1.0 : 0.0;
    if (j < g.ny) ax[c] = v;
    if (i < g.nx) ay[c] = v;
    if (i < g.nx && j < g.ny) {
      alpha[c] = v;
      sx[c] = 0.0;
      sy[c] = 0.0;
    }
    return false;
  }
  double c00 = corner_phi(g, p, i, j);
  double c01 = corner_phi(g, p, i, j + 1);
  double c10 = corner_phi(g, p, i + 1, j);
  if (j < g.ny) ax[c] = edge_fraction(c00, c01);
  if (i < g.nx) ay[c] = edge_fraction(c00, c10);
  if (i < g.nx && j < g.ny) {
    double c11 = corner_phi(g, p, i + 1, j + 1);
    alpha[c] = cell_alpha(c00, c10, c11, c01);
    double axl = edge_fraction(c00, c01), axr = edge_fraction(c10, c11);
    double ayb = edge_fraction(c00, c10), ayt = edge_fraction(c01, c11);
    double Sx = (axr - axl) * g.dy;
    double Sy = (ayt - ayb) * g.dx;
    sx[c] = Sx;
    sy[c] = Sy;
    return Sx != 0.0 || Sy != 0.0;
  }
  return false;
}

__global__ void k_geometry(Grid g, const double *__restrict__ p, double *alpha, double *ax,
                           double *ay, double *sx, double *sy, int *cut, int *ncut) {
  SIF_TICK();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int W = g.nx + 1;
  int i = t % W, j = t / W;
  bool is_cut = false;
  int c = 0;
  if (j <= g.ny) {
    c = gidx(g, i, j);
    is_cut = geom_point(g, p, i, j, alpha, ax, ay, sx, sy);
  }
  append_ballot(is_cut, c, cut, ncut);
}

// the same over the cells of a band list (and the domain's last x-face /
// y-face next to them): after a level-set step, which moves the interface
// by less than a cell and changes phi only inside the band, every grid
// point whose geometry can differ belongs to a cell of the previous band
__global__ void k_geometry_band(Grid g, const double *__restrict__ p, double *alpha, double *ax,
                                double *ay, double *sx, double *sy, const int *__restrict__ band,
                                const int *nband, int *cut, int *ncut) {
  SIF_TICK();
  int n = *nband;
  int nloop = (n + 31) / 32 * 32;  // whole warps for the ballot
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nloop;
       idx += gridDim.x * blockDim.x) {
    bool is_cut = false;
    int c = 0;
    if (idx < n) {
      c = band[idx];
      int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
      is_cut = geom_point(g, p, i, j, alpha, ax, ay, sx, sy);
      if (i == g.nx - 1) geom_point(g, p, g.nx, j, alpha, ax, ay, sx, sy);
      if (j == g.ny - 1) geom_point(g, p, i, g.ny, alpha, ax, ay, sx, sy);
    }
    append_ballot(is_cut, c, cut, ncut);
  }
}

void launch_geometry(const Grid &g, const double *phi, double *alpha, double *ax, double *ay,
                     double *sx, double *sy, int *cut_list, Scalars *sc, cudaStream_t st,
                     const int *band, const int *nband, int band_cap) {
  cudaMemsetAsync(&sc->n_cut, 0, sizeof(int), st);
  if (band) {
    int blocks = (band_cap + 127) / 128;
    if (blocks > 2432) blocks = 2432;
    launch_k(k_geometry_band, blocks < 1 ? 1 : blocks, 128, 0, st, g, phi, alpha, ax, ay, sx, sy,
                                                             band, nband, cut_list, &sc->n_cut);
  } else {
    int n = (g.nx + 1) * (g.ny + 1);
    launch_k(k_geometry, (n + 255) / 256, 256, 0, st, g, phi, alpha, ax, ay, sx, sy, cut_list,
                                                &sc->n_cut);
  }
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// narrow band |phi| < band*h and its face-neighbour extension

__global__ void k_band(Grid g, const double *__restrict__ p, int *band, int *rext, int *nband,
                       int *nrext) {
  SIF_TICK();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i = t % g.nx, j = t / g.nx;
  bool valid = j < g.ny;
  double bw = g.band * g.h;
  bool in = false, inx = false;
  int c = 0;
  if (valid) {
    c = gidx(g, i, j);
    in = fabs(p[c]) < bw;
    inx = in;
    if (i > 0) inx = inx || fabs(p[c - 1]) < bw;
    if (i < g.nx - 1) inx = inx || fabs(p[c + 1]) < bw;
    if (g.dim == 2) {
      if (j > 0) inx = inx || fabs(p[c - g.PX]) < bw;
      if (j < g.ny - 1) inx = inx || fabs(p[c + g.PX]) < bw;
    }
  }
  append_ballot(in, c, band, nband);
  if (rext) append_ballot(inx, c, rext, nrext);
}

void launch_band_lists(const Grid &g, const double *phi, int *band, int *rext, int *counts,
                       cudaStream_t st) {
  cudaMemsetAsync(counts, 0, 2 * sizeof(int), st);
  int n = g.nx * g.ny;
  launch_k(k_band, (n + 255) / 256, 256, 0, st, g, phi, band, rext, &counts[0], &counts[1]);
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// ---------------------------------------------------------------------
// initial data: (alpha U)_k = alpha_k U(W_k) from the primitive fields

__global__ void k_init_q(Grid g, double *qN0, double *qN1, double *qN2, double *qN3,
                         double *qP0, double *qP1, double *qP2, double *qP3, const double *wN0,
                         const double *wN1, const double *wN2, const double *wN3,
                         const double *wP0, const double *wP1, const double *wP2,
                         const double *wP3, const double *alpha) {
  SIF_TICK();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nx * g.ny) return;
  int i = t % g.nx, j = t / g.nx, c = gidx(g, i, j);
  for (int k = 0; k < 2; k++) {
    const double *w[4] = {k ? wP0 : wN0, k ? wP1 : wN1, k ? wP2 : wN2, k ? wP3 : wN3};
    double *q[4] = {k ? qP0 : qN0, k ? qP1 : qN1, k ? qP2 : qN2, k ? qP3 : qN3};
    double gm = g.gamma[k], pi = g.pinf[k];
    double rho = w[0][c], u = w[1][c], v = w[2][c], p = w[3][c];
    double E = (p + gm * pi) / (gm - 1.0) + 0.5 * rho * (u * u + v * v);
    double a = vol_k(alpha, k, c);
    q[0][c] = a * rho;
    q[1][c] = a * (rho * u);
    q[2][c] = a * (rho * v);
    q[3][c] = a * E;
  }
}

void launch_init_state(const Grid &g, double *const qN[4], double *const qP[4],
                       double *const wN[4], double *const wP[4], const double *alpha,
                       cudaStream_t st) {
  int n = g.nx * g.ny;
  launch_k(k_init_q, (n + 255) / 256, 256, 0, st, g, qN[0], qN[1], qN[2], qN[3], qP[0], qP[1], qP[2],
                                            qP[3], wN[0], wN[1], wN[2], wN[3], wP[0], wP[1],
                                            wP[2], wP[3], alpha);
  sif_note_launches(1);
}

SIF_TU_LAUNCH_READER(geom)
