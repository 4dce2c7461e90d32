// kernels3d.cu -- the three-dimensional solver's kernels other than the
// finite-volume stage: ghost layers, cut-cell geometry of the cube (Sec.
// 2.1), primitive recovery and extension (Sec. 2.3), wave maxima, the
// interface Riemann problem (Sec. 2.1), small-cell mixing (Sec. 2.2), the
// level set (Eq. 6) and its reinitialisation, the Eq. 7-9 cycle pieces.
//
// Compiled without FMA contraction: these kernels take the method's
// branch decisions (signs, thresholds, target choices), which therefore
// round like a plain serial evaluation of the same formulas.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "sif3d_internal.cuh"
#include "sif_internal.cuh"

static std::atomic<unsigned long long> g_launches{0};
unsigned long long k3_launches() { return g_launches.load(); }
static inline void tick(int n = 1) { g_launches += (unsigned long long)n; }

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

__device__ inline double sq3(double a) { return a * a; }

__device__ inline void cell_ijk(const Grid3 &g, int t, int &i, int &j, int &k) {
  i = t % g.nx;
  int r = t / g.nx;
  j = r % g.ny;
  k = r / g.ny;
}

__device__ inline bool in3(const Grid3 &g, int i, int j, int k) {
  return i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz;
}

__device__ inline double volk(const double *alphaP, int k, int c) {
  return k == 1 ? alphaP[c] : 1.0 - alphaP[c];
}

__device__ inline void atomic_max_d(unsigned long long *a, double v) {
  if (v > 0.0) atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------
// ghost layers: direction d's ghosts of every line along d; x lines over
// interior (y, z), y lines over all x (ghosts included) and interior z, z
// lines over all (x, y); the three directions run in that order

__global__ void k3_ghost(Grid3 g, Planes3 s, int d) {
  int n = d == 0 ? g.nx : d == 1 ? g.ny : g.nz;
  int la = d == 0 ? g.ny : g.PX;                   // first transverse extent
  int lb = d == 2 ? g.PY : g.nz;                   // second transverse extent
  int oa = d == 0 ? 0 : -S3_GH, ob = d == 2 ? -S3_GH : 0;
  long long total = (long long)la * lb * S3_GH * 2;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int side = (int)(t & 1);
  long long r = t >> 1;
  int m = (int)(r % S3_GH);
  r /= S3_GH;
  int a = (int)(r % la) + oa, b = (int)(r / la) + ob;
  int bc = g.bc[2 * d + side];
  int src;
  if (bc == 0)
    src = side == 0 ? m : n - 1 - m;
  else if (bc == 2)
    src = side == 0 ? n - 1 - m : m;
  else
    src = side == 0 ? 0 : n - 1;
  int dst = side == 0 ? -1 - m : n + m;
  int ci, cj, ck, di, dj, dk;
  if (d == 0) {
    ci = src, cj = a, ck = b, di = dst, dj = a, dk = b;
  } else if (d == 1) {
    ci = a, cj = src, ck = b, di = a, dj = dst, dk = b;
  } else {
    ci = a, cj = b, ck = src, di = a, dj = b, dk = dst;
  }
  int cs = g3(g, ci, cj, ck), cd = g3(g, di, dj, dk);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    if (q >= s.n) break;
    double v = s.p[q][cs];
    s.p[q][cd] = (s.vel[q] == d + 1 && bc == 0) ? -v : v;
  }
}

void k3_launch_ghost(const Grid3 &g, const Planes3 &s, cudaStream_t st) {
  for (int d = 0; d < 3; d++) {
    int la = d == 0 ? g.ny : g.PX, lb = d == 2 ? g.PY : g.nz;
    long long total = (long long)la * lb * S3_GH * 2;
    k3_ghost<<<nblk(total, 256), 256, 0, st>>>(g, s, d);
  }
  tick(3);
}

// ---------------------------------------------------------------------
// geometry

// area fraction of {phi >= 0} on a unit square from its corners
// counter-clockwise, the polygon through the positive corners and the edge
// crossings (a saddle's positive corners as separate triangles)
__device__ inline double sq_fraction(double c0, double c1, double c2, double c3) {
  const double v[4] = {c0, c1, c2, c3};
  const double px[4] = {0.0, 1.0, 1.0, 0.0};
  const double py[4] = {0.0, 0.0, 1.0, 1.0};
  int npos = 0, changes = 0;
  for (int e = 0; e < 4; e++) {
    npos += v[e] >= 0.0;
    changes += (v[e] >= 0.0) != (v[(e + 1) & 3] >= 0.0);
  }
  if (npos == 4) return 1.0;
  if (npos == 0) return 0.0;
  if (changes == 4) {
    double area = 0.0;
    for (int e = 0; e < 4; e++) {
      if (v[e] < 0.0) continue;
      int nx = (e + 1) & 3, pv = (e + 3) & 3;
      area += 0.5 * (v[e] / (v[e] - v[nx])) * (v[e] / (v[e] - v[pv]));
    }
    return area;
  }
  // shoelace over the polygon's vertices in order, streamed (first and
  // previous vertex kept) instead of stored: the same terms summed in the
  // same order, the closing edge last
  double fx = 0.0, fy = 0.0, qx = 0.0, qy = 0.0, a2 = 0.0;
  int m = 0;
  for (int e = 0; e < 4; e++) {
    int nx = (e + 1) & 3;
    for (int part = 0; part < 2; part++) {
      double x, y;
      if (part == 0) {
        if (!(v[e] >= 0.0)) continue;
        x = px[e];
        y = py[e];
      } else {
        if ((v[e] >= 0.0) == (v[nx] >= 0.0)) continue;
        double s = v[e] / (v[e] - v[nx]);
        x = px[e] + s * (px[nx] - px[e]);
        y = py[e] + s * (py[nx] - py[e]);
      }
      if (m == 0) {
        fx = x;
        fy = y;
      } else {
        a2 += qx * y - x * qy;
      }
      qx = x;
      qy = y;
      m++;
    }
  }
  a2 += qx * fy - fx * qy;
  return 0.5 * a2;
}

// corner value at the lower corner of cell (i, j, k): the mean of the
// eight cells sharing it
__device__ inline double corner3(const Grid3 &g, const double *p, int i, int j, int k) {
  int c = g3(g, i, j, k), sx = 1, sy = g.PX, sz = g.PX * g.PY;
  double a = (p[c - sx - sy - sz] + p[c - sy - sz]) + (p[c - sx - sz] + p[c - sz]);
  double b = (p[c - sx - sy] + p[c - sy]) + (p[c - sx] + p[c]);
  return 0.125 * (a + b);
}

// positions of the extended range (indices 0..n along each axis): the
// whole range, or per listed brick its cells and the layer above them (9
// x 9 x 5 positions, one thread each, packed with no idle slots;
// neighbouring bricks share a layer and write the same values there)
#define S3_EXT_SLOTS ((S3_BX + 1) * (S3_BY + 1) * (S3_BZ + 1))
__device__ inline bool region_ext(const Grid3 &g, const Region &R, long long t, int &i, int &j,
                                  int &k) {
  int ex = g.nx + 1, ey = g.ny + 1;
  if (!R.list) {
    if (t >= (long long)ex * ey * (g.nz + 1)) return false;
    i = (int)(t % ex);
    j = (int)((t / ex) % ey);
    k = (int)(t / ((long long)ex * ey));
    return true;
  }
  long long b = t / S3_EXT_SLOTS;
  int l = (int)(t % S3_EXT_SLOTS);
  if (b >= R.count) return false;
  int bi = R.list[b];
  int nbx = (g.nx + S3_BX - 1) / S3_BX, nby = (g.ny + S3_BY - 1) / S3_BY;
  i = (bi % nbx) * S3_BX + l % (S3_BX + 1);
  j = ((bi / nbx) % nby) * S3_BY + (l / (S3_BX + 1)) % (S3_BY + 1);
  k = (bi / (nbx * nby)) * S3_BZ + l / ((S3_BX + 1) * (S3_BY + 1));
  return i <= g.nx && j <= g.ny && k <= g.nz;
}

inline long long region_ext_threads(const Grid3 &g, const Region &R) {
  return R.list ? (long long)R.count * S3_EXT_SLOTS
                : (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
}

// corner values of the lower corners (indices 0..n), each from the eight
// cells around it.  Over the band list: a changed level-set value changes
// only the corners of its own cell and the cell above along each axis,
// both inside its brick's range
__global__ void k3_corners(Grid3 g, Region R, const double *phi, double *corner) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, k;
  if (!region_ext(g, R, t, i, j, k)) return;
  corner[g3(g, i, j, k)] = corner3(g, phi, i, j, k);
}

// one thread per cell of the (nx+1)(ny+1)(nz+1) extended range: the
// apertures of the cell's three lower faces and, for interior cells,
// alpha_P and S from the divergence theorem over the P region
__global__ void k3_geometry(Grid3 g, Region R, const double *corner, double *alpha, double *ax,
                            double *ay, double *az, double *sxo, double *syo, double *szo) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, k;
  if (!region_ext(g, R, t, i, j, k)) return;
  // corners beyond the upper ends (index n + 1) exist only for the faces
  // a thread of the extended range does not write; they read zeros
  double C[8];
#pragma unroll
  for (int v = 0; v < 8; v++) {
    int ci = i + (v & 1), cj = j + ((v >> 1) & 1), ck = k + (v >> 2);
    C[v] = (ci <= g.nx && cj <= g.ny && ck <= g.nz) ? corner[g3(g, ci, cj, ck)] : 0.0;
  }
  // faces in their own (a, b) axes counter-clockwise: x-face (y, z),
  // y-face (x, z), z-face (x, y); C index = di + 2 dj + 4 dk
  double axm = sq_fraction(C[0], C[2], C[6], C[4]);
  double aym = sq_fraction(C[0], C[1], C[5], C[4]);
  double azm = sq_fraction(C[0], C[1], C[3], C[2]);
  int c = g3(g, i, j, k);
  if (j < g.ny && k < g.nz) ax[c] = axm;
  if (i < g.nx && k < g.nz) ay[c] = aym;
  if (i < g.nx && j < g.ny) az[c] = azm;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return;
  double axp = sq_fraction(C[1], C[3], C[7], C[5]);
  double ayp = sq_fraction(C[2], C[3], C[7], C[6]);
  double azp = sq_fraction(C[4], C[5], C[7], C[6]);
  double s0 = axp - axm, s1 = ayp - aym, s2 = azp - azm;
  sxo[c] = s0 * (g.dy * g.dz);
  syo[c] = s1 * (g.dx * g.dz);
  szo[c] = s2 * (g.dx * g.dy);
  int npos = 0;
  for (int v = 0; v < 8; v++) npos += C[v] >= 0.0;
  double al;
  if (npos == 8) {
    al = 1.0;
  } else if (npos == 0) {
    al = 0.0;
  } else {
    // mean of the crossings on the twelve edges: edges along d in the
    // order of the other two coordinates ((d+1) mod 3, (d+2) mod 3)
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    int nc = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      int e1 = d == 2 ? 0 : d + 1, e2 = d == 0 ? 2 : d - 1;
#pragma unroll
      for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
          int lo = (a << e1) | (b << e2);  // corner index bit per axis
          int hi = lo | (1 << d);
          // corner index = di + 2 dj + 4 dk: bit d of the index is axis d
          double va = C[lo], vb = C[hi];
          if ((va >= 0.0) == (vb >= 0.0)) continue;
          double tt = va / (va - vb);
          double xi[3];
          xi[d] = tt;
          xi[e1] = a;
          xi[e2] = b;
          m0 += xi[0];
          m1 += xi[1];
          m2 += xi[2];
          nc++;
        }
    }
    m0 /= nc;
    m1 /= nc;
    m2 /= nc;
    al = (axp + ayp + azp - (m0 * s0 + m1 * s1 + m2 * s2)) / 3.0;
    if (al < 0.0) al = 0.0;
    if (al > 1.0) al = 1.0;
  }
  alpha[c] = al;
}

void k3_launch_geometry(const Grid3 &g, const Region &R, const double *phi, double *corner,
                        double *alpha, double *ax, double *ay, double *az, double *sx,
                        double *sy, double *sz, cudaStream_t st) {
  long long total = region_ext_threads(g, R);
  if (total == 0) return;
  k3_corners<<<nblk(total, 256), 256, 0, st>>>(g, R, phi, corner);
  k3_geometry<<<nblk(total, 128), 128, 0, st>>>(g, R, corner, alpha, ax, ay, az, sx, sy, sz);
  tick(2);
}

// the band list: every brick with a cell closer to the interface than
// thr (|phi| < thr); and per fluid k the band bricks and those holding
// fluid k (alpha_k > the sliver threshold): until the next list, fluid k
// can appear only inside the band, so its real and extended cells lie in
// its list.  One CTA per brick; the counts land in sc->nband, sc->nfluid
__global__ void k3_band_bricks(Grid3 g, const double *phi, const double *alpha, double thr,
                               int *list, int *fl0, int *fl1, Scal3 *sc) {
  const int bi = blockIdx.x, tid = threadIdx.x;
  int nbx = (g.nx + S3_BX - 1) / S3_BX, nby = (g.ny + S3_BY - 1) / S3_BY;
  int i = (bi % nbx) * S3_BX + tid % S3_BX;
  int j = ((bi / nbx) % nby) * S3_BY + (tid / S3_BX) % S3_BY;
  int k = (bi / (nbx * nby)) * S3_BZ + tid / (S3_BX * S3_BY);
  bool valid = i < g.nx && j < g.ny && k < g.nz;
  int c = valid ? g3(g, i, j, k) : 0;
  int near = valid && fabs(phi[c]) < thr;
  int hasN = valid && 1.0 - alpha[c] > S3_ALPHA_REAL;
  int hasP = valid && alpha[c] > S3_ALPHA_REAL;
  int b = __syncthreads_or(near);
  int bN = __syncthreads_or(hasN), bP = __syncthreads_or(hasP);
  if (tid == 0) {
    if (b) list[atomicAdd(&sc->nband, 1)] = bi;
    if (b || bN) fl0[atomicAdd(&sc->nfluid[0], 1)] = bi;
    if (b || bP) fl1[atomicAdd(&sc->nfluid[1], 1)] = bi;
  }
}

void k3_launch_band_bricks(const Grid3 &g, int nbricks, const double *phi, const double *alpha,
                           int *list, int *fl0, int *fl1, Scal3 *sc, cudaStream_t st) {
  cudaMemsetAsync(&sc->nband, 0, 3 * sizeof(int), st);  // nband, nfluid[2]
  k3_band_bricks<<<nbricks, S3_BX * S3_BY * S3_BZ, 0, st>>>(g, phi, alpha, g.bw + 3.0 * g.h,
                                                            list, fl0, fl1, sc);
  tick();
}

// ---------------------------------------------------------------------
// dense <-> padded copies of one plane (the caller's layout has no ghosts)

__global__ void k3_pack(Grid3 g, const double *padded, double *dense, int unpack) {
  long long n = (long long)g.nx * g.ny * g.nz;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i, j, k;
  cell_ijk(g, (int)t, i, j, k);
  int c = g3(g, i, j, k);
  if (unpack)
    ((double *)padded)[c] = dense[t];
  else
    dense[t] = padded[c];
}

void k3_launch_pack(const Grid3 &g, const double *padded, double *dense, int unpack,
                    cudaStream_t st) {
  long long n = (long long)g.nx * g.ny * g.nz;
  k3_pack<<<nblk(n, 256), 256, 0, st>>>(g, padded, dense, unpack);
  tick();
}

// initial conservative state of fluid k from dense primitive planes
// (rho, u, v, w, p): alpha_k U_k, and the stencil states W_k = the primitives
__global__ void k3_init_state(Grid3 g, const double *alpha, const double *pr, int k,
                              Planes3 qs, Planes3 ws) {
  long long n = (long long)g.nx * g.ny * g.nz;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i, j, kk;
  cell_ijk(g, (int)t, i, j, kk);
  int c = g3(g, i, j, kk);
  double rho = pr[t], u = pr[n + t], v = pr[2 * n + t], w = pr[3 * n + t], p = pr[4 * n + t];
  ws.p[0][c] = rho;
  ws.p[1][c] = u;
  ws.p[2][c] = v;
  ws.p[3][c] = w;
  ws.p[4][c] = p;
  double gm = g.gamma[k], pi = g.pinf[k];
  double E = (p + gm * pi) / (gm - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
  double a = volk(alpha, k, c);
  qs.p[0][c] = a * rho;
  qs.p[1][c] = a * (rho * u);
  qs.p[2][c] = a * (rho * v);
  qs.p[3][c] = a * (rho * w);
  qs.p[4][c] = a * E;
}

void k3_launch_init_state(const Grid3 &g, const double *alpha, const double *prim_dense,
                          double *const q[S3_NC], double *const w[S3_NC], int k,
                          cudaStream_t st) {
  Planes3 qs{}, ws{};
  for (int m = 0; m < S3_NC; m++) {
    qs.p[m] = q[m];
    ws.p[m] = w[m];
  }
  qs.n = ws.n = S3_NC;
  long long n = (long long)g.nx * g.ny * g.nz;
  k3_init_state<<<nblk(n, 256), 256, 0, st>>>(g, alpha, prim_dense, k, qs, ws);
  tick();
}

// ---------------------------------------------------------------------
// primitive recovery (Sec. 2.3): W_k = (alpha U)_k / alpha_k in cells that
// hold fluid k; a cut cell whose content is not a physical state is marked
// and treated as empty by the stencils; a full one is an error

__global__ void k3_prim(Grid3 g, Region R, int k, Planes3 q, Planes3 w, const double *alpha,
                        unsigned char *nostate, Scal3 *sc) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  unsigned char *ns = nostate + (size_t)k * g.NP;
  double a = volk(alpha, k, c);
  ns[c] = 0;
  if (!(a > S3_ALPHA_REAL)) return;
  double m = q.p[0][c];
  double rho = m / a;
  double u = q.p[1][c] / m, v = q.p[2][c] / m, ww = q.p[3][c] / m;
  double E = q.p[4][c] / a;
  double gm = g.gamma[k], pi = g.pinf[k];
  double p;
  if (g.tait[k])
    p = g.tB[k] * (pow(rho / g.tr0[k], gm) - 1.0) + g.tp0[k];
  else
    p = (gm - 1.0) * (E - 0.5 * rho * (u * u + v * v + ww * ww)) - gm * pi;
  if (!(rho > 0.0) || !(p + pi > 0.0)) {
    if (a < 1.0) {
      ns[c] = 1;
      return;
    }
    atomicOr(&sc->err, S3_ERR_NONPHYS);
  }
  w.p[0][c] = rho;
  w.p[1][c] = u;
  w.p[2][c] = v;
  w.p[3][c] = ww;
  w.p[4][c] = p;
}

void k3_launch_prim(const Grid3 &g, const Region &R, int k, double *const q[S3_NC],
                    double *const w[S3_NC], const double *alpha, unsigned char *nostate,
                    Scal3 *sc, cudaStream_t st) {
  Planes3 Q{}, W{};
  for (int m = 0; m < S3_NC; m++) {
    Q.p[m] = q[m];
    W.p[m] = w[m];
  }
  long long n = region_threads(g, R);
  if (n == 0) return;
  k3_prim<<<nblk(n, 256), 256, 0, st>>>(g, R, k, Q, W, alpha, nostate, sc);
  tick();
}

// unit normal grad(phi)/|grad(phi)| by central differences
__device__ inline void normal3(const Grid3 &g, const double *p, int c, double n[3]) {
  double gx = (p[c + 1] - p[c - 1]) / (2.0 * g.dx);
  double gy = (p[c + g.PX] - p[c - g.PX]) / (2.0 * g.dy);
  int sz = g.PX * g.PY;
  double gz = (p[c + sz] - p[c - sz]) / (2.0 * g.dz);
  double m = sqrt(gx * gx + gy * gy + gz * gz);
  n[0] = m > 0.0 ? gx / m : 0.0;
  n[1] = m > 0.0 ? gy / m : 0.0;
  n[2] = m > 0.0 ? gz / m : 0.0;
}

// ---------------------------------------------------------------------
// extension (Sec. 2.3): Jacobi sweeps of the upwind discretisation of
// n . grad W = 0 over the band's targets.  group 0/1: the stencil states
// of fluid N/P (targets: band cells that do not hold the fluid; n toward
// the fluid); group 2: the level-set velocity (targets: band cells with no
// interface; n toward the interface).  The plan fixes every target's
// upwind neighbours, their target slots and the weights once per
// interaction step; the sweeps then read the neighbours' previous values
// from the slot buffer (targets) or the plane (everything else).

__global__ void k3_ext_mark(Grid3 g, Region R, int group, const double *phi, const double *alpha,
                            const unsigned char *nostate, const double *sx, const double *sy,
                            const double *sz, int *map, Ext3 *plan, int *count, int cap,
                            int *err) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int grp = group < 2 ? blockIdx.y : 2;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  if (!(fabs(phi[c]) < g.bw)) return;
  if (grp < 2) {
    bool real = volk(alpha, grp, c) > S3_ALPHA_REAL && !nostate[(size_t)grp * g.NP + c];
    if (real) return;
  } else if (sx[c] != 0.0 || sy[c] != 0.0 || sz[c] != 0.0) {
    return;
  }
  int slot = atomicAdd(&count[grp], 1);
  if (slot >= cap) {
    atomicOr(err, S3_ERR_CAP);
    return;
  }
  map[(size_t)grp * g.NP + c] = slot;
  plan[(size_t)grp * cap + slot].cell = c;
}

__device__ inline void ext_setup_one(const Grid3 &g, int grp, const double *phi,
                                     const int *map, Ext3 *plan, int cap, int slot) {
  Ext3 &e = plan[(size_t)grp * cap + slot];
  int c = e.cell;
  int r = c, i = r % g.PX - S3_GH;
  r /= g.PX;
  int j = r % g.PY - S3_GH, kk = r / g.PY - S3_GH;
  double n[3];
  normal3(g, phi, c, n);
  bool flip = grp == 0 || (grp == 2 && phi[c] >= 0.0);
  if (flip)
    for (int d = 0; d < 3; d++) n[d] = -n[d];
  int s0 = n[0] >= 0.0 ? 1 : -1, s1 = n[1] >= 0.0 ? 1 : -1, s2 = n[2] >= 0.0 ? 1 : -1;
  double wx = fabs(n[0]) / g.dx, wy = fabs(n[1]) / g.dy, wz = fabs(n[2]) / g.dz;
  if (!in3(g, i + s0, j, kk)) wx = 0.0;
  if (!in3(g, i, j + s1, kk)) wy = 0.0;
  if (!in3(g, i, j, kk + s2)) wz = 0.0;
  // the upwind-weighted mean sum_d w_d v_d / sum_d w_d with the weights
  // normalised once per interaction step: each sweep then takes one
  // product and two FMAs per field instead of a division
  e.den = wx + wy + wz;
  const double iden = e.den > 0.0 ? 1.0 / e.den : 0.0;
  e.w[0] = wx * iden;
  e.w[1] = wy * iden;
  e.w[2] = wz * iden;
  e.nb[0] = c + s0;
  e.nb[1] = c + s1 * g.PX;
  e.nb[2] = c + s2 * g.PX * g.PY;
  for (int d = 0; d < 3; d++)
    e.slot[d] = e.w[d] > 0.0 ? map[(size_t)grp * g.NP + e.nb[d]] : -1;
}

// the list kernels run a bounded grid over the slots (the lists' lengths
// are known on the device only)
#define S3_LIST_BLOCKS (152 * 4)

__global__ void k3_ext_setup(Grid3 g, int group, const double *phi, const int *map,
                             Ext3 *plan, const int *count, int cap) {
  int grp = group < 2 ? blockIdx.y : 2;
  int n = min(count[grp], cap);
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += gridDim.x * blockDim.x)
    ext_setup_one(g, grp, phi, map, plan, cap, slot);
}

int k3_ext_plan(const Grid3 &g, const Region &R, int group, const double *phi,
                const double *alpha, const unsigned char *nostate, const double *sx,
                const double *sy, const double *sz, int *map, Ext3 *plan, int *count, int cap,
                int *err, cudaStream_t st) {
  // map holds -1 everywhere between plans (set at creation, restored by
  // the last sweep for the cells it marked)
  int groups = group < 2 ? 2 : 1, g0 = group < 2 ? 0 : 2;
  cudaMemsetAsync(count + g0, 0, sizeof(int) * groups, st);
  long long n = region_threads(g, R);
  if (n > 0)
    k3_ext_mark<<<dim3(nblk(n, 256), groups), 256, 0, st>>>(g, R, group, phi, alpha, nostate,
                                                            sx, sy, sz, map, plan, count, cap,
                                                            err);
  k3_ext_setup<<<dim3(std::min(nblk(cap, 128), S3_LIST_BLOCKS), groups), 128, 0, st>>>(
      g, group, phi, map, plan, count,
                                                              cap);
  tick(2);
  return 0;
}

struct ExtBufs {
  double *src[3][S3_NC];  // per group: the planes
  double *a, *b;          // slot buffers, [group][field][cap]
};

// one sweep: new value of each target from its neighbours' previous ones;
// first sweep (first = 1) takes the targets' own start values from the
// planes, the last one (last = 1) writes the results into the planes
__global__ void k3_ext_sweep(Grid3 g, int group, int nf, ExtBufs B, const Ext3 *plan,
                             const int *count, int cap, int first, int last, int iters,
                             int *map) {
  int grp = group < 2 ? blockIdx.y : 2;
  int n = min(count[grp], cap);
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += gridDim.x * blockDim.x) {
  const Ext3 &e = plan[(size_t)grp * cap + slot];
  const double *rd = B.a + (size_t)grp * S3_NC * cap;
  double *wr = B.b + (size_t)grp * S3_NC * cap;
  for (int m = 0; m < nf; m++) {
    double *P = B.src[grp][m];
    double val;
    if (iters == 0 || !(e.den > 0.0)) {
      val = first ? P[e.cell] : rd[(size_t)m * cap + slot];
    } else {
      double num = 0.0;
      for (int d = 0; d < 3; d++) {
        if (!(e.w[d] > 0.0)) continue;
        int s = e.slot[d];
        double v = (s >= 0 && !first) ? rd[(size_t)m * cap + s] : P[e.nb[d]];
        num += e.w[d] * v;
      }
      val = num;
    }
    if (last)
      P[e.cell] = val;
    else
      wr[(size_t)m * cap + slot] = val;
  }
  if (last) map[(size_t)grp * g.NP + e.cell] = -1;
  }
}

void k3_launch_ext_sweeps(const Grid3 &g, int group, int iters, const Ext3 *plan,
                          const int *count, int cap, double *const planes[], int nf,
                          double *bufA, double *bufB, int *map, cudaStream_t st) {
  // planes: for group < 2, 2 * S3_NC pointers (fluid N then P); else nf
  ExtBufs B{};
  int groups = group < 2 ? 2 : 1;
  for (int gr = 0; gr < groups; gr++)
    for (int m = 0; m < nf; m++) B.src[group < 2 ? gr : 2][m] = planes[gr * S3_NC + m];
  dim3 grid(std::min(nblk(cap, 128), S3_LIST_BLOCKS), groups);
  // sweep s reads the previous sweep's values (A) and writes B; the first
  // reads the planes, the last writes the planes (no sweep reads the planes'
  // targets after they changed: the last sweep's reads come from A)
  // (a single sweep writes the slot buffer and a second pass, with no
  // sweeping, copies it to the planes)
  double *a = bufA, *b = bufB;
  for (int s = 0; s < iters; s++) {
    B.a = a;
    B.b = b;
    k3_ext_sweep<<<grid, 128, 0, st>>>(g, group, nf, B, plan, count, cap, s == 0,
                                       iters > 1 && s == iters - 1, iters, map);
    double *t = a;
    a = b;
    b = t;
  }
  if (iters <= 1) {
    // no sweep left to write the planes (and restore the maps): a copy pass
    B.a = a;
    B.b = b;
    k3_ext_sweep<<<grid, 128, 0, st>>>(g, group, nf, B, plan, count, cap, iters == 0, 1, 0,
                                       map);
  }
  tick(iters + (iters <= 1));
}

// ---------------------------------------------------------------------
// Lax-Friedrichs speeds over every cell whose state can enter a stencil
// (real or in the band) and the CFL rate sum_d (|u_d| + c)/h_d over real
// cells; warp maxima, then one atomic per warp

__device__ inline double warp_max3(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// maxima of n values over the block (warp shuffles, then shared memory),
// one atomic per value and block: the maxima of a whole-grid launch would
// otherwise serialise on a few addresses
template <int N>
__device__ inline void block_max_atomic(double (&v)[N], unsigned long long *const (&dst)[N]) {
  __shared__ double part[N][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < N; q++) {
    double x = warp_max3(v[q]);
    if (lane == 0) part[q][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < N; q++) {
      double x = lane < nw ? part[q][lane] : 0.0;
      x = warp_max3(x);
      if (lane == 0) atomic_max_d(dst[q], x);
    }
  }
}

// grid-stride: a few blocks per SM, each thread keeping its maxima over
// many cells, so that few atomics reach the four addresses
__global__ void k3_wave_maxima(Grid3 g, Region R, int k, Planes3 w, const double *alpha,
                               const unsigned char *nostate, const double *phi, Scal3 *sc,
                               long long nthreads) {
  double l[3] = {0.0, 0.0, 0.0}, s = 0.0;
  const double hd[3] = {g.dx, g.dy, g.dz};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nthreads;
       t += (long long)gridDim.x * blockDim.x) {
    int i, j, kk;
    if (!region_cell(g, R, t, i, j, kk)) continue;
    int c = g3(g, i, j, kk);
    bool real = volk(alpha, k, c) > S3_ALPHA_REAL && !nostate[(size_t)k * g.NP + c];
    if (!(real || fabs(phi[c]) < g.bw)) continue;
    double rho = w.p[0][c], pr = w.p[4][c];
    double cs = sqrt(fmax(g.gamma[k] * (pr + g.pinf[k]) / rho, 0.0));
    double r = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      double a = fabs(w.p[1 + d][c]) + cs;
      l[d] = fmax(l[d], a);
      r += a / hd[d];
    }
    // explicit viscous limit 2 nu (1/dx^2 + 1/dy^2 + 1/dz^2)
    if (real && g.mu[k] > 0.0)
      r += 2.0 * g.mu[k] / rho *
           (1.0 / (hd[0] * hd[0]) + 1.0 / (hd[1] * hd[1]) + 1.0 / (hd[2] * hd[2]));
    if (real) s = fmax(s, r);
  }
  double v[4] = {l[0], l[1], l[2], s};
  unsigned long long *const dst[4] = {&sc->lf[k][0], &sc->lf[k][1], &sc->lf[k][2],
                                      &sc->smax[k]};
  block_max_atomic<4>(v, dst);
}

void k3_launch_wave_maxima(const Grid3 &g, const Region &R, int k, double *const w[S3_NC],
                           const double *alpha, const unsigned char *nostate, const double *phi,
                           Scal3 *sc, cudaStream_t st) {
  Planes3 W{};
  for (int m = 0; m < S3_NC; m++) W.p[m] = w[m];
  long long n = region_threads(g, R);
  if (n == 0) return;
  int blocks = std::min(nblk(n, 256), 152 * 8);
  k3_wave_maxima<<<blocks, 256, 0, st>>>(g, R, k, W, alpha, nostate, phi, sc, n);
  tick();
}

// ---------------------------------------------------------------------
// interface interaction: the exact two-material Riemann problem along n
// (fluid N left, P right), Newton on the star pressure from the acoustic
// guess with the pressure floor kept at a distance; either side may be a
// Tait fluid (barotropic shock branch)

// each side's wave function and derivative: the library's form with the
// quantities that do not depend on p taken once per problem and powers of
// the positive pressure ratio as exp2(e log2 r), one per side and iteration
// (sif_internal.cuh: side_const, riemann_side_k, riemann_star_density)

// mean curvature div(grad phi / |grad phi|) by second-order central
// differences: (sum over axes a of phi_aa times the squared gradient across
// a, minus twice the sum over axis pairs of phi_a phi_b phi_ab) / |grad
// phi|^3 (2 / r for a sphere, positive where fluid N is convex)
__device__ inline double curvature3(const Grid3 &g, const double *p, int c) {
  const double h[3] = {g.dx, g.dy, g.dz};
  const int st[3] = {1, g.PX, g.PX * g.PY};
  double gd[3], gg[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    gd[a] = (p[c + st[a]] - p[c - st[a]]) / (2.0 * h[a]);
    gg[a][a] = (p[c + st[a]] - 2.0 * p[c] + p[c - st[a]]) / (h[a] * h[a]);
  }
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = a + 1; b < 3; b++) {
      int sa = st[a], sb = st[b];
      gg[a][b] = (p[c + sa + sb] - p[c + sa - sb] - p[c - sa + sb] + p[c - sa - sb]) /
                 (4.0 * h[a] * h[b]);
    }
  double g2 = gd[0] * gd[0] + gd[1] * gd[1] + gd[2] * gd[2];
  if (!(g2 > 0.0)) return 0.0;
  double num = gg[0][0] * (gd[1] * gd[1] + gd[2] * gd[2]) +
               gg[1][1] * (gd[0] * gd[0] + gd[2] * gd[2]) +
               gg[2][2] * (gd[0] * gd[0] + gd[1] * gd[1]) -
               2.0 * (gd[0] * gd[1] * gg[0][1] + gd[0] * gd[2] * gg[0][2] + gd[1] * gd[2] * gg[1][2]);
  return num / (g2 * sqrt(g2));
}

// the cut cells (S != 0) of the region into a dense list, the exchange
// flux and interface velocity cleared everywhere in it: the Riemann
// problems then run on full warps (FP64 issue is the cost of a warp
// instruction, however few of its lanes hold a cut cell)
__global__ void k3_cut_list(Grid3 g, Region R, const double *sx, const double *sy,
                            const double *sz, Planes3 xn, Planes3 xp, Planes3 ul, int *list,
                            int *count, int cap, int *err) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  for (int m = 0; m < 4; m++) {
    xn.p[m][c] = 0.0;
    xp.p[m][c] = 0.0;
  }
  for (int d = 0; d < 3; d++) ul.p[d][c] = 0.0;
  if (sx[c] == 0.0 && sy[c] == 0.0 && sz[c] == 0.0) return;
  int slot = atomicAdd(count, 1);
  if (slot >= cap) {
    atomicOr(err, S3_ERR_CAP);
    return;
  }
  list[slot] = c;
}

__global__ void k3_interface(Grid3 g, const int *list, const int *count, int cap, Planes3 w0,
                             Planes3 w1, const double *phi, const double *sx, const double *sy,
                             const double *sz, Planes3 xn, Planes3 xp, Planes3 ul, Scal3 *sc) {
  double s0 = 0.0, s1 = 0.0;
  const int ncut = min(*count, cap);
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < ncut;
       slot += gridDim.x * blockDim.x) {
    int c = list[slot];
    double S[3] = {sx[c], sy[c], sz[c]};
    {
      double Sm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
      double nv[3];
      normal3(g, phi, c, nv);
      if (nv[0] == 0.0 && nv[1] == 0.0 && nv[2] == 0.0)
        for (int d = 0; d < 3; d++) nv[d] = S[d] / Sm;
      double rl = w0.p[0][c], pl = w0.p[4][c], gl = g.gamma[0], pil = g.pinf[0];
      double rr = w1.p[0][c], pr = w1.p[4][c], gr = g.gamma[1], pir = g.pinf[1];
      double ul_ = w0.p[1][c] * nv[0] + w0.p[2][c] * nv[1] + w0.p[3][c] * nv[2];
      double ur_ = w1.p[1][c] * nv[0] + w1.p[2][c] * nv[1] + w1.p[3][c] * nv[2];
      int bl = g.tait[0], br = g.tait[1];
      // Eq. 10: the N-side pressure exceeds the P side's by sigma kappa
      const double jump = g.sigma != 0.0 ? g.sigma * curvature3(g, phi, c) : 0.0;
      double cl = sqrt(gl * (pl + pil) / rl), cr = sqrt(gr * (pr + pir) / rr);
      double pscale = fmin(pl + pil, pr + pir);
      double pfloor = fmax(-pir, -pil - jump) + 1e-12 * pscale;
      double p = 0.5 * ((pl - jump) + pr) - 0.125 * (ur_ - ul_) * (rl + rr) * (cl + cr);
      if (p < pfloor) p = pfloor + 0.5 * (fmax(pl - jump, pr) - pfloor);
      int it = 0, conv = 0, done = 0;
      double fl, dfl, fr, dfr;
      const SideConst sl = side_const(rl, pl, gl, pil, cl, bl);
      const SideConst sr = side_const(rr, pr, gr, pir, cr, br);
      while (it < g.newton_iters) {
        it++;
        riemann_side_k(p + jump, sl, fl, dfl);
        riemann_side_k(p, sr, fr, dfr);
        double F = fl + fr + (ur_ - ul_);
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
      if (!(done || conv)) atomicOr(&sc->err, S3_ERR_NOCONV);
      const double plst = p + jump;
      riemann_side_k(plst, sl, fl, dfl);
      riemann_side_k(p, sr, fr, dfr);
      double us = 0.5 * (ul_ + ur_) + 0.5 * (fr - fl);
      double rsl = riemann_star_density(plst, rl, pl, gl, pil, bl);
      double rsr = riemann_star_density(p, rr, pr, gr, pir, br);
      double csl = sqrt(gl * (plst + pil) / rsl), csr = sqrt(gr * (p + pir) / rsr);
      // each fluid receives the exchange flux of its own interface pressure
      for (int d = 0; d < 3; d++) {
        xn.p[d][c] = -plst * S[d];
        xp.p[d][c] = p * S[d];
        ul.p[d][c] = us * nv[d];
      }
      xn.p[3][c] = -plst * us * Sm;
      xp.p[3][c] = p * us * Sm;
      if (g.mu[0] > 0.0 && g.mu[1] > 0.0) {
        // viscous traction across the interface (Eq. 5's interface term):
        // the stress of the velocity field that is continuous across it
        // (each cell's velocity from the fluid on its centre's side), by
        // central differences, with the harmonic-mean viscosity; fluid N
        // receives tau S and its work, fluid P the opposite
        const double muI = 2.0 * g.mu[0] * g.mu[1] / (g.mu[0] + g.mu[1]);
        const int st[3] = {1, g.PX, g.PX * g.PY};
        const double hd[3] = {g.dx, g.dy, g.dz};
        double G[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const int cp = c + st[a], cm = c - st[a];
          const Planes3 &wp = phi[cp] < 0.0 ? w0 : w1, &wm = phi[cm] < 0.0 ? w0 : w1;
#pragma unroll
          for (int b = 0; b < 3; b++) G[a][b] = (wp.p[1 + b][cp] - wm.p[1 + b][cm]) / (2.0 * hd[a]);
        }
        double tau[3][3];
        tau[0][0] = muI * (4.0 / 3.0 * G[0][0] - 2.0 / 3.0 * G[1][1] - 2.0 / 3.0 * G[2][2]);
        tau[1][1] = muI * (4.0 / 3.0 * G[1][1] - 2.0 / 3.0 * G[0][0] - 2.0 / 3.0 * G[2][2]);
        tau[2][2] = muI * (4.0 / 3.0 * G[2][2] - 2.0 / 3.0 * G[0][0] - 2.0 / 3.0 * G[1][1]);
        tau[0][1] = tau[1][0] = muI * (G[1][0] + G[0][1]);
        tau[0][2] = tau[2][0] = muI * (G[2][0] + G[0][2]);
        tau[1][2] = tau[2][1] = muI * (G[2][1] + G[1][2]);
        const Planes3 &wc = phi[c] < 0.0 ? w0 : w1;
        double f[3], e = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++) f[a] = tau[a][0] * S[0] + tau[a][1] * S[1] + tau[a][2] * S[2];
#pragma unroll
        for (int a = 0; a < 3; a++) e += wc.p[1 + a][c] * f[a];
#pragma unroll
        for (int a = 0; a < 3; a++) {
          xn.p[a][c] = xn.p[a][c] + f[a];
          xp.p[a][c] = xp.p[a][c] - f[a];
        }
        xn.p[3][c] = xn.p[3][c] + e;
        xp.p[3][c] = xp.p[3][c] - e;
      }
      double fac = 1.0 / g.dx + 1.0 / g.dy + 1.0 / g.dz;
      s0 = fmax(s0, (fabs(us) + csl) * fac);
      s1 = fmax(s1, (fabs(us) + csr) * fac);
    }
  }
  double v[2] = {s0, s1};
  unsigned long long *const dst[2] = {&sc->smax[0], &sc->smax[1]};
  block_max_atomic<2>(v, dst);
}

void k3_launch_interface(const Grid3 &g, const Region &R, double *const w[2][S3_NC],
                         const double *phi, const double *sx, const double *sy,
                         const double *sz, double *const xn[4], double *const xp[4],
                         double *const ul[3], int *cutlist, int *cutcount, int cap, Scal3 *sc,
                         cudaStream_t st) {
  Planes3 W0{}, W1{}, XN{}, XP{}, UL{};
  for (int m = 0; m < S3_NC; m++) {
    W0.p[m] = w[0][m];
    W1.p[m] = w[1][m];
  }
  for (int m = 0; m < 4; m++) {
    XN.p[m] = xn[m];
    XP.p[m] = xp[m];
  }
  for (int d = 0; d < 3; d++) UL.p[d] = ul[d];
  long long n = region_threads(g, R);
  if (n == 0) return;
  cudaMemsetAsync(cutcount, 0, sizeof(int), st);
  k3_cut_list<<<nblk(n, 256), 256, 0, st>>>(g, R, sx, sy, sz, XN, XP, UL, cutlist, cutcount, cap,
                                            &sc->err);
  // one warp per block: consecutive cut cells fill a warp, warps spread
  // over the SMs
  k3_interface<<<std::min(nblk(cap, 32), 4 * S3_LIST_BLOCKS), 32, 0, st>>>(
      g, cutlist, cutcount, cap, W0, W1, phi, sx, sy, sz, XN, XP, UL, sc);
  tick(2);
}

// ---------------------------------------------------------------------
// small-cell mixing (Sec. 2.2): sources (alpha_k < mix_alpha with content)
// plan their targets and the amounts from the pre-mix state; every cell
// then applies, in the order of the sources' cell indices (itself among
// them), what its neighbourhood's sources move in and out -- the serial
// in-place order, so the sums round alike

// the sources of the region into a dense list (the plan's slots), so that
// the plan's FP64 work runs on full warps
__global__ void k3_mix_sources(Grid3 g, Region R, int k, Planes3 q, const double *alpha,
                               Mix3 *plan, int *count, int cap, int *err) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  double as = volk(alpha, k, c);
  if (as >= g.mix_alpha) return;
  bool empty = as == 0.0;
  for (int m = 0; m < S3_NC; m++) empty = empty && q.p[m][c] == 0.0;
  if (empty) return;
  int slot = atomicAdd(count, 1);
  if (slot >= cap) {
    atomicOr(err, S3_ERR_CAP);
    return;
  }
  plan[slot].cell = c;
}

__device__ void mix_plan_one(const Grid3 &g, int k, const Planes3 &q, const double *alpha,
                             const double *phi, int *srcmap, Mix3 *plan, int slot) {
  Mix3 &P = plan[slot];
  const int c = P.cell;
  int r = c, i = r % g.PX - S3_GH;
  r /= g.PX;
  int j = r % g.PY - S3_GH, kk = r / g.PY - S3_GH;
  double as = volk(alpha, k, c);
  double nv[3];
  normal3(g, phi, c, nv);
  if (k == 0)
    for (int d = 0; d < 3; d++) nv[d] = -nv[d];
  int s0 = nv[0] >= 0.0 ? 1 : -1, s1 = nv[1] >= 0.0 ? 1 : -1, s2 = nv[2] >= 0.0 ? 1 : -1;
  const int di[7] = {s0, 0, 0, s0, s0, 0, s0};
  const int dj[7] = {0, s1, 0, s1, 0, s1, s1};
  const int dk[7] = {0, 0, s2, 0, s2, s2, s2};
  double wt[7] = {nv[0] * nv[0], nv[1] * nv[1], nv[2] * nv[2], fabs(nv[0] * nv[1]),
                  fabs(nv[0] * nv[2]), fabs(nv[1] * nv[2]), 0.0};
  double tri = fabs(nv[0] * nv[1] * nv[2]);
  wt[6] = tri > 0.0 ? pow(tri, 2.0 / 3.0) : 0.0;
  int keep = 0;
  double sum = 0.0;
  for (int q7 = 0; q7 < 7; q7++) {
    int ti = i + di[q7], tj = j + dj[q7], tk = kk + dk[q7];
    if (!in3(g, ti, tj, tk) || !(wt[q7] > 0.0)) continue;
    if (!(volk(alpha, k, g3(g, ti, tj, tk)) >= g.mix_alpha)) continue;
    keep |= 1 << q7;
    sum += wt[q7];
  }
  int single = -1;
  if (!(sum > 0.0)) {
    int best = -1;
    double ab = 0.0;
    const int dzs[3] = {0, -1, 1};
    for (int zz = 0; zz < 3; zz++)
      for (int b = -1; b <= 1; b++)
        for (int a = -1; a <= 1; a++) {
          int z = dzs[zz];
          if ((a == 0 && b == 0 && z == 0) || !in3(g, i + a, j + b, kk + z)) continue;
          int cn = g3(g, i + a, j + b, kk + z);
          double at = volk(alpha, k, cn);
          if (at > ab) {
            ab = at;
            best = cn;
          }
        }
    if (best >= 0 && ab >= g.mix_alpha) {
      single = best;
    } else {
      for (int q7 = 0; q7 < 7; q7++) {
        int ti = i + di[q7], tj = j + dj[q7], tk = kk + dk[q7];
        if (!in3(g, ti, tj, tk) || !(wt[q7] > 0.0)) continue;
        if (!(volk(alpha, k, g3(g, ti, tj, tk)) > as)) continue;
        keep |= 1 << q7;
        sum += wt[q7];
      }
    }
  }
  if (single < 0 && !(sum > 0.0)) {
    P.nt = 0;  // no target: nothing moves
    return;
  }
  int nt = 0;
  for (int q7 = 0; q7 < 7 && single < 0; q7++) {
    if (!(keep >> q7 & 1)) continue;
    P.tc[nt] = g3(g, i + di[q7], j + dj[q7], kk + dk[q7]);
    P.M[nt][0] = wt[q7] / sum;  // beta, replaced by the amounts below
    nt++;
  }
  if (single >= 0) {
    P.tc[0] = single;
    P.M[0][0] = 1.0;
    nt = 1;
  }
  P.nt = nt;
  for (int q7 = 0; q7 < nt; q7++) {
    int tc = P.tc[q7];
    double beta = P.M[q7][0];
    double at = volk(alpha, k, tc);
    double den = as * beta + at;
    for (int m = 0; m < S3_NC; m++)
      P.M[q7][m] = beta * (q.p[m][tc] * as - q.p[m][c] * at) / den;
  }
  srcmap[c] = slot;
}

__global__ void k3_mix_plan(Grid3 g, int k, Planes3 q, const double *alpha, const double *phi,
                            int *srcmap, Mix3 *plan, const int *count, int cap) {
  int n = min(*count, cap);
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += gridDim.x * blockDim.x)
    mix_plan_one(g, k, q, alpha, phi, srcmap, plan, slot);
}

// restores srcmap to -1 at the sources the plan marked
__global__ void k3_mix_unmark(int *srcmap, const Mix3 *plan, const int *count, int cap) {
  int n = min(*count, cap);
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += gridDim.x * blockDim.x)
    srcmap[plan[slot].cell] = -1;
}

__global__ void k3_mix_apply(Grid3 g, Region R, Planes3 q, const int *srcmap, const Mix3 *plan) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  int sz = g.PX * g.PY;
  bool any = false;
  for (int z = -1; z <= 1 && !any; z++)
    for (int b = -1; b <= 1 && !any; b++)
      for (int a = -1; a <= 1; a++)
        if (srcmap[c + a + b * g.PX + z * sz] >= 0) {
          any = true;
          break;
        }
  if (!any) return;
  double v[S3_NC];
  for (int m = 0; m < S3_NC; m++) v[m] = q.p[m][c];
  for (int z = -1; z <= 1; z++)
    for (int b = -1; b <= 1; b++)
      for (int a = -1; a <= 1; a++) {
        int cn = c + a + b * g.PX + z * sz;
        int s = srcmap[cn];
        if (s < 0) continue;
        const Mix3 &P = plan[s];
        for (int q7 = 0; q7 < P.nt; q7++) {
          if (cn == c) {
            for (int m = 0; m < S3_NC; m++) v[m] += P.M[q7][m];
          } else if (P.tc[q7] == c) {
            for (int m = 0; m < S3_NC; m++) v[m] -= P.M[q7][m];
          }
        }
      }
  for (int m = 0; m < S3_NC; m++) q.p[m][c] = v[m];
}

void k3_launch_mix(const Grid3 &g, const Region &R, int k, double *const q[S3_NC],
                   const double *alpha, const double *phi, int *srcmap, Mix3 *plan, int *count,
                   int cap, int *err, cudaStream_t st) {
  // srcmap holds -1 everywhere between calls (set at creation, restored
  // by k3_mix_unmark)
  Planes3 Q{};
  for (int m = 0; m < S3_NC; m++) Q.p[m] = q[m];
  long long n = region_threads(g, R);
  if (n == 0) return;
  cudaMemsetAsync(count, 0, sizeof(int), st);
  k3_mix_sources<<<nblk(n, 256), 256, 0, st>>>(g, R, k, Q, alpha, plan, count, cap, err);
  // one warp per block, as for the interface problems
  k3_mix_plan<<<std::min(nblk(cap, 32), 4 * S3_LIST_BLOCKS), 32, 0, st>>>(g, k, Q, alpha, phi,
                                                                          srcmap, plan, count,
                                                                          cap);
  k3_mix_apply<<<nblk(n, 256), 256, 0, st>>>(g, R, Q, srcmap, plan);
  k3_mix_unmark<<<std::min(nblk(cap, 256), S3_LIST_BLOCKS), 256, 0, st>>>(srcmap, plan, count,
                                                                           cap);
  tick(4);
}

// ---------------------------------------------------------------------
// level set (Eq. 6): narrow band |phi| < band h and its face neighbours,
// upwind HJ-WENO5 advection, RK stages masked to the band

__global__ void k3_band(Grid3 g, const double *phi, unsigned char *band) {
  long long n = (long long)g.nx * g.ny * g.nz;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i, j, kk;
  cell_ijk(g, (int)t, i, j, kk);
  int c = g3(g, i, j, kk);
  band[c] = fabs(phi[c]) < g.bw;
}

__global__ void k3_rext(Grid3 g, const unsigned char *band, unsigned char *rext) {
  long long n = (long long)g.nx * g.ny * g.nz;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i, j, kk;
  cell_ijk(g, (int)t, i, j, kk);
  int c = g3(g, i, j, kk), sz = g.PX * g.PY;
  int r = band[c];
  if (i > 0) r |= band[c - 1];
  if (i < g.nx - 1) r |= band[c + 1];
  if (j > 0) r |= band[c - g.PX];
  if (j < g.ny - 1) r |= band[c + g.PX];
  if (kk > 0) r |= band[c - sz];
  if (kk < g.nz - 1) r |= band[c + sz];
  rext[c] = (unsigned char)r;
}

void k3_launch_band(const Grid3 &g, const double *phi, unsigned char *band,
                    unsigned char *rext, cudaStream_t st) {
  long long n = (long long)g.nx * g.ny * g.nz;
  k3_band<<<nblk(n, 256), 256, 0, st>>>(g, phi, band);
  k3_rext<<<nblk(n, 256), 256, 0, st>>>(g, band, rext);
  tick(2);
}

__device__ inline double weno5_3(double v1, double v2, double v3, double v4, double v5,
                                 double eps) {
  double q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0;
  double q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0;
  double q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0;
  double b0 = 13.0 / 12.0 * sq3(v1 - 2.0 * v2 + v3) + 0.25 * sq3(v1 - 4.0 * v2 + 3.0 * v3);
  double b1 = 13.0 / 12.0 * sq3(v2 - 2.0 * v3 + v4) + 0.25 * sq3(v2 - v4);
  double b2 = 13.0 / 12.0 * sq3(v3 - 2.0 * v4 + v5) + 0.25 * sq3(3.0 * v3 - 4.0 * v4 + v5);
  double a0 = 0.1 / sq3(eps + b0);
  double a1 = 0.6 / sq3(eps + b1);
  double a2 = 0.3 / sq3(eps + b2);
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// one-sided HJ-WENO5 derivative along stride s (backward-biased if bw)
__device__ inline double hj3(const double *p, int c, int s, double h, bool bw, double eps) {
  double v[5];
  if (bw) {
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
  return weno5_3(v[0], v[1], v[2], v[3], v[4], eps);
}

__global__ void k3_ls_rhs(Grid3 g, Region R, const double *phi, Planes3 ul, const unsigned char *band,
                          double *L) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  if (!band[c]) {
    L[c] = 0.0;
    return;
  }
  const int st[3] = {1, g.PX, g.PX * g.PY};
  const double hd[3] = {g.dx, g.dy, g.dz};
  double r = 0.0;
  for (int d = 0; d < 3; d++) {
    double u = ul.p[d][c];
    if (u != 0.0) r += u * hj3(phi, c, st[d], hd[d], u > 0.0, g.eps);
  }
  L[c] = -r;
}

void k3_launch_ls_rhs(const Grid3 &g, const Region &R, const double *phi, double *const ul[3],
                      const unsigned char *band, double *lphi, cudaStream_t st) {
  Planes3 U{};
  for (int d = 0; d < 3; d++) U.p[d] = ul[d];
  long long n = region_threads(g, R);
  if (n == 0) return;
  k3_ls_rhs<<<nblk(n, 128), 128, 0, st>>>(g, R, phi, U, band, lphi);
  tick();
}

// dst = dst + dt L (stage 1) or base/2 + (dst + dt L)/2 (stage 2) where mask
__global__ void k3_rk(Grid3 g, Region R, int stage, double *dst, const double *base, const double *L,
                      double dt, const unsigned char *mask) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  if (mask && !mask[c]) return;
  if (stage == 1)
    dst[c] = dst[c] + dt * L[c];
  else
    dst[c] = 0.5 * base[c] + 0.5 * (dst[c] + dt * L[c]);
}

void k3_launch_rk(const Grid3 &g, const Region &R, int stage, double *dst, const double *base,
                  const double *L, double dt, const unsigned char *mask, cudaStream_t st) {
  long long n = region_threads(g, R);
  if (n == 0) return;
  k3_rk<<<nblk(n, 256), 256, 0, st>>>(g, R, stage, dst, base, L, dt, mask);
  tick();
}

__device__ inline double grad_est3(const double *p, int c, int s, double h) {
  double dm = fabs(p[c] - p[c - s]), dp = fabs(p[c + s] - p[c]);
  double dc = 0.5 * fabs(p[c + s] - p[c - s]);
  return fmax(fmax(dc, dp), dm) / h;
}

// one reinitialisation sweep over the band and its face neighbours: the
// subcell fix where phi0 changes sign across a face, Godunov's Hamiltonian
// with one-sided HJ-WENO5 derivatives elsewhere, no new extremum
__global__ void k3_reinit(Grid3 g, Region R, double *phi, const double *q, const double *z,
                          const unsigned char *rext) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  if (!rext[c]) return;
  const int st[3] = {1, g.PX, g.PX * g.PY};
  const double hd[3] = {g.dx, g.dy, g.dz};
  double s0 = z[c];
  bool pos = s0 >= 0.0;
  bool cut = false;
  for (int d = 0; d < 3; d++)
    cut = cut || (z[c - st[d]] >= 0.0) != pos || (z[c + st[d]] >= 0.0) != pos;
  if (cut) {
    double gd[3], gm = 0.0;
    for (int d = 0; d < 3; d++) {
      gd[d] = (z[c + st[d]] - z[c - st[d]]) / (2.0 * hd[d]);
      gm += gd[d] * gd[d];
    }
    gm = sqrt(gm);
    if (!(gm > 1e-8)) {
      gm = 0.0;
      for (int d = 0; d < 3; d++) {
        gd[d] = grad_est3(z, c, st[d], hd[d]);
        gm += gd[d] * gd[d];
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
    phi[c] = q[c] - 0.5 * (sg * fabs(q[c]) - D);
  } else {
    if (s0 == 0.0) return;
    double h = g.h;
    double S = s0 / sqrt(s0 * s0 + h * h);
    double G = 0.0;
    for (int d = 0; d < 3; d++) {
      double a = hj3(q, c, st[d], hd[d], true, g.eps);
      double b = hj3(q, c, st[d], hd[d], false, g.eps);
      if (s0 > 0.0)
        G += fmax(sq3(fmax(a, 0.0)), sq3(fmin(b, 0.0)));
      else
        G += fmax(sq3(fmin(a, 0.0)), sq3(fmax(b, 0.0)));
    }
    double nv = q[c] - 0.5 * h * S * (sqrt(G) - 1.0);
    double lo = q[c - 1], hi = q[c - 1];
    for (int d = 0; d < 3; d++)
      for (int sd = -1; sd <= 1; sd += 2) {
        lo = fmin(lo, q[c + sd * st[d]]);
        hi = fmax(hi, q[c + sd * st[d]]);
      }
    if (s0 > 0.0 && nv < lo) nv = lo;
    if (s0 < 0.0 && nv > hi) nv = hi;
    phi[c] = nv;
  }
}

void k3_launch_reinit(const Grid3 &g, const Region &R, double *phi, const double *old,
                      const double *p0, const unsigned char *rext, cudaStream_t st) {
  long long n = region_threads(g, R);
  if (n == 0) return;
  k3_reinit<<<nblk(n, 128), 128, 0, st>>>(g, R, phi, old, p0, rext);
  tick();
}

// ---------------------------------------------------------------------
// the accelerated cycle's pieces: Eq. 8-9 records, Eq. 7 interpolation,
// the final correction, and the volume integrals

__global__ void k3_record(Grid3 g, Region R, int shared, Planes3 x1, Planes3 xc, double dt1,
                          double dt2) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  for (int m = 0; m < 4; m++) {
    double x = x1.p[m][c];
    double v = xc.p[m][c];
    if (shared) v = v + (-0.5 * x) * dt1;
    xc.p[m][c] = v + (0.5 * x) * dt2;
  }
}

void k3_launch_record(const Grid3 &g, const Region &R, int shared, double *const x1[4],
                      double *const xc[4], double dt1, double dt2, cudaStream_t st) {
  Planes3 X{}, C{};
  for (int m = 0; m < 4; m++) {
    X.p[m] = x1[m];
    C.p[m] = xc[m];
  }
  long long n = region_threads(g, R);
  if (n == 0) return;
  k3_record<<<nblk(n, 256), 256, 0, st>>>(g, R, shared, X, C, dt1, dt2);
  tick();
}

__global__ void k3_interp(Grid3 g, Region R, Planes3 qi, Planes3 prev, Planes3 fut, double th) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, kk;
  if (!region_cell(g, R, t, i, j, kk)) return;
  int c = g3(g, i, j, kk);
  for (int m = 0; m < S3_NC; m++) qi.p[m][c] = (1.0 - th) * prev.p[m][c] + th * fut.p[m][c];
}

void k3_launch_interp(const Grid3 &g, const Region &R, double *const qi[S3_NC],
                      double *const prev[S3_NC], double *const fut[S3_NC], double th,
                      cudaStream_t st) {
  Planes3 A{}, B{}, C{};
  for (int m = 0; m < S3_NC; m++) {
    A.p[m] = qi[m];
    B.p[m] = prev[m];
    C.p[m] = fut[m];
  }
  long long n = region_threads(g, R);
  if (n == 0) return;
  k3_interp<<<nblk(n, 256), 256, 0, st>>>(g, R, A, B, C, th);
  tick();
}

__global__ void k3_correction(Grid3 g, Planes3 q, Planes3 xc, double dv) {
  long long n = (long long)g.nx * g.ny * g.nz;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i, j, kk;
  cell_ijk(g, (int)t, i, j, kk);
  int c = g3(g, i, j, kk);
  // cells with nothing recorded (all but those an evaluation found cut)
  // would add 0 / dv
  if (xc.p[0][c] == 0.0 && xc.p[1][c] == 0.0 && xc.p[2][c] == 0.0 && xc.p[3][c] == 0.0) return;
  for (int m = 0; m < 4; m++) q.p[m + 1][c] += xc.p[m][c] / dv;
}

void k3_launch_correction(const Grid3 &g, double *const q[S3_NC], double *const xc[4],
                          double dv, cudaStream_t st) {
  Planes3 Q{}, X{};
  for (int m = 0; m < S3_NC; m++) Q.p[m] = q[m];
  for (int m = 0; m < 4; m++) X.p[m] = xc[m];
  long long n = (long long)g.nx * g.ny * g.nz;
  k3_correction<<<nblk(n, 256), 256, 0, st>>>(g, Q, X, dv);
  tick();
}

// per (fluid, component, z-slab of cells) partial sums in a fixed order;
// the host adds the partials
__global__ void k3_integrals(Grid3 g, Planes3 q0, Planes3 q1, double *partial) {
  int comp = blockIdx.y, k = comp / S3_NC, m = comp % S3_NC;
  int kk = blockIdx.x;
  const double *p = (k ? q1 : q0).p[m];
  __shared__ double red[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < g.nx * g.ny; t += blockDim.x) {
    int i = t % g.nx, j = t / g.nx;
    s += p[g3(g, i, j, kk)];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(size_t)comp * g.nz + kk] = red[0];
}

void k3_launch_integrals(const Grid3 &g, double *const q[2][S3_NC], double *partial,
                         cudaStream_t st) {
  Planes3 A{}, B{};
  for (int m = 0; m < S3_NC; m++) {
    A.p[m] = q[0][m];
    B.p[m] = q[1][m];
  }
  k3_integrals<<<dim3(g.nz, 2 * S3_NC), 256, 0, st>>>(g, A, B, partial);
  tick();
}
