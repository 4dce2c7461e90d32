// sif_internal.cuh -- device-side data structures and the pointwise
// formulas shared by the CUDA translation units of libsif.
//
// Layout: every field is an FP64 plane of PX x PY doubles with GH ghost
// layers on each side; cell (i, j), -GH <= i < nx + GH, lives at
// (i + GH) + (j + GH) * PX.  PX is padded to a multiple of 16 doubles so
// that every row starts on a 128-byte boundary relative to the plane base.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sif.h"

#define SIF_GH 3
// a cell holds fluid k for stencil/CFL purposes only if alpha_k exceeds
// this; round-off slivers take extended states instead
#define SIF_ALPHA_REAL 1e-6

// default finite-volume tile (outputs per CTA); others: sif_set_tile_shape
#define FV_TX 32
#define FV_TY 8

// device error bits
#define DERR_NONPHYS 1
#define DERR_NOCONV 2
#define DERR_TIMEOUT 4

struct Grid {
  int dim, nx, ny, PX, PY;
  double dx, dy, h;
  int bc[4];
  double gamma[2], pinf[2];
  double cfl, weno_eps, mix_alpha, band;
  int ext_iters, reinit_iters;
  int weno_char;  // finite-volume reconstruction on characteristic fields
  int flux;       // face flux: 0 WENO5-LF, 1 HLLC on WENO5 primitive states
  double sigma;   // surface tension coefficient (Eq. 10), 0 = none
  double mu[2];   // dynamic viscosities of fluids N and P, 0 = inviscid
  int tx, ty;    // finite-volume tile shape (output cells per CTA)
  int ntx, nty;  // tiles per direction
  int newton_max;  // Newton iterations allowed per interface Riemann problem
  // Tait's equation (Eq. 4) per fluid: p = tB ((rho/trho0)^gamma - 1) + tp0
  // (pinf is then tB - tp0)
  int tait[2];
  double tB[2], trho0[2], tp0[2];
};

// Scalars that live in device memory so that a whole step can run without
// a host round trip.  Maxima of non-negative doubles are kept as their bit
// patterns (ordered like the values) for atomicMax.
struct Scalars {
  unsigned long long smax[2];   // CFL wave-speed sums per fluid
  unsigned long long lf[2][2];  // Lax-Friedrichs alpha per fluid, direction
  double t, t_end;
  double dt;                    // single-dt step
  double dt1, dt2, t2, theta;   // multi-dt cycle
  double n_raw, n_used;
  int f1, mode, last, sub;
  int err;
  int n_band, n_etile;        // interaction-step band and its extension tiles
  int n_tiles[2];             // finite-volume tiles per fluid (cleared with the two above)
  int n_band_ls, n_rext;      // level-set step band and its face neighbours
  int n_cut, n_pad_;
  double dtk_raw[2];
  double dt2_first;             // fluid-2 step chosen at the start of the cycle
  unsigned long long updates;   // (cell, fluid) stage updates issued (active-tile cells)
  unsigned long long open_updates;  // of those, cells with an open face of the fluid
  // RK3 cycle: the sub-step boundaries around fluid 1's third-stage time
  // (t^n + dt1/2) whose level sets are kept, and the copy decisions
  double ta, tb;
  int have_a, have_b, snap_a, snap_b, single, pad_;  // (pad_ keeps the timer block aligned)
  // finite-volume launch timing on the GPU's global timer (graph-safe):
  // each launch keeps its earliest block start and latest block end, the
  // last block to finish adds the span to fv_ns
  int timing;
  unsigned int fv_blocks_done;
  unsigned long long fv_t0, fv_t1, fv_ns, fv_launches;
};

// every kernel counts its own launches on the device (one atomic by the
// first thread of the first block); each translation unit has its counter
static __device__ unsigned long long g_tu_launches;
#define SIF_TICK()                                                                    \
  do {                                                                                \
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)     \
      atomicAdd(&g_tu_launches, 1ull);                                                \
  } while (0)

// kernel launch through the launch-configuration form (the geometry, band,
// plan and adjoint kernels; the finite-volume stage sets its priority)
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}
unsigned long long sif_launches_geom();
unsigned long long sif_launches_band();
unsigned long long sif_launches_plan();
unsigned long long sif_launches_fv();
#define SIF_TU_LAUNCH_READER(name)                                                    \
  unsigned long long sif_launches_##name() {                                          \
    unsigned long long v = 0;                                                         \
    cudaMemcpyFromSymbol(&v, g_tu_launches, sizeof(v));                               \
    return v;                                                                         \
  }

// upwind neighbours (cell indices, -1 = unused) and normalised weights of
// one extension target; cx = cy = -1 marks a cell that is not a target
struct ExtPlan {
  int cx, cy;  // upwind neighbours (cell index) or -1
  int bx, by;  // their band positions, -1 outside the band
  double wx, wy;
};

// a small-cell mixing source: its targets (cell indices), weights and
// volume fractions; nt = 0 marks a cell that is not a source
struct MixPlan {
  int tc[3];
  int nt;
  double beta[3], at[3], as;
  double M[3][4];  // conserved amount moved from target t to the source
};

__host__ __device__ inline int gidx(const Grid &g, int i, int j) {
  return (i + SIF_GH) + (j + SIF_GH) * g.PX;
}

__device__ inline double ull_as_double(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ inline unsigned long long double_as_ull(double v) { return (unsigned long long)__double_as_longlong(v); }

// max of non-negative doubles via the ordered bit pattern
__device__ inline void atomic_max_pos(unsigned long long *addr, double v) {
  if (v > 0.0) atomicMax(addr, double_as_ull(v));
}

__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------
// geometry (Sec. 2.1, Fig. 1); operation order identical to the CPU
// reference so that sign and threshold decisions agree

__device__ inline double edge_fraction(double a, double b) {
  if (a >= 0.0 && b >= 0.0) return 1.0;
  if (a < 0.0 && b < 0.0) return 0.0;
  if (a >= 0.0) return a / (a - b);
  return b / (b - a);
}

__device__ inline double cell_alpha(double c00, double c10, double c11, double c01) {
  const double v[4] = {c00, c10, c11, c01};
  const double px[4] = {0.0, 1.0, 1.0, 0.0};
  const double py[4] = {0.0, 0.0, 1.0, 1.0};
  int npos = 0, changes = 0;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    if (v[e] >= 0.0) npos++;
    if ((v[e] >= 0.0) != (v[(e + 1) & 3] >= 0.0)) changes++;
  }
  if (npos == 4) return 1.0;
  if (npos == 0) return 0.0;
  if (changes == 4) {
    double area = 0.0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      if (v[e] < 0.0) continue;
      int n = (e + 1) & 3, p = (e + 3) & 3;
      double l1 = v[e] / (v[e] - v[n]);
      double l2 = v[e] / (v[e] - v[p]);
      area += 0.5 * l1 * l2;
    }
    return area;
  }
  // the positive part's polygon, its vertices taken in order around the
  // cell; the shoelace sum gathers each edge's term as its end vertex
  // comes and closes with the edge back to the first (the same terms in
  // the same order as over a stored vertex list, in registers)
  double x0 = 0.0, y0 = 0.0, xl = 0.0, yl = 0.0, a2 = 0.0;
  bool first = true;
  auto vertex = [&](double x, double y) {
    if (first) {
      x0 = x;
      y0 = y;
      first = false;
    } else {
      a2 += xl * y - x * yl;
    }
    xl = x;
    yl = y;
  };
#pragma unroll
  for (int e = 0; e < 4; e++) {
    int n = (e + 1) & 3;
    if (v[e] >= 0.0) vertex(px[e], py[e]);
    if ((v[e] >= 0.0) != (v[n] >= 0.0)) {
      double s = v[e] / (v[e] - v[n]);
      vertex(px[e] + s * (px[n] - px[e]), py[e] + s * (py[n] - py[e]));
    }
  }
  a2 += xl * y0 - x0 * yl;
  return 0.5 * a2;
}

// level set at the lower-left corner of cell (i, j)
__device__ inline double corner_phi(const Grid &g, const double *p, int i, int j) {
  return 0.25 * ((p[gidx(g, i - 1, j - 1)] + p[gidx(g, i, j - 1)]) +
                 (p[gidx(g, i - 1, j)] + p[gidx(g, i, j)]));
}

__device__ inline void unit_normal(const Grid &g, const double *p, int i, int j,
                                   double &nx, double &ny) {
  double gx = (p[gidx(g, i + 1, j)] - p[gidx(g, i - 1, j)]) / (2.0 * g.dx);
  double gy = g.dim == 2 ? (p[gidx(g, i, j + 1)] - p[gidx(g, i, j - 1)]) / (2.0 * g.dy) : 0.0;
  double m = sqrt(gx * gx + gy * gy);
  if (m > 0.0) {
    nx = gx / m;
    ny = gy / m;
  } else {
    nx = 0.0;
    ny = 0.0;
  }
}

// index of the interior cell whose value ghost index i (of n interior
// cells, boundary kinds bl / br) takes, and whether a reflecting wall lies
// between them (the velocity component normal to it changes sign)
__device__ inline int ghost_image(int i, int n, int bl, int br, bool &flip) {
  flip = false;
  if (i < 0) {
    int m = -1 - i;
    if (bl == SIF_BC_REFLECT) {
      flip = true;
      return m;
    }
    return bl == SIF_BC_PERIODIC ? n - 1 - m : 0;
  }
  if (i >= n) {
    int m = i - n;
    if (br == SIF_BC_REFLECT) {
      flip = true;
      return n - 1 - m;
    }
    return br == SIF_BC_PERIODIC ? m : n - 1;
  }
  return i;
}

// the indices along one direction that take interior cell a's value: a
// itself and the ghost indices whose image is a (at most 1 + 2 SIF_GH)
__device__ inline int ghost_preimages(int a, int n, int bl, int br, int out[1 + 2 * SIF_GH]) {
  int k = 0;
  out[k++] = a;
  for (int m = 0; m < SIF_GH; m++) {
    bool f;
    if (ghost_image(-1 - m, n, bl, br, f) == a) out[k++] = -1 - m;
    if (ghost_image(n + m, n, bl, br, f) == a) out[k++] = n + m;
  }
  return k;
}

__device__ inline bool inside(const Grid &g, int i, int j) {
  return i >= 0 && i < g.nx && j >= 0 && j < g.ny;
}

__device__ inline double vol_k(const double *alphaP, int k, int c) {
  return k == 1 ? alphaP[c] : 1.0 - alphaP[c];
}

// ---------------------------------------------------------------------
// 1/d for a positive normal d below 2^1000 (so that 1/d is normal too):
// Newton's iteration for the reciprocal, x <- x + x e with e = 1 - d x,
// taken to third order, x <- x + x (e + e^2), from the device's approximate
// reciprocal (rcp.approx.ftz.f64).  The relative error after the step is
// the cube of the seed's; measured on GB300 the seed is good to 2^-19.9 and
// the result within 1 ulp of the correctly rounded 1/d
// (sif_probe_reciprocal checks it against IEEE division).
__device__ inline double recip_newton3(double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  double e = fma(-d, x, 1.0);
  return fma(x, fma(e, e, e), x);
}

// ---------------------------------------------------------------------
// WENO5-JS reconstruction in the plain form (used by the level set and
// reinitialisation kernels, which follow the CPU reference op by op)

__device__ inline double sqd(double a) { return a * a; }

__device__ inline double weno5_plain(double v1, double v2, double v3, double v4, double v5,
                                     double eps) {
  double q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0;
  double q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0;
  double q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0;
  double b0 = 13.0 / 12.0 * sqd(v1 - 2.0 * v2 + v3) + 0.25 * sqd(v1 - 4.0 * v2 + 3.0 * v3);
  double b1 = 13.0 / 12.0 * sqd(v2 - 2.0 * v3 + v4) + 0.25 * sqd(v2 - v4);
  double b2 = 13.0 / 12.0 * sqd(v3 - 2.0 * v4 + v5) + 0.25 * sqd(3.0 * v3 - 4.0 * v4 + v5);
  double a0 = 0.1 / sqd(eps + b0);
  double a1 = 0.6 / sqd(eps + b1);
  double a2 = 0.3 / sqd(eps + b2);
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// ---------------------------------------------------------------------
// exact two-material stiffened-gas Riemann problem (interface interaction);
// the Newton derivative shares the rarefaction power with the function, and
// powers of a positive pressure ratio are taken as exp2(e log2 r) (shorter
// dependent chains than a general pow), so iterates differ from the CPU
// reference by rounding while the converged star state agrees to round-off

// r^e for r > 0
__device__ inline double pos_pow(double r, double e) { return exp2(e * log2(r)); }

__device__ inline void riemann_side(double p, double rho, double pk, double g, double pi,
                                    double ck, double &f, double &df, int baro = 0) {
  double P = pk + pi, Pp = p + pi;
  if (p > pk && baro) {
    // barotropic shock (Tait's equation): u jump^2 = (p - pk)(1/rho -
    // 1/rho*), rho* = rho r^(1/g), r = (p + pi)/(pk + pi); 1 - r^(-1/g)
    // taken without cancellation for r near 1
    double x = (p - pk) / P;
    double a = -expm1(-log1p(x) / g);
    double gsq = (p - pk) * a / rho;
    double dg = (a + (p - pk) * pos_pow(1.0 + x, -1.0 / g - 1.0) / (g * P)) / rho;
    f = sqrt(gsq);
    df = dg / (2.0 * f);
  } else if (p > pk) {
    double A = 2.0 / ((g + 1.0) * rho);
    double B = (g - 1.0) / (g + 1.0) * P;
    double qr = sqrt(A / (Pp + B));
    f = (p - pk) * qr;
    df = qr * (1.0 - 0.5 * (p - pk) / (Pp + B));
  } else {
    // r^(-(g+1)/(2g)) = r^((g-1)/(2g)) / r: one power per side and iteration
    double r = Pp / P;
    double ra = pos_pow(r, (g - 1.0) / (2.0 * g));
    f = 2.0 * ck / (g - 1.0) * (ra - 1.0);
    df = 1.0 / (rho * ck) * (ra / r);
  }
}

// riemann_side with the quantities that do not depend on p computed once
// per Riemann problem (the same operations, so the same values)
struct SideConst {
  double rho, pk, g, pi, P, A, B, fr, dr, e, eb, gP;
  int baro;
};

__device__ inline SideConst side_const(double rho, double pk, double g, double pi, double ck,
                                       int baro) {
  SideConst s;
  s.rho = rho, s.pk = pk, s.g = g, s.pi = pi, s.baro = baro;
  s.P = pk + pi;
  s.A = 2.0 / ((g + 1.0) * rho);
  s.B = (g - 1.0) / (g + 1.0) * s.P;
  s.fr = 2.0 * ck / (g - 1.0);
  s.dr = 1.0 / (rho * ck);
  s.e = (g - 1.0) / (2.0 * g);
  s.eb = -1.0 / g - 1.0;
  s.gP = g * s.P;
  return s;
}

__device__ inline void riemann_side_k(double p, const SideConst &s, double &f, double &df) {
  const double Pp = p + s.pi;
  if (p > s.pk && s.baro) {
    double x = (p - s.pk) / s.P;
    double a = -expm1(-log1p(x) / s.g);
    double gsq = (p - s.pk) * a / s.rho;
    double dg = (a + (p - s.pk) * pos_pow(1.0 + x, s.eb) / s.gP) / s.rho;
    f = sqrt(gsq);
    df = dg / (2.0 * f);
  } else if (p > s.pk) {
    double qr = sqrt(s.A / (Pp + s.B));
    f = (p - s.pk) * qr;
    df = qr * (1.0 - 0.5 * (p - s.pk) / (Pp + s.B));
  } else {
    double r = Pp / s.P;
    double ra = pos_pow(r, s.e);
    f = s.fr * (ra - 1.0);
    df = s.dr * (ra / r);
  }
}

__device__ inline double riemann_star_density(double p, double rho, double pk, double g, double pi,
                                             int baro = 0) {
  double r = (p + pi) / (pk + pi);
  if (p > pk && !baro) {
    double qq = (g - 1.0) / (g + 1.0);
    return rho * (r + qq) / (qq * r + 1.0);
  }
  return rho * pos_pow(r, 1.0 / g);
}

// returns 0 or DERR_NOCONV; out: p*, u*, c*_L, c*_R
__device__ inline int riemann_solve(double rl, double ul, double pl, double gl, double pil,
                                    double rr, double ur, double pr, double gr, double pir,
                                    double &ps, double &us, double &csl, double &csr) {
  double cl = sqrt(gl * (pl + pil) / rl), cr = sqrt(gr * (pr + pir) / rr);
  double pscale = fmin(pl + pil, pr + pir);
  double pfloor = -fmin(pil, pir) + 1e-12 * pscale;
  double p = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
  if (p < pfloor) p = pfloor + 0.5 * (fmax(pl, pr) - pfloor);
  int it = 0, conv = 0, done = 0;
  double fl, dfl, fr, dfr;
  while (it < 50) {
    it++;
    riemann_side(p, rl, pl, gl, pil, cl, fl, dfl);
    riemann_side(p, rr, pr, gr, pir, cr, fr, dfr);
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
  riemann_side(p, rl, pl, gl, pil, cl, fl, dfl);
  riemann_side(p, rr, pr, gr, pir, cr, fr, dfr);
  us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  double rsl = riemann_star_density(p, rl, pl, gl, pil);
  double rsr = riemann_star_density(p, rr, pr, gr, pir);
  ps = p;
  csl = sqrt(gl * (p + pil) / rsl);
  csr = sqrt(gr * (p + pir) / rsr);
  return (done || conv) ? 0 : DERR_NOCONV;
}

// ---------------------------------------------------------------------
// host-side launch wrappers (defined in the .cu files); each reports the
// number of kernels it launched to the profiling counter
void sif_note_launches(int n);

// ghost layers of up to 8 planes; vel[m]: 0 scalar, 1 x-velocity, 2 y-velocity
struct GhostSet {
  double *p[8];
  int vel[8];
  int n;
};
void launch_fill_ghost(const Grid &g, const GhostSet &s, cudaStream_t st);
// band != null: only the cells of that band list (the band of the phi the
// geometry was last computed from, with a level-set step since)
void launch_geometry(const Grid &g, const double *phi, double *alpha, double *ax, double *ay,
                     double *sx, double *sy, int *cut_list, Scalars *sc, cudaStream_t st,
                     const int *band = nullptr, const int *nband = nullptr, int band_cap = 0);
// counts[0] = band size, counts[1] = band + face neighbours (if rext)
void launch_band_lists(const Grid &g, const double *phi, int *band, int *rext, int *counts,
                       cudaStream_t st);
// band list and map, the list of SIF_ETILE^2 tiles holding band cells (for
// the blocked extension) and the finite-volume tile lists of both fluids,
// in one launch (counts in sc->n_band, n_etile, n_tiles)
void launch_band_tiles(const Grid &g, const double *phi, int *band, int *map, int *etiles,
                       int *tiles0, int *tiles1, Scalars *sc, cudaStream_t st);
// edge of the square tiles of the blocked extension
#define SIF_ETILE 16
// sweep counts the blocked extension takes (its tile's halo is that wide)
#define SIF_EXT_BLOCKED_MAX 12
int ext_tiles(const Grid &g);
bool ext_blocked_ok(const Grid &g);
// all g.ext_iters Jacobi sweeps of fields [f0, f0 + nf) (W_N and W_P
// together, from the band values launch_ext_setup copied to tmp, or the
// level-set velocity alone) over the band tiles, with the write-back of the
// band values (and the stencil states' wave speeds)
void launch_ext_blocked(const Grid &g, double *const wN[4], double *const wP[4], double *ul0,
                        double *ul1, int f0, int nf, const ExtPlan *plan, int cap,
                        const int *etiles, const int *nband, const int *map, const int *band,
                        int work, double *tmp, const double *alpha,
                        const unsigned char *const nostate[2], Scalars *sc, int num_sms,
                        cudaStream_t st);
void ext_prepare();
void launch_mix2(const Grid &g, int mask, double *const qN[4], double *const qP[4],
                 const double *alpha, const double *phi, const int *band, const int *map,
                 const int *nband, MixPlan *plan, int cap, int work, double *tmp,
                 cudaStream_t st);
// nostate[k]: 1 where a cut cell of fluid k holds no physical state (set by
// the primitive recovery of the same interaction step)
// sweep0 != null: also the first Jacobi sweep of both fluids' stencil
// states wN, wP into the sweep buffer (then launch_ext_sweeps with
// first_done), or with copy the band cells' own values (then
// launch_ext_blocked, which reads them there)
void launch_ext_setup(const Grid &g, const double *alpha, const double *phi, const double *sx,
                      const double *sy, const int *band, const int *nband, const int *map,
                      ExtPlan *plan, int cap, int work, const unsigned char *const nostate[2],
                      cudaStream_t st, double *const wN[4] = nullptr,
                      double *const wP[4] = nullptr, double *sweep0 = nullptr, int copy = 0);
// f0 = 0, nf = 2: stencil states of both fluids; f0 = 2, nf = 1: level-set velocity
void launch_ext_sweeps(const Grid &g, double *const wN[4], double *const wP[4], double *ul0,
                       double *ul1, int f0, int nf, const ExtPlan *plan, int cap, int work,
                       const int *band, const int *nband, double *tmp, const double *alpha,
                       const unsigned char *const nostate[2], Scalars *sc, cudaStream_t st,
                       int first_done = 0);

// band_fluid >= 0: that fluid's states are recovered in the interaction
// band only (band, nband), unless band_flag is non-null and *band_flag != 0
void launch_prim2(const Grid &g, double *const qN[4], double *const qP[4], double *const wN[4],
                  double *const wP[4], const double *alpha, const int *tilesN,
                  const int *tilesP, int tile_cap, unsigned char *const nostate[2], Scalars *sc,
                  int band_fluid, const int *band_flag, const int *band, const int *nband,
                  cudaStream_t st, int skip_fluid = -1);
// viscous part of a finite-volume stage of fluid k (mu[k] > 0): dst +=
// b dt div(A Fv) over the cells of fluid k's active tiles
void launch_viscous(const Grid &g, int k, int s, int rk, double *const dst[4],
                    double *const w[4], const double *ax, const double *ay, const int *tiles,
                    int tile_cap, const double *dtp, Scalars *sc, cudaStream_t st);
// viscous stress with Stokes' hypothesis
__device__ inline void visc_stress(double mu, double ux, double uy, double vx, double vy,
                                   double &txx, double &txy, double &tyy) {
  txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy);
  tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux);
  txy = mu * (uy + vx);
}
void launch_interface(const Grid &g, double *const wN[4], double *const wP[4], const double *phi,
                      const double *sx, const double *sy, const int *cut, int cut_cap,
                      double *const xn[3], double *const xm[3], double *ul0, double *ul1,
                      Scalars *sc, cudaStream_t st);
void launch_ls_stage(const Grid &g, int s, int rk, double *phi, const double *phi0,
                     const double *ul0, const double *ul1, const int *band, const int *nband,
                     int band_cap, double *tmp, const double *dtp, cudaStream_t st);
void launch_reinit(const Grid &g, double *phi, double *phi0, const int *rext, const int *nrext,
                   int rext_cap, double *tmp, cudaStream_t st);
// Eq. 8-9 with the RK stage weight bw: shared (fluid 1 used the
// evaluation: -bw dt1 X_1) is 1 or 0, or decided on the device: -1 on the
// first sub-step, -2 on the last, -3 when the cycle has one sub-step;
// fluid2 (fluid 2 used it: +bw dt2 X_1)
void launch_record(const Grid &g, int shared, const int *cut, int cut_cap, double *const xn[3],
                   double *const xm[3], double *xc0, double *xc1, double *xc2, Scalars *sc,
                   cudaStream_t st, double bw = 0.5, int fluid2 = 1);
// a whole plane (ghosts included) copied when *flag is set
void launch_copy_if(const int *flag, const double *src, double *dst, size_t n, cudaStream_t st);
// phi = (1 - th) a + th b over the interior, a where a == b (th on the device)
void launch_phi_interp(const Grid &g, double *phi, const double *a, const double *b,
                       const double *thp, cudaStream_t st);
// zero the exchange flux planes of both fluids in the cells of the cut list
void launch_zero_cut(const Grid &g, double *const xn[3], double *const xm[3], const int *cut,
                     const int *ncut, int cut_cap, cudaStream_t st);
// Eq. 7 interpolation of fluid 1 at theta over the cells of a band list
void launch_interp(const Grid &g, double *const qi[4], double *const prev[4],
                   double *const fut[4], const double *thp, const int *band, const int *nband,
                   int band_cap, cudaStream_t st);
void launch_correction(const Grid &g, double *const q[4], const double *xc0, const double *xc1,
                       const double *xc2, cudaStream_t st);
void launch_init_state(const Grid &g, double *const qN[4], double *const qP[4],
                       double *const wN[4], double *const wP[4], const double *alpha,
                       cudaStream_t st);
void launch_integrals(const Grid &g, double *const qN[4], double *const qP[4], double *partial,
                      int nblk, double *out, cudaStream_t st);
void launch_sched(int op, Scalars *sc, double cfl, double thr, int force1, cudaStream_t st);

void fv_prepare();
bool fv_shape_supported(int tx, int ty);
void launch_fv_stage(const Grid &g, int k, int s, int rk, double *const dst[4],
                     double *const base[4], double *const cur[4], double *const w[4],
                     const double *ax, const double *ay, const double *sx, const double *sy,
                     const double *xn0, const double *xn1, const double *xn2, const int *tiles,
                     int tile_cap, int num_sms, const double *dtp, Scalars *sc,
                     cudaStream_t st);

// adjoint of the frozen single-time-step step (adjoint.cu, kernels_plan.cu)
void launch_adj_rhs(const Grid &g, double *const W[2][4], const unsigned long long *lf,
                    const double *dtp, double fac, double *const mu[2][4], const double *ax,
                    const double *ay, const double *phi, const double *sx, const double *sy,
                    const int *cut, const int *ncut, int cut_cap, double *const G[40],
                    double *const SP[8], double *const lw[2][4], cudaStream_t st);
void launch_adj_extension(const Grid &g, double *const lw[2][4], const ExtPlan *plan, int cap,
                          int work, const int *band, const int *nband, const int *map,
                          double *tmp, cudaStream_t st);
void launch_adj_prim(const Grid &g, double *const W[2][4], const double *alpha,
                     const unsigned char *const nostate[2], double *const lw[2][4],
                     double *const out[2][4], double *const A[2][4], double ca,
                     double *const B[2][4], double cb, cudaStream_t st);
void launch_adj_init(const Grid &g, double *const prim[2][4], const double *alpha,
                     double *const lam[2][4], double *const out[2][4], cudaStream_t st);
void launch_mix_adjoint(const Grid &g, double *const lN[4], double *const lP[4],
                        const double *alpha, const double *phi, const int *band, const int *map,
                        const int *nband, MixPlan *plan, int cap, int work, double *tmp,
                        cudaStream_t st);
unsigned long long sif_launches_adj();

// scheduler ops
#define SCHED_SINGLE_DT 0   // dt = min over fluids, capped by t_end
#define SCHED_CYCLE_BEGIN 1 // roles, ratio, truncation
#define SCHED_SUBSTEP 2     // fluid-2 dt from the latest interaction, last-substep test
#define SCHED_ADVANCE 3     // t2 += dt2 or finish the cycle
#define SCHED_FIRST_SUB 4   // last-substep test for the first sub-step
#define SCHED_RESET_MAX 5   // zero the CFL / LF maxima before an interaction step
#define SCHED_T_SINGLE 6    // t += dt
#define SCHED_T_CYCLE 7     // t += dt1
#define SCHED_DT2 8         // fluid-2 dt from the latest interaction
#define SCHED_LAST 9        // count the sub-step, last-substep test, theta
#define SCHED_THETA3 10     // theta of the RK3 third stage, (t2 + dt2/2) / dt1
#define SCHED_SNAPB 11      // keep the level set at the end of this sub-step?
#define SCHED_W3 12         // theta of fluid 1's third stage between the kept level sets

// conditions of the device-driven cycle graph (cudaGraphSetConditional)
#define COND_CYCLE 0        // h0 = single step, h1 = cycle with f1 = 0, h2 = cycle with f1 = 1
#define COND_NOT_FIRST 1    // h0 = sub-step after the first
#define COND_LAST 2         // h0 = last sub-step, h1 = not last
#define COND_LOOP 3         // h0 = keep sub-cycling
#define COND_SINGLE 4       // h0 = the cycle has a single sub-step, h1 = it has more
// the same tests setting h0 only: every op sets exactly the handles it
// names (a handle that was not created for this graph is never set)
#define COND_LAST_ONLY 5    // h0 = last sub-step
#define COND_SINGLE_ONLY 6  // h0 = a single sub-step
#define COND_MULTI_ONLY 7   // h0 = more than one sub-step
void launch_cond(int op, Scalars *sc, cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1,
                 cudaGraphConditionalHandle h2, int max_sub, cudaStream_t st);
