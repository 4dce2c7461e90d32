// sif3d_internal.cuh -- shared declarations of the three-dimensional
// solver's kernels (kernels3d.cu, fv3d.cu) and its host context (api3d.cu).
//
// Layout in HBM: every field is one padded plane of (nx+6)(ny+6)(nz+6)
// doubles, x fastest, three ghost layers per side (the WENO5 stencil's
// reach); (alpha U)_k and the stencil states W_k are five such planes per
// fluid.  The finite-volume stage works on bricks of 8 x 8 x 4 cells, one
// CTA per brick.
#pragma once

#include <cuda_runtime.h>

#define S3_GH 3
#define S3_NC 5
#define S3_BX 8
#define S3_BY 8
#define S3_BZ 4
#define S3_ALPHA_REAL 1e-6

struct Grid3 {
  int nx, ny, nz, PX, PY, PZ, NP;
  int bc[6];
  double dx, dy, dz, h, bw;  // bw: band half-width in length units
  double gamma[2], pinf[2];
  int tait[2];
  double tB[2], tr0[2], tp0[2];
  double eps, mix_alpha;
  double sigma;  // surface tension coefficient (Eq. 10), 0 = none
  double mu[2];  // dynamic viscosities (Eq. 3, 5), 0 = inviscid
  int newton_iters;  // limit of each interface Newton iteration
};

__host__ __device__ inline int g3(const Grid3 &g, int i, int j, int k) {
  return (i + S3_GH) + g.PX * ((j + S3_GH) + g.PY * (k + S3_GH));
}

// device-reduced quantities of an interaction step: the Lax-Friedrichs
// speeds per fluid and direction, the CFL rates, error bits, counters
// (maxima of non-negative doubles as ordered bit patterns)
struct Scal3 {
  unsigned long long lf[2][3];
  unsigned long long smax[2];
  int err;
  int nband;      // bricks in the band list
  int nfluid[2];  // bricks in each fluid's list (band and the fluid's cells)
  int pad;
  unsigned long long cells, open;  // finite-volume stage updates
  unsigned long long launches;
};

#define S3_ERR_NONPHYS 1
#define S3_ERR_NOCONV 2
#define S3_ERR_CAP 4  // a band list outgrew its capacity

// where a kernel works: the whole grid (list == nullptr; one thread per
// cell) or the cells of the listed bricks (count bricks of S3_BX x S3_BY x
// S3_BZ cells, 256 threads each).  The band list holds every brick with a
// cell within band + 3 cells of the interface, rebuilt after each
// interaction step: everything the next stage changes near the interface
// (level set, geometry, exchange fluxes, extension targets, small cells)
// lies in it, and outside it those fields keep their values.
struct Region {
  const int *list;
  int count;
};

__device__ inline bool region_cell(const Grid3 &g, const Region &R, long long t, int &i, int &j,
                                   int &k) {
  if (!R.list) {
    if (t >= (long long)g.nx * g.ny * g.nz) return false;
    int tt = (int)t;
    i = tt % g.nx;
    int r = tt / g.nx;
    j = r % g.ny;
    k = r / g.ny;
    return true;
  }
  long long b = t >> 8;
  if (b >= R.count) return false;
  int bi = R.list[b], l = (int)(t & 255);
  int nbx = (g.nx + S3_BX - 1) / S3_BX, nby = (g.ny + S3_BY - 1) / S3_BY;
  i = (bi % nbx) * S3_BX + l % S3_BX;
  j = ((bi / nbx) % nby) * S3_BY + (l / S3_BX) % S3_BY;
  k = (bi / (nbx * nby)) * S3_BZ + l / (S3_BX * S3_BY);
  return i < g.nx && j < g.ny && k < g.nz;
}

inline long long region_threads(const Grid3 &g, const Region &R) {
  return R.list ? (long long)R.count * 256 : (long long)g.nx * g.ny * g.nz;
}

// an extension target: its upwind neighbours (cells), their target slots
// (-1: not a target, value read from the plane) and weights; den = 0 marks
// a target with no upwind neighbour (it keeps its value)
struct Ext3 {
  int cell;
  int nb[3], slot[3];
  double w[3], den;
};

// a small-cell mixing source: its targets and the amounts moved from each
struct Mix3 {
  int cell;
  int nt;
  int tc[7];
  double M[7][S3_NC];
};

// a group of up to five planes for the ghost fill; vel[m] = d + 1 marks a
// velocity component odd at walls normal to d
struct Planes3 {
  double *p[8];
  int vel[8];
  int n;
};

// one TVD-RK2 stage of fluid k: dst = cur + dt L (stage 1) or
// dst = base / 2 + (cur + dt L) / 2 (stage 2), L the Eq. 2 right-hand side
// from the stencil states w.  A brick where no face is open to the fluid
// has L = 0: stage 1 leaves it as it is (dst must be cur or already hold
// it) and records in touched[brick] whether it changed the brick; stage 2
// applies the plain combination to closed bricks that stage 1 touched and
// leaves the others (there base = cur)
struct Fv3Args {
  unsigned char *touched;
  int k, stage;
  double dt;
  double lf[3];        // Lax-Friedrichs speeds of fluid k per direction
  const double *w[S3_NC];
  double *dst[S3_NC];
  const double *cur[S3_NC];
  const double *base[S3_NC];
  const double *ax, *ay, *az;
  const double *x[4];  // exchange flux as applied to fluid k
};

// host launch wrappers (each launch adds to the launch counter); R is the
// region a kernel works on
void k3_launch_ghost(const Grid3 &g, const Planes3 &s, cudaStream_t st);
void k3_launch_geometry(const Grid3 &g, const Region &R, const double *phi, double *corner,
                        double *alpha, double *ax, double *ay, double *az, double *sx,
                        double *sy, double *sz, cudaStream_t st);
void k3_launch_band_bricks(const Grid3 &g, int nbricks, const double *phi, const double *alpha,
                           int *list, int *fl0, int *fl1, Scal3 *sc, cudaStream_t st);
void k3_launch_init_state(const Grid3 &g, const double *alpha, const double *prim_dense,
                          double *const q[S3_NC], double *const w[S3_NC], int k,
                          cudaStream_t st);
void k3_launch_prim(const Grid3 &g, const Region &R, int k, double *const q[S3_NC],
                    double *const w[S3_NC], const double *alpha, unsigned char *nostate,
                    Scal3 *sc, cudaStream_t st);
int k3_ext_plan(const Grid3 &g, const Region &R, int group, const double *phi,
                const double *alpha, const unsigned char *nostate, const double *sx,
                const double *sy, const double *sz, int *map, Ext3 *plan, int *count, int cap,
                int *err, cudaStream_t st);
void k3_launch_ext_sweeps(const Grid3 &g, int group, int iters, const Ext3 *plan,
                          const int *count, int cap, double *const planes[], int nf,
                          double *bufA, double *bufB, int *map, cudaStream_t st);
void k3_launch_wave_maxima(const Grid3 &g, const Region &R, int k, double *const w[S3_NC],
                           const double *alpha, const unsigned char *nostate, const double *phi,
                           Scal3 *sc, cudaStream_t st);
void k3_launch_interface(const Grid3 &g, const Region &R, double *const w[2][S3_NC],
                         const double *phi, const double *sx, const double *sy,
                         const double *sz, double *const xn[4], double *const xp[4],
                         double *const ul[3], int *cutlist, int *cutcount, int cap, Scal3 *sc,
                         cudaStream_t st);
void k3_launch_mix(const Grid3 &g, const Region &R, int k, double *const q[S3_NC],
                   const double *alpha, const double *phi, int *srcmap, Mix3 *plan, int *count,
                   int cap, int *err, cudaStream_t st);
void k3_launch_band(const Grid3 &g, const double *phi, unsigned char *band,
                    unsigned char *rext, cudaStream_t st);
void k3_launch_ls_rhs(const Grid3 &g, const Region &R, const double *phi, double *const ul[3],
                      const unsigned char *band, double *lphi, cudaStream_t st);
void k3_launch_rk(const Grid3 &g, const Region &R, int stage, double *dst, const double *base,
                  const double *L, double dt, const unsigned char *mask, cudaStream_t st);
void k3_launch_reinit(const Grid3 &g, const Region &R, double *phi, const double *old,
                      const double *p0, const unsigned char *rext, cudaStream_t st);
void k3_launch_record(const Grid3 &g, const Region &R, int shared, double *const x1[4],
                      double *const xc[4], double dt1, double dt2, cudaStream_t st);
void k3_launch_interp(const Grid3 &g, const Region &R, double *const qi[S3_NC],
                      double *const prev[S3_NC], double *const fut[S3_NC], double th,
                      cudaStream_t st);
void k3_launch_correction(const Grid3 &g, double *const q[S3_NC], double *const xc[4],
                          double dv, cudaStream_t st);
void k3_launch_integrals(const Grid3 &g, double *const q[2][S3_NC], double *partial,
                         cudaStream_t st);
void k3_launch_pack(const Grid3 &g, const double *padded, double *dense, int unpack,
                    cudaStream_t st);
// small = 1 runs the stage on bricks of 4 x 4 x 4 cells (for a fluid on few
// bricks: many short CTAs instead of a few long ones); the touched flags
// are per brick of the shape used, which stage 1 and stage 2 must share
void k3_launch_fv(const Grid3 &g, const Fv3Args &a, Scal3 *sc, cudaStream_t st, int small);
int k3_fv_bricks(const Grid3 &g, int small);
// with viscosity: the aperture-weighted divergence of the viscous face
// fluxes of fluid k (Eq. 5), b dt times it added to the stage result dst
void k3_launch_viscous(const Grid3 &g, const Fv3Args &a, cudaStream_t st);
unsigned long long k3_launches();
