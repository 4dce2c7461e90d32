// kernels_fv.cu -- the cut-cell finite-volume stage of one fluid (Eq. 2):
// WENO5-JS reconstruction of the Lax-Friedrichs split fluxes on every open
// face, face fluxes weighted by the fluid's apertures, the interface
// exchange flux X in cut cells and the Runge-Kutta stage combination.
//
// One CTA owns a FV_TX x FV_TY tile of output cells.  The split fluxes of
// the tile and its 3-cell halo are built once in shared memory, every
// face flux is reconstructed once per CTA, and the update is written in
// place (a cell reads only its own conserved values).  Only the tiles in
// which the fluid can have an open face are launched.  FP64 throughout;
// the reconstruction uses one division per face and component.
#include "sif_internal.cuh"

#define HX (FV_TX + 6)
#define HY (FV_TY + 6)

struct FvArgs {
  Grid g;
  int k, s;
  double a, b;           // RK stage weights
  double *dst[4];
  const double *base[4];
  const double *cur[4];
  const double *w[4];
  const double *ax, *ay, *sx, *sy;
  const double *xn[3];
  const int *tiles;
  const int *ntiles;
  const double *dtp;
  double lfx_dummy;
  const Scalars *sc;
};

__device__ __forceinline__ double weno5_fast(double v1, double v2, double v3, double v4, double v5,
                                             double eps) {
  const double c13_12 = 13.0 / 12.0, s6 = 1.0 / 6.0;
  double d0 = (v1 + v3) - 2.0 * v2;
  double e0 = (v1 + 3.0 * v3) - 4.0 * v2;
  double d1 = (v2 + v4) - 2.0 * v3;
  double e1 = v2 - v4;
  double d2 = (v3 + v5) - 2.0 * v4;
  double e2 = (3.0 * v3 + v5) - 4.0 * v4;
  double b0 = c13_12 * d0 * d0 + 0.25 * e0 * e0;
  double b1 = c13_12 * d1 * d1 + 0.25 * e1 * e1;
  double b2 = c13_12 * d2 * d2 + 0.25 * e2 * e2;
  double q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) * s6;
  double q1 = (-v2 + 5.0 * v3 + 2.0 * v4) * s6;
  double q2 = (2.0 * v3 + 5.0 * v4 - v5) * s6;
  double t0 = eps + b0, t1 = eps + b1, t2 = eps + b2;
  t0 *= t0;
  t1 *= t1;
  t2 *= t2;
  // weights d_r / t_r normalised with a single division
  double w0 = 0.1 * (t1 * t2), w1 = 0.6 * (t0 * t2), w2 = 0.3 * (t0 * t1);
  return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// end-of-block bookkeeping of the launch timer: the last block of the
// launch adds the launch span and re-arms the timer for the next launch
__device__ void fv_timer_block_done(const Scalars *csc, bool worked) {
  Scalars *sc = (Scalars *)csc;
  if (worked) atomicMax((unsigned long long *)&sc->fv_t1, globaltimer_ns());
  __threadfence();
  unsigned int done = atomicAdd(&sc->fv_blocks_done, 1u);
  if (done == gridDim.x - 1) {
    __threadfence();
    unsigned long long t0 = atomicAdd((unsigned long long *)&sc->fv_t0, 0ull);
    unsigned long long t1 = atomicAdd((unsigned long long *)&sc->fv_t1, 0ull);
    if (t1 > t0 && t0 != ~0ull) atomicAdd((unsigned long long *)&sc->fv_ns, t1 - t0);
    atomicAdd((unsigned long long *)&sc->fv_launches, 1ull);
    atomicExch((unsigned long long *)&sc->fv_t0, ~0ull);
    atomicExch((unsigned long long *)&sc->fv_t1, 0ull);
    atomicExch(&sc->fv_blocks_done, 0u);
  }
}

__device__ __forceinline__ void fv_update_cell(const FvArgs &A, int k, int i, int j, int li, int lj,
                                               const double *Fx, const double *Fy, bool d2);

__global__ void __launch_bounds__(FV_TX *FV_TY) k_fv_stage(FvArgs A) {
  SIF_TICK();
  const Grid &g = A.g;
  const int k = A.k;
  if ((int)blockIdx.x >= A.ntiles[k]) {
    if (A.sc->timing && threadIdx.x == 0) fv_timer_block_done(A.sc, false);
    return;
  }
  extern __shared__ double smem[];
  // split fluxes: x for rows of the tile with x-halo, y for columns with y-halo
  double *fxp = smem;                       // [4][HX*FV_TY]
  double *fxm = fxp + 4 * HX * FV_TY;       // [4][HX*FV_TY]
  double *fyp = fxm + 4 * HX * FV_TY;       // [4][FV_TX*HY]
  double *fym = fyp + 4 * FV_TX * HY;       // [4][FV_TX*HY]
  double *Fx = fym + 4 * FV_TX * HY;        // [4][(FV_TX+1)*FV_TY]
  double *Fy = Fx + 4 * (FV_TX + 1) * FV_TY;  // [4][FV_TX*(FV_TY+1)]

  int tile = A.tiles[blockIdx.x];
  int i0 = (tile % g.ntx) * FV_TX, j0 = (tile / g.ntx) * FV_TY;
  if (threadIdx.x == 0) {
    int w_ = min(FV_TX, g.nx - i0), h_ = min(FV_TY, g.ny - j0);
    atomicAdd((unsigned long long *)&A.sc->updates, (unsigned long long)(w_ * h_));
  }
  const bool timed = A.sc->timing;
  if (timed && threadIdx.x == 0) atomicMin((unsigned long long *)&A.sc->fv_t0, globaltimer_ns());
  const double gm = g.gamma[k], pi = g.pinf[k];
  const double inv_gm1 = 1.0 / (gm - 1.0), e0c = gm * pi * inv_gm1;
  const double lfx = ull_as_double(A.sc->lf[k][0]), lfy = ull_as_double(A.sc->lf[k][1]);
  const bool d2 = g.dim == 2;
  const int tid = threadIdx.x, nth = blockDim.x;

  // phase 1: Lax-Friedrichs split fluxes of the stencil states
  for (int r = tid; r < HX * FV_TY; r += nth) {
    int i = i0 - 3 + r % HX, j = j0 + r / HX;
    double fp[4] = {0, 0, 0, 0}, fm[4] = {0, 0, 0, 0};
    if (i <= g.nx + 2 && j < g.ny) {
      int c = gidx(g, i, j);
      double rho = A.w[0][c], u = A.w[1][c], v = A.w[2][c], p = A.w[3][c];
      double E = p * inv_gm1 + e0c + 0.5 * rho * (u * u + v * v);
      double mu = rho * u;
      double F[4] = {mu, mu * u + p, mu * v, u * (E + p)};
      double U[4] = {rho, mu, rho * v, E};
#pragma unroll
      for (int m = 0; m < 4; m++) {
        fp[m] = 0.5 * (F[m] + lfx * U[m]);
        fm[m] = 0.5 * (F[m] - lfx * U[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; m++) {
      fxp[m * HX * FV_TY + r] = fp[m];
      fxm[m * HX * FV_TY + r] = fm[m];
    }
  }
  if (d2) {
    for (int r = tid; r < FV_TX * HY; r += nth) {
      int i = i0 + r % FV_TX, j = j0 - 3 + r / FV_TX;
      double fp[4] = {0, 0, 0, 0}, fm[4] = {0, 0, 0, 0};
      if (i < g.nx && j <= g.ny + 2) {
        int c = gidx(g, i, j);
        double rho = A.w[0][c], u = A.w[1][c], v = A.w[2][c], p = A.w[3][c];
        double E = p * inv_gm1 + e0c + 0.5 * rho * (u * u + v * v);
        double mv = rho * v;
        double F[4] = {mv, mv * u, mv * v + p, v * (E + p)};
        double U[4] = {rho, rho * u, mv, E};
#pragma unroll
        for (int m = 0; m < 4; m++) {
          fp[m] = 0.5 * (F[m] + lfy * U[m]);
          fm[m] = 0.5 * (F[m] - lfy * U[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; m++) {
        fyp[m * FV_TX * HY + r] = fp[m];
        fym[m * FV_TX * HY + r] = fm[m];
      }
    }
  }
  __syncthreads();

  // phase 2: x faces (left face of cell i0 + fi), one (face, component) per item
  const double eps = g.weno_eps;
  for (int r = tid; r < 4 * (FV_TX + 1) * FV_TY; r += nth) {
    int m = r / ((FV_TX + 1) * FV_TY), f = r % ((FV_TX + 1) * FV_TY);
    int fi = f % (FV_TX + 1), fj = f / (FV_TX + 1);
    int i = i0 + fi, j = j0 + fj;
    double val = 0.0;
    if (i <= g.nx && j < g.ny) {
      double A_ = A.ax[gidx(g, i, j)];
      if (k == 0) A_ = 1.0 - A_;
      if (A_ != 0.0) {
        // cells i-3..i+2 are at halo columns fi..fi+5
        const double *P = fxp + m * HX * FV_TY + fj * HX + fi;
        const double *M = fxm + m * HX * FV_TY + fj * HX + fi;
        double fl = weno5_fast(P[0], P[1], P[2], P[3], P[4], eps);
        double fr = weno5_fast(M[5], M[4], M[3], M[2], M[1], eps);
        val = A_ * (fl + fr);
      }
    }
    Fx[m * (FV_TX + 1) * FV_TY + f] = val;
  }
  if (d2) {
    for (int r = tid; r < 4 * FV_TX * (FV_TY + 1); r += nth) {
      int m = r / (FV_TX * (FV_TY + 1)), f = r % (FV_TX * (FV_TY + 1));
      int fi = f % FV_TX, fj = f / FV_TX;
      int i = i0 + fi, j = j0 + fj;
      double val = 0.0;
      if (i < g.nx && j <= g.ny) {
        double A_ = A.ay[gidx(g, i, j)];
        if (k == 0) A_ = 1.0 - A_;
        if (A_ != 0.0) {
          const double *P = fyp + m * FV_TX * HY + fj * FV_TX + fi;
          const double *M = fym + m * FV_TX * HY + fj * FV_TX + fi;
          double fl = weno5_fast(P[0], P[FV_TX], P[2 * FV_TX], P[3 * FV_TX], P[4 * FV_TX], eps);
          double fr = weno5_fast(M[5 * FV_TX], M[4 * FV_TX], M[3 * FV_TX], M[2 * FV_TX],
                                 M[FV_TX], eps);
          val = A_ * (fl + fr);
        }
      }
      Fy[m * FV_TX * (FV_TY + 1) + f] = val;
    }
  }
  __syncthreads();

  // phase 3: update of the tile's cells
  int li = tid % FV_TX, lj = tid / FV_TX;
  int i = i0 + li, j = j0 + lj;
  if (i < g.nx && j < g.ny) fv_update_cell(A, k, i, j, li, lj, Fx, Fy, d2);
  if (timed) {
    __syncthreads();
    if (threadIdx.x == 0) fv_timer_block_done(A.sc, true);
  }
}

__device__ __forceinline__ void fv_update_cell(const FvArgs &A, int k, int i, int j, int li, int lj,
                                               const double *Fx, const double *Fy, bool d2) {
  const Grid &g = A.g;
  int c = gidx(g, i, j);
  double dt = *A.dtp;
  double inv_dx = 1.0 / g.dx, inv_dy = 1.0 / g.dy, inv_dxdy = 1.0 / (g.dx * g.dy);
  bool cut = (A.sx[c] != 0.0 || A.sy[c] != 0.0);
  double sgn = k == 0 ? 1.0 : -1.0;
#pragma unroll
  for (int m = 0; m < 4; m++) {
    const double *fx = Fx + m * (FV_TX + 1) * FV_TY + lj * (FV_TX + 1) + li;
    double L = (fx[0] - fx[1]) * inv_dx;
    if (d2) {
      const double *fy = Fy + m * FV_TX * (FV_TY + 1) + lj * FV_TX + li;
      L += (fy[0] - fy[FV_TX]) * inv_dy;
    }
    if (m > 0 && cut) L += sgn * A.xn[m - 1][c] * inv_dxdy;
    double cur = A.cur[m][c];
    double out = A.s == 1 ? cur + dt * L : A.a * A.base[m][c] + A.b * (cur + dt * L);
    A.dst[m][c] = out;
  }
}

static size_t fv_smem_bytes();

// opt the finite-volume kernel into its shared-memory size on the current
// device (outside any stream capture)
void fv_prepare() {
  cudaFuncSetAttribute(k_fv_stage, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fv_smem_bytes());
}

static size_t fv_smem_bytes() {
  return sizeof(double) * (size_t)(8 * HX * FV_TY + 8 * FV_TX * HY + 4 * (FV_TX + 1) * FV_TY +
                                   4 * FV_TX * (FV_TY + 1));
}

void launch_fv_stage(const Grid &g, int k, int s, int rk, double *const dst[4],
                     double *const base[4], double *const cur[4], double *const w[4],
                     const double *ax, const double *ay, const double *sx, const double *sy,
                     const double *xn0, const double *xn1, const double *xn2, const int *tiles,
                     int tile_cap, const double *dtp, Scalars *sc, cudaStream_t st) {
  static const double A2[3] = {0.0, 0.0, 0.5}, B2[3] = {0.0, 1.0, 0.5};
  static const double A3[4] = {0.0, 0.0, 0.75, 1.0 / 3.0}, B3[4] = {0.0, 1.0, 0.25, 2.0 / 3.0};
  size_t smem = fv_smem_bytes();
  FvArgs A;
  A.g = g;
  A.k = k;
  A.s = s;
  A.a = rk == 3 ? A3[s] : A2[s];
  A.b = rk == 3 ? B3[s] : B2[s];
  for (int m = 0; m < 4; m++) {
    A.dst[m] = dst[m];
    A.base[m] = base[m];
    A.cur[m] = cur[m];
    A.w[m] = w[m];
  }
  A.ax = ax;
  A.ay = ay;
  A.sx = sx;
  A.sy = sy;
  A.xn[0] = xn0;
  A.xn[1] = xn1;
  A.xn[2] = xn2;
  A.tiles = tiles;
  A.ntiles = sc->n_tiles;
  A.dtp = dtp;
  A.lfx_dummy = 0.0;
  A.sc = sc;
  k_fv_stage<<<tile_cap, FV_TX * FV_TY, smem, st>>>(A);
  sif_note_launches(1);
}

SIF_TU_LAUNCH_READER(fv)
