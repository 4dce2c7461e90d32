// fv3d.cu -- the three-dimensional cut-cell finite-volume stage (Eq. 2
// with six faces): one CTA per brick of 8 x 8 x 4 cells.
//
// The CTA first checks whether any face of its cells is open to the fluid;
// a closed brick has L = 0 and is left as it is.  Otherwise each face of
// the brick (the cells' lower faces and the brick's upper boundary faces:
// 9 x 8 x 4 + 8 x 9 x 4 + 8 x 8 x 5 = 896) is computed once: the stencil
// states of its six cells along the normal give the Lax-Friedrichs split
// fluxes f+- = (F_d +- a_d U)/2 (a_d the fluid's global speed, Sec. 4's
// WENO-LF), each conserved component is reconstructed by WENO5-JS from
// both sides, and the face value times the aperture A_k goes to shared
// memory (36 KB).  Each thread then forms its cell's divergence plus the
// interface exchange X / V and applies the RK stage in registers.
#include <atomic>

#include "sif3d_internal.cuh"

static std::atomic<unsigned long long> g_fv_launches{0};
unsigned long long k3_fv_launches() { return g_fv_launches.load(); }

#define NFX (S3_BX + 1) * S3_BY * S3_BZ
#define NFY S3_BX * (S3_BY + 1) * S3_BZ
#define NFZ S3_BX * S3_BY * (S3_BZ + 1)

__device__ inline double sqf(double a) { return a * a; }

__device__ inline double weno5_fv(double v1, double v2, double v3, double v4, double v5,
                                  double eps) {
  double q0 = (2.0 * v1 - 7.0 * v2 + 11.0 * v3) / 6.0;
  double q1 = (-v2 + 5.0 * v3 + 2.0 * v4) / 6.0;
  double q2 = (2.0 * v3 + 5.0 * v4 - v5) / 6.0;
  double b0 = 13.0 / 12.0 * sqf(v1 - 2.0 * v2 + v3) + 0.25 * sqf(v1 - 4.0 * v2 + 3.0 * v3);
  double b1 = 13.0 / 12.0 * sqf(v2 - 2.0 * v3 + v4) + 0.25 * sqf(v2 - v4);
  double b2 = 13.0 / 12.0 * sqf(v3 - 2.0 * v4 + v5) + 0.25 * sqf(3.0 * v3 - 4.0 * v4 + v5);
  double a0 = 0.1 / sqf(eps + b0);
  double a1 = 0.6 / sqf(eps + b1);
  double a2 = 0.3 / sqf(eps + b2);
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// WENO5-LF flux of every component at the lower d-face of cell c
__device__ inline void face_flux3(const Grid3 &g, const Fv3Args &a, int c, int s, int d,
                                  double *Fh) {
  const double gm = g.gamma[a.k], pi = g.pinf[a.k], ad = a.lf[d];
  double U[6][S3_NC], F[6][S3_NC];
#pragma unroll
  for (int r = 0; r < 6; r++) {
    int cc = c + (r - 3) * s;
    double rho = a.w[0][cc], u = a.w[1][cc], v = a.w[2][cc], w = a.w[3][cc], p = a.w[4][cc];
    double E = (p + gm * pi) / (gm - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
    double un = d == 0 ? u : d == 1 ? v : w;
    U[r][0] = rho;
    U[r][1] = rho * u;
    U[r][2] = rho * v;
    U[r][3] = rho * w;
    U[r][4] = E;
    F[r][0] = rho * un;
    F[r][1] = rho * u * un + (d == 0 ? p : 0.0);
    F[r][2] = rho * v * un + (d == 1 ? p : 0.0);
    F[r][3] = rho * w * un + (d == 2 ? p : 0.0);
    F[r][4] = un * (E + p);
  }
#pragma unroll
  for (int m = 0; m < S3_NC; m++) {
    double fp[6], fm[6];
#pragma unroll
    for (int r = 0; r < 6; r++) {
      fp[r] = 0.5 * (F[r][m] + ad * U[r][m]);
      fm[r] = 0.5 * (F[r][m] - ad * U[r][m]);
    }
    Fh[m] = weno5_fv(fp[0], fp[1], fp[2], fp[3], fp[4], g.eps) +
            weno5_fv(fm[5], fm[4], fm[3], fm[2], fm[1], g.eps);
  }
}

__device__ inline double ap3(const double *A, int k, int c) {
  return k == 1 ? A[c] : 1.0 - A[c];
}

__global__ void __launch_bounds__(256) k3_fv(Grid3 g, Fv3Args a, Scal3 *sc) {
  __shared__ double fx[S3_NC][NFX];
  __shared__ double fy[S3_NC][NFY];
  __shared__ double fz[S3_NC][NFZ];
  const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
  const int tid = threadIdx.x;
  const int li = tid % S3_BX, lj = (tid / S3_BX) % S3_BY, lk = tid / (S3_BX * S3_BY);
  const int i = bx * S3_BX + li, j = by * S3_BY + lj, kk = bz * S3_BZ + lk;
  const bool valid = i < g.nx && j < g.ny && kk < g.nz;
  const int k = a.k, sx = 1, sy = g.PX, sz = g.PX * g.PY;
  int c = valid ? g3(g, i, j, kk) : 0;
  int open = 0;
  if (valid)
    open = ap3(a.ax, k, c) != 0.0 || ap3(a.ax, k, c + sx) != 0.0 || ap3(a.ay, k, c) != 0.0 ||
           ap3(a.ay, k, c + sy) != 0.0 || ap3(a.az, k, c) != 0.0 || ap3(a.az, k, c + sz) != 0.0;
  int nopen = __syncthreads_count(open);
  const int brick = bx + gridDim.x * (by + gridDim.y * bz);
  if (nopen == 0) {
    if (a.stage == 1) {
      if (tid == 0) a.touched[brick] = 0;
      return;
    }
    if (!a.touched[brick] || !valid) return;
    for (int m = 0; m < S3_NC; m++)
      a.dst[m][c] = 0.5 * a.base[m][c] + 0.5 * (a.cur[m][c] + a.dt * 0.0);
    return;
  }
  if (tid == 0 && a.stage == 1) a.touched[brick] = 1;
  if (tid == 0) {
    int ncell = min(S3_BX, g.nx - bx * S3_BX) * min(S3_BY, g.ny - by * S3_BY) *
                min(S3_BZ, g.nz - bz * S3_BZ);
    atomicAdd(&sc->cells, (unsigned long long)ncell);
    atomicAdd(&sc->open, (unsigned long long)nopen);
  }
  // faces: x-faces (ii in 0..8) then y-faces (jj in 0..8) then z-faces
  for (int f = tid; f < NFX + NFY + NFZ; f += blockDim.x) {
    int d, fi, fj, fk, slot;
    if (f < NFX) {
      d = 0;
      slot = f;
      fi = f % (S3_BX + 1);
      fj = (f / (S3_BX + 1)) % S3_BY;
      fk = f / ((S3_BX + 1) * S3_BY);
    } else if (f < NFX + NFY) {
      d = 1;
      slot = f - NFX;
      fi = slot % S3_BX;
      fj = (slot / S3_BX) % (S3_BY + 1);
      fk = slot / (S3_BX * (S3_BY + 1));
    } else {
      d = 2;
      slot = f - NFX - NFY;
      fi = slot % S3_BX;
      fj = (slot / S3_BX) % S3_BY;
      fk = slot / (S3_BX * S3_BY);
    }
    int gi = bx * S3_BX + fi, gj = by * S3_BY + fj, gk = bz * S3_BZ + fk;
    // a face belongs to the domain if its cell (the one above it) is
    // inside along the other two axes and at most n along its own
    bool ok = d == 0 ? (gi <= g.nx && gj < g.ny && gk < g.nz)
                     : d == 1 ? (gi < g.nx && gj <= g.ny && gk < g.nz)
                              : (gi < g.nx && gj < g.ny && gk <= g.nz);
    double Fh[S3_NC] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (ok) {
      int cf = g3(g, gi, gj, gk);
      const double *A = d == 0 ? a.ax : d == 1 ? a.ay : a.az;
      double Ak = ap3(A, k, cf);
      if (Ak != 0.0) {
        face_flux3(g, a, cf, d == 0 ? sx : d == 1 ? sy : sz, d, Fh);
        for (int m = 0; m < S3_NC; m++) Fh[m] = Ak * Fh[m];
      }
    }
    double *dst = d == 0 ? &fx[0][0] : d == 1 ? &fy[0][0] : &fz[0][0];
    int stride = d == 0 ? NFX : d == 1 ? NFY : NFZ;
    for (int m = 0; m < S3_NC; m++) dst[m * stride + slot] = Fh[m];
  }
  __syncthreads();
  if (!valid) return;
  const int ix = li + (S3_BX + 1) * (lj + S3_BY * lk);
  const int iy = li + S3_BX * (lj + (S3_BY + 1) * lk);
  const int iz = li + S3_BX * (lj + S3_BY * lk);
  const double dv = g.dx * g.dy * g.dz;
  for (int m = 0; m < S3_NC; m++) {
    double r = 0.0;
    r += (fx[m][ix] - fx[m][ix + 1]) / g.dx;
    r += (fy[m][iy] - fy[m][iy + S3_BX]) / g.dy;
    r += (fz[m][iz] - fz[m][iz + S3_BX * S3_BY]) / g.dz;
    if (m > 0) r += a.x[m - 1][c] / dv;
    double cur = a.cur[m][c];
    double v = a.stage == 1 ? cur + a.dt * r : 0.5 * a.base[m][c] + 0.5 * (cur + a.dt * r);
    a.dst[m][c] = v;
  }
}

void k3_launch_fv(const Grid3 &g, const Fv3Args &a, Scal3 *sc, cudaStream_t st) {
  dim3 grid((g.nx + S3_BX - 1) / S3_BX, (g.ny + S3_BY - 1) / S3_BY, (g.nz + S3_BZ - 1) / S3_BZ);
  k3_fv<<<grid, S3_BX * S3_BY * S3_BZ, 0, st>>>(g, a, sc);
  g_fv_launches++;
}
