// fv3d.cu -- the three-dimensional cut-cell finite-volume stage (Eq. 2
// with six faces): one CTA of 256 threads per brick of 8 x 8 x 4 cells,
// one thread per cell.
//
// The CTA first checks whether any face of its cells is open to the fluid;
// a closed brick has L = 0 (see Fv3Args for what the RK stage then does).
// Otherwise the three directions are taken in turn, each in three phases
// separated by barriers: (1) the Lax-Friedrichs split fluxes f+- = (F_d +-
// a_d U)/2 (a_d the fluid's global speed, Sec. 4's WENO-LF) of every cell
// of the brick and of the three cells beyond it on either side along d go
// to shared memory, each computed once; (2) each (face, component) of the
// brick's faces along d -- its cells' lower faces and the brick's upper
// boundary -- is reconstructed by WENO5-JS from both sides and multiplied
// by the aperture A_k (the two reconstructions as fractions over one
// reciprocal, weno_frac.cuh), into shared memory; (3) each thread adds its
// cell's difference of the two faces times 1/h_d to its right-hand side in
// registers.  The interface exchange X / V and the RK stage follow in
// registers.  Two shapes are instantiated: 8 x 8 x 4 (256 threads, 64 KB of
// shared memory, three CTAs per SM) and 4 x 4 x 4 (64 threads, 16 KB) for a
// fluid on few bricks, whose launch lasts about one CTA lifetime.
#include <atomic>

#include "sif3d_internal.cuh"
#include "weno_frac.cuh"

static std::atomic<unsigned long long> g_fv_launches{0};
unsigned long long k3_fv_launches() { return g_fv_launches.load(); }

__device__ inline double ap3(const double *A, int k, int c) {
  return k == 1 ? A[c] : 1.0 - A[c];
}

// a brick shape of the stage: BX x BY x BZ cells, one thread each.
// Extents of the direction-d pass: the brick plus three cells on either
// side along d (the split fluxes a face's stencil reads), and its faces
template <int BX, int BY, int BZ>
struct FvBrick {
  static constexpr int threads = BX * BY * BZ;
  __host__ __device__ static constexpr int len(int d) { return d == 0 ? BX : d == 1 ? BY : BZ; }
  __host__ __device__ static constexpr int reg(int d) { return len(d) + 6; }
  static constexpr int reg_max = (BZ + 6) * BX * BY > (BX + 6) * BY * BZ
                                     ? ((BZ + 6) * BX * BY > (BY + 6) * BX * BZ
                                            ? (BZ + 6) * BX * BY
                                            : (BY + 6) * BX * BZ)
                                     : ((BX + 6) * BY * BZ > (BY + 6) * BX * BZ
                                            ? (BX + 6) * BY * BZ
                                            : (BY + 6) * BX * BZ);
  static constexpr int face_max = BX * BY * BZ + (BX * BY > BY * BZ
                                                      ? (BX * BY > BX * BZ ? BX * BY : BX * BZ)
                                                      : (BY * BZ > BX * BZ ? BY * BZ : BX * BZ));
  static constexpr size_t smem = sizeof(double) * S3_NC * (2 * reg_max + face_max);
};

template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k3_fv(Grid3 g, Fv3Args a, Scal3 *sc) {
  using B = FvBrick<BX, BY, BZ>;
  constexpr int S3_REG_MAX = B::reg_max, S3_FACE_MAX = B::face_max;
  extern __shared__ double smem[];
  double *sp = smem;                              // f+ [m][cell of the pass]
  double *sm = sp + S3_NC * S3_REG_MAX;           // f- [m][cell of the pass]
  double *sf = sm + S3_NC * S3_REG_MAX;           // A_k F [m][face of the pass]
  const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
  const int tid = threadIdx.x;
  const int li = tid % BX, lj = (tid / BX) % BY, lk = tid / (BX * BY);
  const int i = bx * BX + li, j = by * BY + lj, kk = bz * BZ + lk;
  const bool valid = i < g.nx && j < g.ny && kk < g.nz;
  const int k = a.k;
  const int st[3] = {1, g.PX, g.PX * g.PY};
  const int nn[3] = {g.nx, g.ny, g.nz};
  const int b0[3] = {bx * BX, by * BY, bz * BZ};
  const double *Ad[3] = {a.ax, a.ay, a.az};
  // reciprocals of the cell sizes and volume, one division each per thread
  const double ih[3] = {1.0 / g.dx, 1.0 / g.dy, 1.0 / g.dz};
  int c = valid ? g3(g, i, j, kk) : 0;
  int open = 0;
  if (valid)
    for (int d = 0; d < 3; d++)
      open |= ap3(Ad[d], k, c) != 0.0 || ap3(Ad[d], k, c + st[d]) != 0.0;
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
  if (tid == 0) {
    if (a.stage == 1) a.touched[brick] = 1;
    int ncell = min(BX, g.nx - b0[0]) * min(BY, g.ny - b0[1]) * min(BZ, g.nz - b0[2]);
    atomicAdd(&sc->cells, (unsigned long long)ncell);
    atomicAdd(&sc->open, (unsigned long long)nopen);
  }
  const double gm = g.gamma[k], pi = g.pinf[k];
  const double eps = g.eps * (12.0 / 13.0);  // see weno5_frac
  double r[S3_NC] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    // pass layout: position along d fastest, then the two other axes in
    // (x, y, z) order
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
    const int L = B::reg(d), n1 = B::len(e1), n2 = B::len(e2);
    const int ncells = L * n1 * n2, nfaces = (B::len(d) + 1) * n1 * n2;
    const double ad = a.lf[d];
    // split fluxes of every cell of the pass
    for (int t = tid; t < ncells; t += blockDim.x) {
      int p = t % L, q1 = (t / L) % n1, q2 = t / (L * n1);
      int x[3];
      x[d] = b0[d] - 3 + p;
      x[e1] = b0[e1] + q1;
      x[e2] = b0[e2] + q2;
      bool in = x[d] >= -3 && x[d] < nn[d] + 3 && x[e1] < nn[e1] && x[e2] < nn[e2];
      double fp[S3_NC] = {0.0, 0.0, 0.0, 0.0, 0.0}, fm[S3_NC] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (in) {
        int cc = g3(g, x[0], x[1], x[2]);
        double rho = a.w[0][cc], u = a.w[1][cc], v = a.w[2][cc], w = a.w[3][cc];
        double pr = a.w[4][cc];
        double E = (pr + gm * pi) / (gm - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
        double un = d == 0 ? u : d == 1 ? v : w;
        double U[S3_NC] = {rho, rho * u, rho * v, rho * w, E};
        double F[S3_NC] = {rho * un, rho * u * un + (d == 0 ? pr : 0.0),
                           rho * v * un + (d == 1 ? pr : 0.0),
                           rho * w * un + (d == 2 ? pr : 0.0), un * (E + pr)};
#pragma unroll
        for (int m = 0; m < S3_NC; m++) {
          fp[m] = 0.5 * (F[m] + ad * U[m]);
          fm[m] = 0.5 * (F[m] - ad * U[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < S3_NC; m++) {
        sp[m * S3_REG_MAX + t] = fp[m];
        sm[m * S3_REG_MAX + t] = fm[m];
      }
    }
    __syncthreads();
    // (face, component) items: WENO5 from both sides times the aperture
    for (int t = tid; t < nfaces * S3_NC; t += blockDim.x) {
      int f = t % nfaces, m = t / nfaces;
      int p = f % (B::len(d) + 1), q = f / (B::len(d) + 1);
      int q1 = q % n1, q2 = q / n1;
      int x[3];
      x[d] = b0[d] + p;
      x[e1] = b0[e1] + q1;
      x[e2] = b0[e2] + q2;
      double Fh = 0.0;
      if (x[d] <= nn[d] && x[e1] < nn[e1] && x[e2] < nn[e2]) {
        double Ak = ap3(Ad[d], k, g3(g, x[0], x[1], x[2]));
        if (Ak != 0.0) {
          // the face between pass cells p + 2 and p + 3
          const double *P = sp + m * S3_REG_MAX + q * L + p;
          const double *M = sm + m * S3_REG_MAX + q * L + p;
          double nl, dl, nr, dr;
          weno5_frac(P[0], P[1], P[2], P[3], P[4], eps, nl, dl);
          weno5_frac(M[5], M[4], M[3], M[2], M[1], eps, nr, dr);
          Fh = face_value(Ak, nl, dl, nr, dr);
        }
      }
      sf[m * S3_FACE_MAX + f] = Fh;
    }
    __syncthreads();
    if (valid) {
      int x[3] = {li, lj, lk};
      int lo = x[d] + (B::len(d) + 1) * (x[e1] + n1 * x[e2]);
#pragma unroll
      for (int m = 0; m < S3_NC; m++)
        r[m] += (sf[m * S3_FACE_MAX + lo] - sf[m * S3_FACE_MAX + lo + 1]) * ih[d];
    }
    __syncthreads();
  }
  if (!valid) return;
  const double idv = 1.0 / (g.dx * g.dy * g.dz);
#pragma unroll
  for (int m = 0; m < S3_NC; m++) {
    double rr = r[m];
    if (m > 0) rr += a.x[m - 1][c] * idv;
    double cur = a.cur[m][c];
    a.dst[m][c] = a.stage == 1 ? cur + a.dt * rr : 0.5 * a.base[m][c] + 0.5 * (cur + a.dt * rr);
  }
}

// ---------------------------------------------------------------------
// viscous face fluxes (Eq. 3, 5): through the lower d-face of cell cf
// (between cf - s and cf) from the stencil states by central differences,
// the normal derivatives across the face and the tangential ones as the
// mean of the two cells' central differences; Stokes' stress

__device__ inline void viscous_face3(const Grid3 &g, const Fv3Args &a, int cf, int d,
                                     double mu, double Fv[4]) {
  const int st[3] = {1, g.PX, g.PX * g.PY};
  const double hd[3] = {g.dx, g.dy, g.dz};
  const int cl = cf - st[d];
  double G[3][3];
#pragma unroll
  for (int b = 0; b < 3; b++) {
    const double *u = a.w[1 + b];
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == d)
        G[e][b] = (u[cf] - u[cl]) / hd[e];
      else
        G[e][b] = ((u[cf + st[e]] - u[cf - st[e]]) + (u[cl + st[e]] - u[cl - st[e]])) /
                  (4.0 * hd[e]);
    }
  }
  // the row d of the stress tensor
  double t[3];
#pragma unroll
  for (int b = 0; b < 3; b++) {
    // the other two diagonal terms in axis order, as in the stress tensor
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    if (b == d)
      t[b] = mu * (4.0 / 3.0 * G[d][d] - 2.0 / 3.0 * G[o1][o1] - 2.0 / 3.0 * G[o2][o2]);
    else
      t[b] = mu * (G[b][d] + G[d][b]);
  }
  double e = 0.0;
#pragma unroll
  for (int b = 0; b < 3; b++) {
    Fv[b] = t[b];
    e += 0.5 * (a.w[1 + b][cl] + a.w[1 + b][cf]) * t[b];
  }
  Fv[3] = e;
}

// one thread per cell of a brick with a face open to the fluid: the
// viscous part of Eq. 2, -sum_d (A Fv)_lower - (A Fv)_upper over h_d, b dt
// times it added to the stage result (b = 1 at stage 1, 1/2 at stage 2)
__global__ void __launch_bounds__(256) k3_viscous(Grid3 g, Fv3Args a) {
  const int tid = threadIdx.x;
  const int li = tid % S3_BX, lj = (tid / S3_BX) % S3_BY, lk = tid / (S3_BX * S3_BY);
  const int i = blockIdx.x * S3_BX + li, j = blockIdx.y * S3_BY + lj,
            kk = blockIdx.z * S3_BZ + lk;
  const bool valid = i < g.nx && j < g.ny && kk < g.nz;
  const int k = a.k, st[3] = {1, g.PX, g.PX * g.PY};
  const double *Ad[3] = {a.ax, a.ay, a.az};
  const double hd[3] = {g.dx, g.dy, g.dz};
  int c = valid ? g3(g, i, j, kk) : 0;
  int open = 0;
  if (valid)
    for (int d = 0; d < 3; d++)
      open |= ap3(Ad[d], k, c) != 0.0 || ap3(Ad[d], k, c + st[d]) != 0.0;
  if (!__syncthreads_or(open) || !valid) return;
  const double mu = g.mu[k];
  double r[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double lo[4] = {0.0, 0.0, 0.0, 0.0}, hi[4] = {0.0, 0.0, 0.0, 0.0};
    double Al = ap3(Ad[d], k, c), Ah = ap3(Ad[d], k, c + st[d]);
    if (Al != 0.0) {
      viscous_face3(g, a, c, d, mu, lo);
      for (int m = 0; m < 4; m++) lo[m] = Al * lo[m];
    }
    if (Ah != 0.0) {
      viscous_face3(g, a, c + st[d], d, mu, hi);
      for (int m = 0; m < 4; m++) hi[m] = Ah * hi[m];
    }
    for (int m = 0; m < 4; m++) r[m] += (hi[m] - lo[m]) / hd[d];
  }
  const double b = a.stage == 1 ? 1.0 : 0.5;
  for (int m = 0; m < 4; m++) a.dst[1 + m][c] += b * a.dt * r[m];
}

void k3_launch_viscous(const Grid3 &g, const Fv3Args &a, cudaStream_t st) {
  dim3 grid((g.nx + S3_BX - 1) / S3_BX, (g.ny + S3_BY - 1) / S3_BY, (g.nz + S3_BZ - 1) / S3_BZ);
  k3_viscous<<<grid, S3_BX * S3_BY * S3_BZ, 0, st>>>(g, a);
  g_fv_launches++;
}

template <int BX, int BY, int BZ>
static void launch_fv_shape(const Grid3 &g, const Fv3Args &a, Scal3 *sc, cudaStream_t st) {
  using B = FvBrick<BX, BY, BZ>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k3_fv<BX, BY, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)B::smem);
    attr = true;
  }
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + BZ - 1) / BZ);
  k3_fv<BX, BY, BZ><<<grid, B::threads, B::smem, st>>>(g, a, sc);
}

int k3_fv_bricks(const Grid3 &g, int small) {
  return small ? ((g.nx + 3) / 4) * ((g.ny + 3) / 4) * ((g.nz + 3) / 4)
               : ((g.nx + S3_BX - 1) / S3_BX) * ((g.ny + S3_BY - 1) / S3_BY) *
                     ((g.nz + S3_BZ - 1) / S3_BZ);
}

void k3_launch_fv(const Grid3 &g, const Fv3Args &a, Scal3 *sc, cudaStream_t st, int small) {
  if (small)
    launch_fv_shape<4, 4, 4>(g, a, sc, st);
  else
    launch_fv_shape<S3_BX, S3_BY, S3_BZ>(g, a, sc, st);
  g_fv_launches++;
}
