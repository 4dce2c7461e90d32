// kernels_fv.cu -- the cut-cell finite-volume stage of one fluid (Eq. 2):
// WENO5-JS reconstruction of the Lax-Friedrichs split fluxes on every open
// face, face fluxes weighted by the fluid's apertures, the interface
// exchange flux X in cut cells and the Runge-Kutta stage combination.
//
// One CTA owns a TX x TY tile of output cells (a compile-time shape chosen
// per context from a small set; see sif_set_tile_shape).  The split fluxes
// of the tile and its 3-cell halo are built once in shared memory, every
// face flux is reconstructed once per CTA, and the update is written in
// place (a cell reads only its own conserved values).  Only the tiles in
// which the fluid can have an open face are launched.  FP64 throughout;
// the two reconstructions of a face and component share one division.
#include "sif_internal.cuh"
#include "weno_frac.cuh"

struct FvArgs {
  Grid g;
  int k, s;
  double a, b;  // RK stage weights
  double *dst[4];
  const double *base[4];
  const double *cur[4];
  const double *w[4];
  const double *ax, *ay, *sx, *sy;
  const double *xn[3];  // exchange flux planes: X applied to fluid k is (k ? -1 : 1) xn
  const int *tiles;
  const int *ntiles;
  int split_below;  // tile count under which each tile is split over two CTAs
  const double *dtp;
  const Scalars *sc;
};

// Characteristic reconstruction: the state of a face is the mean of the
// stencil states of the two cells beside it (cl, cr), taken in the face's
// frame (un along the face normal, ut across it).  For a stiffened gas the
// Euler flux Jacobian has the ideal-gas eigenstructure with c^2 = g (p +
// p_inf) / rho and H = c^2 / (g - 1) + q, q = (u^2 + v^2) / 2.
struct CharFace {
  double un, ut, c, ic, q, H, b1, b2;  // ic = 1 / c
};
constexpr int kCharFaceVals = 8;

__device__ __forceinline__ CharFace char_face(const FvArgs &A, int cl, int cr, bool ydir,
                                              double gm, double pi) {
  double rho = 0.5 * (A.w[0][cl] + A.w[0][cr]);
  double u = 0.5 * (A.w[1][cl] + A.w[1][cr]);
  double v = 0.5 * (A.w[2][cl] + A.w[2][cr]);
  double p = 0.5 * (A.w[3][cl] + A.w[3][cr]);
  CharFace f;
  f.un = ydir ? v : u;
  f.ut = ydir ? u : v;
  f.c = sqrt(gm * (p + pi) / rho);
  f.ic = 1.0 / f.c;
  f.q = 0.5 * (u * u + v * v);
  f.H = f.c * f.c / (gm - 1.0) + f.q;
  f.b1 = (gm - 1.0) / (f.c * f.c);
  f.b2 = f.b1 * f.q;
  return f;
}

// the face states of a block live in shared memory as kCharFaceVals planes
// of nf values
__device__ __forceinline__ void char_store(double *fs, int nf, int face, const CharFace &f) {
  fs[face] = f.un, fs[nf + face] = f.ut, fs[2 * nf + face] = f.c, fs[3 * nf + face] = f.ic;
  fs[4 * nf + face] = f.q, fs[5 * nf + face] = f.H, fs[6 * nf + face] = f.b1;
  fs[7 * nf + face] = f.b2;
}

__device__ __forceinline__ CharFace char_load(const double *fs, int nf, int face) {
  CharFace f;
  f.un = fs[face], f.ut = fs[nf + face], f.c = fs[2 * nf + face], f.ic = fs[3 * nf + face];
  f.q = fs[4 * nf + face], f.H = fs[5 * nf + face], f.b1 = fs[6 * nf + face];
  f.b2 = fs[7 * nf + face];
  return f;
}

// left eigenvector of field fld (0: un - c, 1: entropy, 2: shear, 3: un + c)
// over the grid's conserved components (rho, rho u, rho v, E)
__device__ __forceinline__ void char_left(const CharFace &f, int fld, bool ydir, double l[4]) {
  double n0, n1, n2, n3;  // over (rho, rho un, rho ut, E)
  if (fld == 0 || fld == 3) {
    const double s = fld == 0 ? 1.0 : -1.0, ic = f.ic;
    n0 = 0.5 * (f.b2 + s * f.un * ic);
    n1 = 0.5 * (-f.b1 * f.un - s * ic);
    n2 = 0.5 * (-f.b1 * f.ut);
    n3 = 0.5 * f.b1;
  } else if (fld == 1) {
    n0 = 1.0 - f.b2;
    n1 = f.b1 * f.un;
    n2 = f.b1 * f.ut;
    n3 = -f.b1;
  } else {
    n0 = -f.ut;
    n1 = 0.0;
    n2 = 1.0;
    n3 = 0.0;
  }
  l[0] = n0;
  l[1] = ydir ? n2 : n1;
  l[2] = ydir ? n1 : n2;
  l[3] = n3;
}

// row m (grid component) of the right eigenvectors, over the four fields
__device__ __forceinline__ void char_right_row(const CharFace &f, int m, bool ydir, double r[4]) {
  const int nm = (m == 1 || m == 2) && ydir ? 3 - m : m;  // row in (rho, rho un, rho ut, E)
  if (nm == 0) {
    r[0] = 1.0, r[1] = 1.0, r[2] = 0.0, r[3] = 1.0;
  } else if (nm == 1) {
    r[0] = f.un - f.c, r[1] = f.un, r[2] = 0.0, r[3] = f.un + f.c;
  } else if (nm == 2) {
    r[0] = f.ut, r[1] = f.ut, r[2] = 1.0, r[3] = f.ut;
  } else {
    r[0] = f.H - f.un * f.c, r[1] = f.q, r[2] = f.ut, r[3] = f.H + f.un * f.c;
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// end-of-block bookkeeping of the launch timer, by the blocks that had a
// tile (nwork of them): the last one adds the launch span and re-arms the
// timer for the next launch.  Blocks without a tile return at once and
// touch nothing.
__device__ void fv_timer_block_done(const Scalars *csc, unsigned int nwork) {
  Scalars *sc = (Scalars *)csc;
  atomicMax((unsigned long long *)&sc->fv_t1, globaltimer_ns());
  __threadfence();
  unsigned int done = atomicAdd(&sc->fv_blocks_done, 1u);
  if (done == nwork - 1) {
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

template <int TX, int TY>
struct FvShape {
  static constexpr int HX = TX + 6, HY = TY + 6;
  static constexpr int nfaces = (TX + 1) * TY + TX * (TY + 1);
  static constexpr size_t smem() {
    return sizeof(double) *
           (size_t)4 * (2 * HX * TY + 2 * TX * HY + (TX + 1) * TY + TX * (TY + 1));
  }
  // the characteristic form also keeps one face state per face
  static constexpr size_t smem_char() {
    return smem() + sizeof(double) * (size_t)kCharFaceVals * nfaces;
  }
  // two threads per output cell: a CTA's phases finish in half the time,
  // which matters when a fluid has few tiles (the sub-cycled fluid)
  static constexpr int threads = 2 * TX * TY;
  static_assert(threads >= TX * TY, "the open-cell count needs a thread per cell");
  // the HLLC form's stencil states and reconstructed face states fit the
  // split-flux layout's storage
  static_assert(4 * (HX * TY + TX * HY) + 8 * nfaces <=
                    4 * (2 * HX * TY + 2 * TX * HY) + 4 * nfaces,
                "HLLC shared memory");
};

// phase 3: update of the block's SX x SY cells from the aperture-weighted
// face fluxes FXo ([4][(SX+1)*SY]) and FYo ([4][SX*(SY+1)]) in shared
// memory; count the cells with an open face of fluid k (the work unit of
// the throughput figures)
template <int SX, int SY>
__device__ __forceinline__ void fv_update(const FvArgs &A, const double *FXo, const double *FYo,
                                          int i0, int j0) {
  const Grid &g = A.g;
  const int k = A.k;
  const bool d2 = g.dim == 2;
  const int tid = threadIdx.x, nth = blockDim.x;
  const double dt = *A.dtp;
  const double inv_dx = 1.0 / g.dx, inv_dy = 1.0 / g.dy, inv_dxdy = 1.0 / (g.dx * g.dy);
  const double sgn = k == 0 ? 1.0 : -1.0;
  const double closed = k == 0 ? 1.0 : 0.0;  // aperture A_P of a face closed to fluid k
  int open_cells = 0;
  for (int r = tid; r < SX * SY; r += nth) {
    int li = r % SX, lj = r / SX;
    int i = i0 + li, j = j0 + lj;
    if (i >= g.nx || j >= g.ny) continue;
    int c = gidx(g, i, j);
    bool open = A.ax[c] != closed || A.ax[c + 1] != closed;
    if (d2) open = open || A.ay[c] != closed || A.ay[c + g.PX] != closed;
    open_cells += open ? 1 : 0;
    bool cut = (A.sx[c] != 0.0 || A.sy[c] != 0.0);
#pragma unroll
    for (int m = 0; m < 4; m++) {
      const double *fx = FXo + m * (SX + 1) * SY + lj * (SX + 1) + li;
      double L = (fx[0] - fx[1]) * inv_dx;
      if (d2) {
        const double *fy = FYo + m * SX * (SY + 1) + lj * SX + li;
        L += (fy[0] - fy[SX]) * inv_dy;
      }
      if (m > 0 && cut) L += sgn * A.xn[m - 1][c] * inv_dxdy;
      double cur = A.cur[m][c];
      double out = A.s == 1 ? cur + dt * L : A.a * A.base[m][c] + A.b * (cur + dt * L);
      A.dst[m][c] = out;
    }
  }
  // every thread holds at most one cell here (a CTA has two threads per
  // cell of its tile, see FvShape), so the count is a barrier count
  const int nopen = __syncthreads_count(open_cells);
  if (tid == 0 && nopen > 0)
    atomicAdd((unsigned long long *)&A.sc->open_updates, (unsigned long long)nopen);
}

// the three phases over an SX x SY block of output cells at (i0, j0), with
// the CTA's threads (any count)
template <int SX, int SY, bool CH>
__device__ __forceinline__ void fv_cells(const FvArgs &A, double *smem, int i0, int j0) {
  constexpr int HX = SX + 6, HY = SY + 6;
  const Grid &g = A.g;
  const int k = A.k;
  // split fluxes: x for rows of the block with x-halo, y for columns with y-halo
  double *fxp = smem;                   // [4][HX*SY]
  double *fxm = fxp + 4 * HX * SY;      // [4][HX*SY]
  double *fyp = fxm + 4 * HX * SY;      // [4][SX*HY]
  double *fym = fyp + 4 * SX * HY;      // [4][SX*HY]
  double *Fx = fym + 4 * SX * HY;       // [4][(SX+1)*SY]
  double *Fy = Fx + 4 * (SX + 1) * SY;  // [4][SX*(SY+1)]
  // characteristic form: face states, x faces then y faces
  constexpr int NXF = (SX + 1) * SY, NF = NXF + SX * (SY + 1);
  double *fs = Fy + 4 * SX * (SY + 1);  // [kCharFaceVals][NF]
  const double gm = g.gamma[k], pi = g.pinf[k];
  const double inv_gm1 = 1.0 / (gm - 1.0), e0c = gm * pi * inv_gm1;
  // Lax-Friedrichs splitting f+- = F/2 +- (alpha/2) U
  const double hlx = 0.5 * ull_as_double(A.sc->lf[k][0]);
  const double hly = 0.5 * ull_as_double(A.sc->lf[k][1]);
  const bool d2 = g.dim == 2;
  const int tid = threadIdx.x, nth = blockDim.x;

  // phase 1: Lax-Friedrichs split fluxes of the stencil states
  for (int r = tid; r < HX * SY; r += nth) {
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
        fp[m] = 0.5 * F[m] + hlx * U[m];
        fm[m] = 0.5 * F[m] - hlx * U[m];
      }
    }
#pragma unroll
    for (int m = 0; m < 4; m++) {
      fxp[m * HX * SY + r] = fp[m];
      fxm[m * HX * SY + r] = fm[m];
    }
  }
  if (d2) {
    for (int r = tid; r < SX * HY; r += nth) {
      int i = i0 + r % SX, j = j0 - 3 + r / SX;
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
          fp[m] = 0.5 * F[m] + hly * U[m];
          fm[m] = 0.5 * F[m] - hly * U[m];
        }
      }
#pragma unroll
      for (int m = 0; m < 4; m++) {
        fyp[m * SX * HY + r] = fp[m];
        fym[m * SX * HY + r] = fm[m];
      }
    }
  }
  if constexpr (CH) {
    // the state of every open face (2D: also the y faces)
    const int nf = d2 ? NF : NXF;
    for (int r = tid; r < nf; r += nth) {
      const bool yd = r >= NXF;
      const int f = yd ? r - NXF : r;
      const int fi = yd ? f % SX : f % (SX + 1), fj = yd ? f / SX : f / (SX + 1);
      const int i = i0 + fi, j = j0 + fj;
      const bool open = yd ? (i < g.nx && j <= g.ny) : (i <= g.nx && j < g.ny);
      if (!open) continue;
      double A_ = yd ? A.ay[gidx(g, i, j)] : A.ax[gidx(g, i, j)];
      if (k == 0) A_ = 1.0 - A_;
      if (A_ == 0.0) continue;
      const int cr = gidx(g, i, j), cl = yd ? gidx(g, i, j - 1) : gidx(g, i - 1, j);
      char_store(fs, NF, r, char_face(A, cl, cr, yd, gm, pi));
    }
  }
  __syncthreads();

  // phase 2: one (face, component) per item, x faces (left face of cell
  // i0 + fi) then y faces (bottom face of cell j0 + fj) in one item range,
  // so that no thread takes more than one item above the CTA's average
  const double eps = g.weno_eps * (12.0 / 13.0);  // see weno5_frac
  constexpr int NXI = 4 * (SX + 1) * SY;
  const int NI = NXI + (d2 ? 4 * SX * (SY + 1) : 0);
  for (int r = tid; r < NI; r += nth) {
    const double *P, *M;
    double *out;
    int st;
    bool open;
    double A_ = 0.0;
    if (r < NXI) {
      int m = r / ((SX + 1) * SY), f = r % ((SX + 1) * SY);
      int fi = f % (SX + 1), fj = f / (SX + 1);
      int i = i0 + fi, j = j0 + fj;
      open = i <= g.nx && j < g.ny;
      if (open) A_ = A.ax[gidx(g, i, j)];
      // cells i-3..i+2 are at halo columns fi..fi+5
      P = fxp + m * HX * SY + fj * HX + fi;
      M = fxm + m * HX * SY + fj * HX + fi;
      st = 1;
      out = Fx + m * (SX + 1) * SY + f;
    } else {
      int q = r - NXI;
      int m = q / (SX * (SY + 1)), f = q % (SX * (SY + 1));
      int fi = f % SX, fj = f / SX;
      int i = i0 + fi, j = j0 + fj;
      open = i < g.nx && j <= g.ny;
      if (open) A_ = A.ay[gidx(g, i, j)];
      P = fyp + m * SX * HY + fj * SX + fi;
      M = fym + m * SX * HY + fj * SX + fi;
      st = SX;
      out = Fy + m * SX * (SY + 1) + f;
    }
    if (k == 0) A_ = 1.0 - A_;
    double val = 0.0;
    if (open && A_ != 0.0) {
      double nl, dl, nr, dr;
      if constexpr (CH) {
        // item (field, face): the field's left eigenvector applied to the
        // four components of each stencil value, then the field's
        // reconstructed split fluxes (the aperture comes with the mapping
        // back)
        const bool yd = r >= NXI;
        const int fld = yd ? (r - NXI) / (SX * (SY + 1)) : r / ((SX + 1) * SY);
        const int cs = yd ? SX * HY : HX * SY;  // component stride of the split fluxes
        const int f = yd ? (r - NXI) % (SX * (SY + 1)) : r % ((SX + 1) * SY);
        const CharFace cf = char_load(fs, NF, yd ? NXF + f : f);
        double l[4];
        char_left(cf, fld, yd, l);
        const double *P0 = P - fld * cs, *M0 = M - fld * cs;
        double vp[5], vm[5];
#pragma unroll
        for (int q = 0; q < 5; q++) {
          vp[q] = l[0] * P0[q * st] + l[1] * P0[cs + q * st] + l[2] * P0[2 * cs + q * st] +
                  l[3] * P0[3 * cs + q * st];
          vm[q] = l[0] * M0[(5 - q) * st] + l[1] * M0[cs + (5 - q) * st] +
                  l[2] * M0[2 * cs + (5 - q) * st] + l[3] * M0[3 * cs + (5 - q) * st];
        }
        weno5_frac(vp[0], vp[1], vp[2], vp[3], vp[4], eps, nl, dl);
        weno5_frac(vm[0], vm[1], vm[2], vm[3], vm[4], eps, nr, dr);
        val = face_value(1.0, nl, dl, nr, dr);
      } else {
        weno5_frac(P[0], P[st], P[2 * st], P[3 * st], P[4 * st], eps, nl, dl);
        weno5_frac(M[5 * st], M[4 * st], M[3 * st], M[2 * st], M[st], eps, nr, dr);
        val = face_value(A_, nl, dl, nr, dr);
      }
    }
    *out = val;
  }
  __syncthreads();

  // characteristic reconstruction: map the four fields of each face back
  // to the conserved components with the face's right eigenvectors, times
  // the aperture, into the split-flux storage (free after phase 2)
  double *FXo = Fx, *FYo = Fy;
  if constexpr (CH) {
    FXo = fxp;
    FYo = fyp;
    for (int r = tid; r < NI; r += nth) {
      const bool yd = r >= NXI;
      const int q = yd ? r - NXI : r;
      const int nf = yd ? SX * (SY + 1) : (SX + 1) * SY;
      const int m = q / nf, f = q % nf;
      const int fi = yd ? f % SX : f % (SX + 1), fj = yd ? f / SX : f / (SX + 1);
      const int i = i0 + fi, j = j0 + fj;
      const bool open = yd ? (i < g.nx && j <= g.ny) : (i <= g.nx && j < g.ny);
      double A_ = 0.0;
      if (open) A_ = yd ? A.ay[gidx(g, i, j)] : A.ax[gidx(g, i, j)];
      if (k == 0) A_ = 1.0 - A_;
      double val = 0.0;
      if (open && A_ != 0.0) {
        const CharFace cf = char_load(fs, NF, yd ? NXF + f : f);
        double rr[4];
        char_right_row(cf, m, yd, rr);
        const double *h = (yd ? Fy : Fx) + f;
        val = A_ * (rr[0] * h[0] + rr[1] * h[nf] + rr[2] * h[2 * nf] + rr[3] * h[3 * nf]);
      }
      (yd ? FYo : FXo)[m * nf + f] = val;
    }
    __syncthreads();
  }

  fv_update<SX, SY>(A, FXo, FYo, i0, j0);
}

// ---------------------------------------------------------------------
// HLLC face flux (option flux = 1; Toro, Riemann Solvers and Numerical
// Methods for Fluid Dynamics, Sec. 10.4): Davis's bounds S_L, S_R on the
// outer waves, the contact speed S* from the momentum balance across them,
// the star states U*_K = rho_K (S_K - un_K) / (S_K - S*) (1, S*, ut_K,
// E_K / rho_K + (S* - un_K) (S* + p_K / (rho_K (S_K - un_K)))) and the
// flux of the region holding the face.  W = (rho, u, v, p); F over (rho,
// rho u, rho v, E) of direction d.

__device__ __forceinline__ void euler_flux_state(const double W[4], double inv_gm1, double e0c,
                                                 bool yd, double F[4], double U[4]) {
  const double rho = W[0], u = W[1], v = W[2], p = W[3];
  const double E = p * inv_gm1 + e0c + 0.5 * rho * (u * u + v * v);
  const double un = yd ? v : u;
  const double mn = rho * un;
  U[0] = rho, U[1] = rho * u, U[2] = rho * v, U[3] = E;
  F[0] = mn, F[1] = mn * u, F[2] = mn * v, F[3] = un * (E + p);
  if (yd) F[2] += p;
  else F[1] += p;
}

__device__ __forceinline__ void hllc_flux(const double WL[4], const double WR[4], double gm,
                                          double pi, double inv_gm1, double e0c, bool yd,
                                          double F[4]) {
  const double rl = WL[0], rr = WR[0], pl = WL[3], pr = WR[3];
  const double ul = yd ? WL[2] : WL[1], ur = yd ? WR[2] : WR[1];
  const double cl = sqrt(gm * (pl + pi) / rl), cr = sqrt(gm * (pr + pi) / rr);
  const double SL = fmin(ul - cl, ur - cr), SR = fmax(ul + cl, ur + cr);
  double U[4];
  if (SL >= 0.0 || SR <= 0.0) {
    euler_flux_state(SL >= 0.0 ? WL : WR, inv_gm1, e0c, yd, F, U);
    return;
  }
  const double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
                    (rl * (SL - ul) - rr * (SR - ur));
  // the side of the contact the face lies on
  const bool left = Ss >= 0.0;
  const double *W = left ? WL : WR;
  const double SK = left ? SL : SR, uK = left ? ul : ur;
  euler_flux_state(W, inv_gm1, e0c, yd, F, U);
  const double fac = W[0] * (SK - uK) / (SK - Ss);
  double Us[4];
  Us[0] = fac;
  Us[1] = fac * (yd ? W[1] : Ss);
  Us[2] = fac * (yd ? Ss : W[2]);
  Us[3] = fac * (U[3] / W[0] + (Ss - uK) * (Ss + W[3] / (W[0] * (SK - uK))));
#pragma unroll
  for (int m = 0; m < 4; m++) F[m] = F[m] + SK * (Us[m] - U[m]);
}

// a WENO5 reconstruction as one value (the fraction over a reciprocal, a
// division where the denominator leaves the reciprocal's range)
__device__ __forceinline__ double weno5_value(double v1, double v2, double v3, double v4,
                                              double v5, double eps12_13) {
  double n, d;
  weno5_frac(v1, v2, v3, v4, v5, eps12_13, n, d);
  if (d < 0x1p1000 && isfinite(n)) return n * recip_newton3(d);
  return n / d;
}

// the HLLC stage over an SX x SY block: (1) the stencil states of the
// block's rows with x-halo and columns with y-halo, (2) per (face,
// component) the WENO5 reconstructions from the left and from the right,
// (3) per face the HLLC flux of the two reconstructed states (a state with
// rho <= 0 or p + pinf <= 0 replaced by its cell's), times the aperture,
// into the storage of (1), (4) the update
template <int SX, int SY>
__device__ __forceinline__ void fv_cells_hllc(const FvArgs &A, double *smem, int i0, int j0) {
  constexpr int HX = SX + 6, HY = SY + 6;
  constexpr int NXF = (SX + 1) * SY, NYF = SX * (SY + 1);
  const Grid &g = A.g;
  const int k = A.k;
  double *wx = smem;                // [4][HX*SY]
  double *wy = wx + 4 * HX * SY;    // [4][SX*HY]
  double *WL = wy + 4 * SX * HY;    // [4][NXF + NYF], x faces then y faces
  double *WR = WL + 4 * (NXF + NYF);
  double *Fx = wx;                  // [4][NXF] (over wx, free after (2))
  double *Fy = wy;                  // [4][NYF]
  const double gm = g.gamma[k], pi = g.pinf[k];
  const double inv_gm1 = 1.0 / (gm - 1.0), e0c = gm * pi * inv_gm1;
  const bool d2 = g.dim == 2;
  const int tid = threadIdx.x, nth = blockDim.x;

  for (int r = tid; r < HX * SY; r += nth) {
    int i = i0 - 3 + r % HX, j = j0 + r / HX;
    const bool ok = i <= g.nx + 2 && j < g.ny;
    const int c = ok ? gidx(g, i, j) : 0;
#pragma unroll
    for (int m = 0; m < 4; m++) wx[m * HX * SY + r] = ok ? A.w[m][c] : 0.0;
  }
  if (d2)
    for (int r = tid; r < SX * HY; r += nth) {
      int i = i0 + r % SX, j = j0 - 3 + r / SX;
      const bool ok = i < g.nx && j <= g.ny + 2;
      const int c = ok ? gidx(g, i, j) : 0;
#pragma unroll
      for (int m = 0; m < 4; m++) wy[m * SX * HY + r] = ok ? A.w[m][c] : 0.0;
    }
  __syncthreads();

  const double eps = g.weno_eps * (12.0 / 13.0);  // see weno5_frac
  constexpr int NXI = 4 * NXF;
  const int NI = NXI + (d2 ? 4 * NYF : 0);
  for (int r = tid; r < NI; r += nth) {
    const double *P;
    int st, slot;
    if (r < NXI) {
      const int m = r / NXF, f = r % NXF;
      const int fi = f % (SX + 1), fj = f / (SX + 1);
      // cells i-3..i+2 of face i are at halo columns fi..fi+5
      P = wx + m * HX * SY + fj * HX + fi;
      st = 1;
      slot = m * (NXF + NYF) + f;
    } else {
      const int q = r - NXI, m = q / NYF, f = q % NYF;
      const int fi = f % SX, fj = f / SX;
      P = wy + m * SX * HY + fj * SX + fi;
      st = SX;
      slot = m * (NXF + NYF) + NXF + f;
    }
    WL[slot] = weno5_value(P[0], P[st], P[2 * st], P[3 * st], P[4 * st], eps);
    WR[slot] = weno5_value(P[5 * st], P[4 * st], P[3 * st], P[2 * st], P[st], eps);
  }
  __syncthreads();

  const int nfc = NXF + (d2 ? NYF : 0);
  for (int r = tid; r < nfc; r += nth) {
    const bool yd = r >= NXF;
    const int f = yd ? r - NXF : r;
    const int fi = yd ? f % SX : f % (SX + 1), fj = yd ? f / SX : f / (SX + 1);
    const int i = i0 + fi, j = j0 + fj;
    const bool open = yd ? (i < g.nx && j <= g.ny) : (i <= g.nx && j < g.ny);
    double A_ = 0.0;
    if (open) A_ = yd ? A.ay[gidx(g, i, j)] : A.ax[gidx(g, i, j)];
    if (k == 0) A_ = 1.0 - A_;
    double Fh[4] = {0.0, 0.0, 0.0, 0.0};
    if (open && A_ != 0.0) {
      const int cr = gidx(g, i, j), cl = yd ? gidx(g, i, j - 1) : gidx(g, i - 1, j);
      double wl[4], wr[4];
#pragma unroll
      for (int m = 0; m < 4; m++) {
        wl[m] = WL[m * (NXF + NYF) + r];
        wr[m] = WR[m * (NXF + NYF) + r];
      }
      if (!(wl[0] > 0.0) || !(wl[3] + pi > 0.0))
#pragma unroll
        for (int m = 0; m < 4; m++) wl[m] = A.w[m][cl];
      if (!(wr[0] > 0.0) || !(wr[3] + pi > 0.0))
#pragma unroll
        for (int m = 0; m < 4; m++) wr[m] = A.w[m][cr];
      hllc_flux(wl, wr, gm, pi, inv_gm1, e0c, yd, Fh);
    }
    double *out = yd ? Fy + f : Fx + f;
    const int nf = yd ? NYF : NXF;
#pragma unroll
    for (int m = 0; m < 4; m++) out[m * nf] = A_ * Fh[m];
  }
  __syncthreads();
  fv_update<SX, SY>(A, Fx, Fy, i0, j0);
}

// A fluid with fewer active tiles than the GPU has SMs (the sub-cycled
// fluid of a small region) has each tile computed by two CTAs, one half of
// the tile each along its longer side, and with at most a quarter as many
// tiles as SMs by four CTAs, quarters of the tile (along x when the tile is
// at least four times as wide as high, else two by two): more SMs for the
// same face fluxes (the halo share grows, the arithmetic per face is the
// same).  Quarters of more tiles than that would put two CTAs on some SMs
// and finish later than halves.
template <int TX, int TY>
struct FvHalf {
  static constexpr bool along_x = TX >= TY;
  static constexpr int SX = along_x ? TX / 2 : TX, SY = along_x ? TY : TY / 2;
  __device__ static void origin(int part, int &i0, int &j0) {
    if (part) {
      if (along_x) i0 += SX;
      else j0 += SY;
    }
  }
};
template <int TX, int TY>
struct FvQuarter {
  static constexpr bool along_x = TX >= 4 * TY;
  static constexpr int SX = along_x ? TX / 4 : TX / 2, SY = along_x ? TY : TY / 2;
  __device__ static void origin(int part, int &i0, int &j0) {
    if (along_x) {
      i0 += part * SX;
    } else {
      i0 += (part & 1) * SX;
      j0 += (part >> 1) * SY;
    }
  }
};

// MODE: 0 WENO5-LF per component, 1 WENO5-LF on characteristic fields, 2
// HLLC (1 and 2 take more registers a thread: two CTAs per SM, not three)
template <int TX, int TY, int MODE>
__global__ void __launch_bounds__(FvShape<TX, TY>::threads,
                                  (MODE == 0 ? 1536 : 1024) / FvShape<TX, TY>::threads)
k_fv_stage(FvArgs A) {
  SIF_TICK();
  const Grid &g = A.g;
  const int ntiles = A.ntiles[A.k];
  // CTAs per tile (the grid holds at least twice as many CTAs as SMs):
  // quarters only while every quarter still gets an SM of its own
  const int parts = 4 * ntiles <= A.split_below ? 4 : (ntiles < A.split_below ? 2 : 1);
  const int t = (int)blockIdx.x / parts, part = (int)blockIdx.x % parts;
  if (t >= ntiles) return;
  extern __shared__ double smem[];
  const int tile = A.tiles[t];
  int i0 = (tile % g.ntx) * TX, j0 = (tile / g.ntx) * TY;
  using H = FvHalf<TX, TY>;
  using Q = FvQuarter<TX, TY>;
  if (parts == 2) H::origin(part, i0, j0);
  if (parts == 4) Q::origin(part, i0, j0);
  if (threadIdx.x == 0) {
    const int bw = parts == 4 ? Q::SX : (parts == 2 ? H::SX : TX);
    const int bh = parts == 4 ? Q::SY : (parts == 2 ? H::SY : TY);
    int w_ = min(bw, g.nx - i0), h_ = min(bh, g.ny - j0);
    if (w_ > 0 && h_ > 0)
      atomicAdd((unsigned long long *)&A.sc->updates, (unsigned long long)(w_ * h_));
  }
  const bool timed = A.sc->timing;
  if (timed && threadIdx.x == 0) atomicMin((unsigned long long *)&A.sc->fv_t0, globaltimer_ns());
  if constexpr (MODE == 2) {
    if (parts == 4) fv_cells_hllc<Q::SX, Q::SY>(A, smem, i0, j0);
    else if (parts == 2) fv_cells_hllc<H::SX, H::SY>(A, smem, i0, j0);
    else fv_cells_hllc<TX, TY>(A, smem, i0, j0);
  } else {
    constexpr bool CH = MODE == 1;
    if (parts == 4) fv_cells<Q::SX, Q::SY, CH>(A, smem, i0, j0);
    else if (parts == 2) fv_cells<H::SX, H::SY, CH>(A, smem, i0, j0);
    else fv_cells<TX, TY, CH>(A, smem, i0, j0);
  }
  if (timed) {
    __syncthreads();
    if (threadIdx.x == 0) fv_timer_block_done(A.sc, (unsigned int)(parts * ntiles));
  }
}

// the supported tile shapes (output cells per CTA)
#define FV_SHAPES(X) X(32, 8) X(32, 4) X(16, 8) X(16, 16) X(64, 4)

bool fv_shape_supported(int tx, int ty) {
#define FV_IS(a, b) \
  if (tx == a && ty == b) return true;
  FV_SHAPES(FV_IS)
#undef FV_IS
  return false;
}

// opt every instantiation into its shared-memory size on the current
// device (outside any stream capture)
// launch priority of the finite-volume stage: the device's greatest, so
// that its pending CTAs go before those of work branched beside it (the
// level-set velocity's extension in a captured cycle)
static int g_fv_priority = 0;

void fv_prepare() {
#define FV_PREP(a, b)                                                                      \
  cudaFuncSetAttribute(k_fv_stage<a, b, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)FvShape<a, b>::smem());                                      \
  cudaFuncSetAttribute(k_fv_stage<a, b, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)FvShape<a, b>::smem_char());                                 \
  cudaFuncSetAttribute(k_fv_stage<a, b, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)FvShape<a, b>::smem());
  FV_SHAPES(FV_PREP)
#undef FV_PREP
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess) g_fv_priority = greatest;
  cudaGetLastError();
}

void launch_fv_stage(const Grid &g, int k, int s, int rk, double *const dst[4],
                     double *const base[4], double *const cur[4], double *const w[4],
                     const double *ax, const double *ay, const double *sx, const double *sy,
                     const double *xn0, const double *xn1, const double *xn2, const int *tiles,
                     int tile_cap, int num_sms, const double *dtp, Scalars *sc,
                     cudaStream_t st) {
  static const double A2[3] = {0.0, 0.0, 0.5}, B2[3] = {0.0, 1.0, 0.5};
  static const double A3[4] = {0.0, 0.0, 0.75, 1.0 / 3.0}, B3[4] = {0.0, 1.0, 0.25, 2.0 / 3.0};
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
  A.sc = sc;
  A.split_below = num_sms;
  const int grid = tile_cap > 2 * num_sms ? tile_cap : 2 * num_sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributePriority;
  at.val.priority = g_fv_priority;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
#define FV_LAUNCH(a, b)                                    \
  if (g.tx == a && g.ty == b) {                           \
    cfg.blockDim = dim3(FvShape<a, b>::threads);          \
    if (g.weno_char) {                                    \
      cfg.dynamicSmemBytes = FvShape<a, b>::smem_char();  \
      cudaLaunchKernelEx(&cfg, k_fv_stage<a, b, 1>, A);   \
    } else if (g.flux == 1) {                             \
      cfg.dynamicSmemBytes = FvShape<a, b>::smem();       \
      cudaLaunchKernelEx(&cfg, k_fv_stage<a, b, 2>, A);   \
    } else {                                              \
      cfg.dynamicSmemBytes = FvShape<a, b>::smem();       \
      cudaLaunchKernelEx(&cfg, k_fv_stage<a, b, 0>, A);   \
    }                                                     \
    return;                                               \
  }
  FV_SHAPES(FV_LAUNCH)
#undef FV_LAUNCH
}

// ---------------------------------------------------------------------
// viscous fluxes (Eq. 5's face terms): the viscous face flux from the
// stencil states by central differences (normal derivatives across the
// face, tangential ones averaged over the two cells), times the aperture;
// the stage result gains b dt times their divergence.  One thread per cell,
// each face computed by both of its cells.

// viscous flux of fluid k through the face between cells cl and cr of
// direction d (0: x, cr = cl + 1; 1: y, cr = cl + PX)
__device__ __forceinline__ void viscous_face(const Grid &g, double mu, const double *u,
                                             const double *v, int cl, int cr, int d,
                                             double Fv[3]) {
  double ux, uy, vx, vy;
  if (d == 0) {
    ux = (u[cr] - u[cl]) / g.dx;
    vx = (v[cr] - v[cl]) / g.dx;
    if (g.dim == 2) {
      const int t = g.PX;
      uy = ((u[cr + t] - u[cr - t]) + (u[cl + t] - u[cl - t])) / (4.0 * g.dy);
      vy = ((v[cr + t] - v[cr - t]) + (v[cl + t] - v[cl - t])) / (4.0 * g.dy);
    } else {
      uy = vy = 0.0;
    }
  } else {
    uy = (u[cr] - u[cl]) / g.dy;
    vy = (v[cr] - v[cl]) / g.dy;
    ux = ((u[cr + 1] - u[cr - 1]) + (u[cl + 1] - u[cl - 1])) / (4.0 * g.dx);
    vx = ((v[cr + 1] - v[cr - 1]) + (v[cl + 1] - v[cl - 1])) / (4.0 * g.dx);
  }
  double txx, txy, tyy;
  visc_stress(mu, ux, uy, vx, vy, txx, txy, tyy);
  const double uf = 0.5 * (u[cl] + u[cr]), vf = 0.5 * (v[cl] + v[cr]);
  if (d == 0) {
    Fv[0] = txx, Fv[1] = txy, Fv[2] = uf * txx + vf * txy;
  } else {
    Fv[0] = txy, Fv[1] = tyy, Fv[2] = uf * txy + vf * tyy;
  }
}

__global__ void k_viscous(Grid g, int k, double bw, const double *dtp, const int *tiles,
                          const int *ntiles, const double *__restrict__ u,
                          const double *__restrict__ v, const double *__restrict__ ax,
                          const double *__restrict__ ay, double *d1, double *d2, double *d3) {
  SIF_TICK();
  if ((int)blockIdx.x >= ntiles[k]) return;
  const int tile = tiles[blockIdx.x];
  const int i0 = (tile % g.ntx) * g.tx, j0 = (tile / g.ntx) * g.ty;
  const double mu = g.mu[k], dt = *dtp;
  for (int r = threadIdx.x; r < g.tx * g.ty; r += blockDim.x) {
    const int i = i0 + r % g.tx, j = j0 + r / g.tx;
    if (i >= g.nx || j >= g.ny) continue;
    const int c = gidx(g, i, j);
    double L[3] = {0.0, 0.0, 0.0};
    // x faces: left (i) and right (i + 1)
    for (int side = 0; side < 2; side++) {
      const int cf = c + side;  // the face's right cell
      double A_ = ax[cf];
      if (k == 0) A_ = 1.0 - A_;
      if (A_ == 0.0) continue;
      double Fv[3];
      viscous_face(g, mu, u, v, cf - 1, cf, 0, Fv);
      const double w_ = (side ? A_ : -A_) / g.dx;
      for (int m = 0; m < 3; m++) L[m] += w_ * Fv[m];
    }
    if (g.dim == 2)
      for (int side = 0; side < 2; side++) {
        const int cf = c + side * g.PX;
        double A_ = ay[cf];
        if (k == 0) A_ = 1.0 - A_;
        if (A_ == 0.0) continue;
        double Fv[3];
        viscous_face(g, mu, u, v, cf - g.PX, cf, 1, Fv);
        const double w_ = (side ? A_ : -A_) / g.dy;
        for (int m = 0; m < 3; m++) L[m] += w_ * Fv[m];
      }
    const double f = bw * dt;
    d1[c] += f * L[0];
    d2[c] += f * L[1];
    d3[c] += f * L[2];
  }
}

void launch_viscous(const Grid &g, int k, int s, int rk, double *const dst[4],
                    double *const w[4], const double *ax, const double *ay, const int *tiles,
                    int tile_cap, const double *dtp, Scalars *sc, cudaStream_t st) {
  static const double B2[3] = {0.0, 1.0, 0.5}, B3[4] = {0.0, 1.0, 0.25, 2.0 / 3.0};
  const double bw = rk == 3 ? B3[s] : B2[s];
  launch_k(k_viscous, tile_cap > 0 ? tile_cap : 1, 128, 0, st, g, k, bw, dtp, tiles, sc->n_tiles,
                                                        w[1], w[2], ax, ay, dst[1], dst[2],
                                                        dst[3]);
  sif_note_launches(1);
}

SIF_TU_LAUNCH_READER(fv)
