// kernels_band.cu -- stencil states of each fluid (real cells and the
// ghost-state extension of Sec. 2.3), the interface interaction (exact
// two-material Riemann problem giving the exchange flux X of Eq. 2 and the
// level-set velocity of Eq. 6), level-set advection and reinitialisation,
// the multi-time-step bookkeeping (Eq. 7 interpolation, Eq. 8-9 correction
// quantities), conserved totals and the device-side scheduler.
//
// Compiled without FMA contraction, like kernels_geom.cu: these kernels
// follow the CPU reference operation by operation so that threshold and
// branch decisions agree with it -- except the level-set derivatives, whose
// WENO5 weights take one division (rounding-level differences; their only
// decisions are clamps, continuous in the value).
#include "sif_internal.cuh"

static int grid_for(int n, int per = 256, int cap = 4096) {
  int b = (n + per - 1) / per;
  if (b > cap) b = cap;
  return b < 1 ? 1 : b;
}

__device__ inline void block_max2(double a, double b, unsigned long long *pa,
                                  unsigned long long *pb) {
  __shared__ double sa[32], sb[32];
  a = warp_max(a);
  b = warp_max(b);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    a = warp_max(a);
    b = warp_max(b);
    if (lane == 0) {
      if (pa) atomic_max_pos(pa, a);
      if (pb) atomic_max_pos(pb, b);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------
// real-cell stencil states W = prim((alpha U)/alpha) and wave maxima

struct PrimArgs {
  const double *q[2][4];
  double *w[2][4];
  const int *tiles[2];
  unsigned char *nostate[2];
  // fluid whose states are needed in the interaction band only (-1: none),
  // unless *band_flag is set (then everywhere, like the other fluid)
  int band_fluid;
  const int *band_flag;
  const int *band;
  const int *nband;
  int skip_fluid;  // fluid whose states are not recovered at all (-1: none)
};

// blockIdx.y = fluid; the cells of the fluid's tiles, or of the band
__global__ void k_prim(Grid g, PrimArgs P, const double *__restrict__ alpha, const int *ntiles,
                       Scalars *sc) {
  SIF_TICK();
  const int k = blockIdx.y;
  if (k == P.skip_fluid) return;
  const bool band_only = k == P.band_fluid && !(P.band_flag && *P.band_flag);
  bool valid;
  int c = 0;
  if (band_only) {
    int nb = *P.nband;
    if ((int)(blockIdx.x * blockDim.x) >= nb) return;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    valid = idx < nb;
    if (valid) c = P.band[idx];
  } else {
    if ((int)blockIdx.x >= ntiles[k]) return;
    int tile = P.tiles[k][blockIdx.x];
    int tx = tile % g.ntx, ty = tile / g.ntx;
    int i = tx * g.tx + (threadIdx.x % g.tx), j = ty * g.ty + threadIdx.x / g.tx;
    valid = i < g.nx && j < g.ny;
    if (valid) c = gidx(g, i, j);
  }
  const double *q0 = P.q[k][0], *q1 = P.q[k][1], *q2 = P.q[k][2], *q3 = P.q[k][3];
  double *w0 = P.w[k][0], *w1 = P.w[k][1], *w2 = P.w[k][2], *w3 = P.w[k][3];
  const double idx_ = 1.0 / g.dx, idy_ = 1.0 / g.dy;
  double lx = 0.0, ly = 0.0, sm = 0.0;
  if (valid) {
    double a = vol_k(alpha, k, c);
    unsigned char nostate = 0;
    if (a > SIF_ALPHA_REAL) {
      double gm = g.gamma[k], pi = g.pinf[k];
      // one reciprocal of the mass serves u, v and 1/rho = alpha / (alpha
      // rho); a full cell divides by exactly 1 and skips two more divisions
      double iq = 1.0 / q0[c];
      double rho = a == 1.0 ? q0[c] : q0[c] / a;
      double u = q1[c] * iq;
      double v = q2[c] * iq;
      double E = a == 1.0 ? q3[c] : q3[c] / a;
      // Tait's equation (Eq. 4): the pressure of the density alone
      double p = g.tait[k] ? g.tB[k] * (pow(rho / g.trho0[k], gm) - 1.0) + g.tp0[k]
                           : (gm - 1.0) * (E - 0.5 * rho * (u * u + v * v)) - gm * pi;
      bool phys = rho > 0.0 && p + pi > 0.0;
      // a cut cell whose content is not a physical state takes an
      // extended state like a sliver; a full cell with such content is an
      // error
      if (!phys && a < 1.0) {
        nostate = 1;
      } else {
        if (!phys) atomicOr(&sc->err, DERR_NONPHYS);
        w0[c] = rho;
        w1[c] = u;
        w2[c] = v;
        w3[c] = p;
        double cs = sqrt(fmax(gm * (p + pi) * (a * iq), 0.0));
        lx = fabs(u) + cs;
        ly = fabs(v) + cs;
        // CFL rate (|u| + c) / dx + (|v| + c) / dy with the reciprocals
        // taken once (an ulp from the quotients in the step size)
        double s = lx * idx_;
        if (g.dim == 2) s += ly * idy_;
        // explicit viscous limit: 2 nu (1/dx^2 + 1/dy^2) added to the rate
        if (g.mu[k] > 0.0) {
          const double id2 = 1.0 / (g.dx * g.dx) + (g.dim == 2 ? 1.0 / (g.dy * g.dy) : 0.0);
          s += 2.0 * g.mu[k] / rho * id2;
        }
        sm = s;
      }
    }
    P.nostate[k][c] = nostate;
  }
  // two reductions share the helper: (lx, ly), then (sm, -)
  block_max2(lx, ly, &sc->lf[k][0], &sc->lf[k][1]);
  block_max2(sm, 0.0, &sc->smax[k], nullptr);
}

void launch_prim2(const Grid &g, double *const qN[4], double *const qP[4], double *const wN[4],
                  double *const wP[4], const double *alpha, const int *tilesN,
                  const int *tilesP, int tile_cap, unsigned char *const nostate[2], Scalars *sc,
                  int band_fluid, const int *band_flag, const int *band, const int *nband,
                  cudaStream_t st, int skip_fluid) {
  PrimArgs P;
  P.skip_fluid = skip_fluid;
  P.band_fluid = band_fluid;
  P.band_flag = band_flag;
  P.band = band;
  P.nband = nband;
  P.nostate[0] = nostate[0];
  P.nostate[1] = nostate[1];
  for (int m = 0; m < 4; m++) {
    P.q[0][m] = qN[m];
    P.q[1][m] = qP[m];
    P.w[0][m] = wN[m];
    P.w[1][m] = wP[m];
  }
  P.tiles[0] = tilesN;
  P.tiles[1] = tilesP;
  launch_k(k_prim, dim3(tile_cap, 2), g.tx * g.ty, 0, st, g, P, alpha, sc->n_tiles, sc);
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// interface interaction in every cut cell

// riemann_solve with one side of the problem per lane of a lane pair (even
// lane: fluid N on the left, odd lane: fluid P on the right).  Each lane
// evaluates its own side's wave function and derivative, the pair
// exchanges them, and both lanes take the same Newton step with the same
// operations in the same order as riemann_solve, so the star state is the
// same to the bit.  With surface tension the left star pressure exceeds
// the right one by jump (Eq. 10): Newton runs on the right star pressure p,
// the left lane evaluating its wave function at p + jump.  Returns 0 or
// DERR_NOCONV; out: the lane's own star pressure, u*, and the lane's own
// star sound speed.
__device__ inline int riemann_solve_pair(unsigned pair, int side, double rho, double un,
                                         double pk, double gk, double pik, double jump,
                                         int maxit, int baro, double &ps, double &us,
                                         double &cs) {
  double ck = sqrt(gk * (pk + pik) / rho);
  double ro = __shfl_xor_sync(pair, rho, 1), uo = __shfl_xor_sync(pair, un, 1);
  double po = __shfl_xor_sync(pair, pk, 1), pio = __shfl_xor_sync(pair, pik, 1);
  double co = __shfl_xor_sync(pair, ck, 1);
  const bool L = side == 0;
  double rl = L ? rho : ro, ul = L ? un : uo, pl = L ? pk : po, pil = L ? pik : pio;
  double rr = L ? ro : rho, ur = L ? uo : un, pr = L ? po : pk, pir = L ? pio : pik;
  double cl = L ? ck : co, cr = L ? co : ck;
  double pscale = fmin(pl + pil, pr + pir);
  double pfloor = fmax(-pir, -pil - jump) + 1e-12 * pscale;
  double p = 0.5 * ((pl - jump) + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
  // iterates stay above the floor without landing on it (a rarefaction's
  // derivative diverges there and a tiny step would pass for convergence)
  if (p < pfloor) p = pfloor + 0.5 * (fmax(pl - jump, pr) - pfloor);
  const double own = L ? jump : 0.0;  // this lane's star pressure is p + own
  const SideConst sk = side_const(rho, pk, gk, pik, ck, baro);
  int it = 0, conv = 0, done = 0;
  double f, df;
  while (it < maxit) {
    it++;
    riemann_side_k(p + own, sk, f, df);
    double fo = __shfl_xor_sync(pair, f, 1), dfo = __shfl_xor_sync(pair, df, 1);
    double fl = L ? f : fo, fr = L ? fo : f, dfl = L ? df : dfo, dfr = L ? dfo : df;
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
  ps = p + own;
  riemann_side_k(ps, sk, f, df);
  double fo = __shfl_xor_sync(pair, f, 1);
  double fl = L ? f : fo, fr = L ? fo : f;
  us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  double rs = riemann_star_density(ps, rho, pk, gk, pik, baro);
  cs = sqrt(gk * (ps + pik) / rs);
  return (done || conv) ? 0 : DERR_NOCONV;
}

// curvature div(grad phi / |grad phi|) at cell (i, j): (phi_xx phi_y^2 -
// 2 phi_x phi_y phi_xy + phi_yy phi_x^2) / |grad phi|^3 from second-order
// central differences; 0 in 1D or where grad phi vanishes
__device__ inline double curvature(const Grid &g, const double *phi, int i, int j) {
  if (g.dim != 2) return 0.0;
  const double dx = g.dx, dy = g.dy;
  const double c0 = phi[gidx(g, i, j)];
  const double e = phi[gidx(g, i + 1, j)], w = phi[gidx(g, i - 1, j)];
  const double n = phi[gidx(g, i, j + 1)], s = phi[gidx(g, i, j - 1)];
  const double px = (e - w) / (2.0 * dx), py = (n - s) / (2.0 * dy);
  const double pxx = (e - 2.0 * c0 + w) / (dx * dx), pyy = (n - 2.0 * c0 + s) / (dy * dy);
  const double pxy = (phi[gidx(g, i + 1, j + 1)] - phi[gidx(g, i + 1, j - 1)] -
                      phi[gidx(g, i - 1, j + 1)] + phi[gidx(g, i - 1, j - 1)]) /
                     (4.0 * dx * dy);
  const double g2 = px * px + py * py;
  if (!(g2 > 0.0)) return 0.0;
  return (pxx * py * py - 2.0 * px * py * pxy + pyy * px * px) / (g2 * sqrt(g2));
}

// two lanes per cut cell (blockDim a multiple of 32)
__global__ void k_interface(Grid g, const double *__restrict__ n0, const double *__restrict__ n1,
                            const double *__restrict__ n2, const double *__restrict__ n3,
                            const double *__restrict__ p0, const double *__restrict__ p1,
                            const double *__restrict__ p2, const double *__restrict__ p3,
                            const double *__restrict__ phi, const double *__restrict__ sx,
                            const double *__restrict__ sy, const int *__restrict__ cut,
                            const int *ncut, double *xn0, double *xn1, double *xn2,
                            double *xm0, double *xm1, double *xm2, double *ul0, double *ul1,
                            Scalars *sc) {
  SIF_TICK();
  int n = *ncut;
  double fac = 1.0 / g.dx + (g.dim == 2 ? 1.0 / g.dy : 0.0);
  double sN = 0.0, sP = 0.0;
  const int side = threadIdx.x & 1;
  const unsigned pair = 3u << (threadIdx.x & 30);
  // the stride is even: both lanes of a pair stay on the same cell
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; (t >> 1) < n; t += gridDim.x * blockDim.x) {
    int c = cut[t >> 1];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    double Sx = sx[c], Sy = sy[c];
    double Sm = sqrt(Sx * Sx + Sy * Sy);
    double nxv, nyv;
    unit_normal(g, phi, i, j, nxv, nyv);
    if (nxv == 0.0 && nyv == 0.0) {
      nxv = Sx / Sm;
      nyv = Sy / Sm;
    }
    double rho, un, pk;
    if (side == 0) {
      rho = n0[c];
      un = n1[c] * nxv + n2[c] * nyv;
      pk = n3[c];
    } else {
      rho = p0[c];
      un = p1[c] * nxv + p2[c] * nyv;
      pk = p3[c];
    }
    // surface tension: the pressure jumps by sigma kappa from fluid P into
    // fluid N (Eq. 10; kappa > 0 where fluid N is convex)
    const double jump = g.sigma != 0.0 ? g.sigma * curvature(g, phi, i, j) : 0.0;
    double ps, us, cs;
    int e = riemann_solve_pair(pair, side, rho, un, pk, g.gamma[side], g.pinf[side], jump,
                               g.newton_max, g.tait[side], ps,
                               us, cs);
    if (e && side == 0) atomicOr(&sc->err, e);
    // each fluid's exchange flux with its own interface pressure: fluid N
    // -p_N (S, u* |S|) in xn, fluid P +p_P (S, u* |S|), stored negated in xm
    // (so that without surface tension xm equals xn bitwise)
    if (side == 0) {
      xn0[c] = -ps * Sx;
      xn1[c] = -ps * Sy;
      xn2[c] = -ps * us * Sm;
      ul0[c] = us * nxv;
      ul1[c] = us * nyv;
      sN = fmax(sN, (fabs(us) + cs) * fac);
    } else {
      xm0[c] = -ps * Sx;
      xm1[c] = -ps * Sy;
      xm2[c] = -ps * us * Sm;
      sP = fmax(sP, (fabs(us) + cs) * fac);
    }
    // viscous traction across the interface: the stress of the velocity
    // field that is continuous across it (at every cell the velocity of
    // the fluid on whose side its centre lies) by central differences at
    // the cut cell, with the harmonic mean of the viscosities; fluid N
    // receives it through S, fluid P the opposite (its planes hold the
    // negated flux, so both lanes add the same values), each with its work
    // at that field's velocity in the cut cell
    if (g.mu[0] > 0.0 && g.mu[1] > 0.0) {
      const double muI = 2.0 * g.mu[0] * g.mu[1] / (g.mu[0] + g.mu[1]);
      auto U = [&](int ii, int jj) {
        const int cc = gidx(g, ii, jj);
        return phi[cc] < 0.0 ? n1[cc] : p1[cc];
      };
      auto V = [&](int ii, int jj) {
        const int cc = gidx(g, ii, jj);
        return phi[cc] < 0.0 ? n2[cc] : p2[cc];
      };
      const double ux = (U(i + 1, j) - U(i - 1, j)) / (2.0 * g.dx);
      const double vx = (V(i + 1, j) - V(i - 1, j)) / (2.0 * g.dx);
      double uy = 0.0, vy = 0.0;
      if (g.dim == 2) {
        uy = (U(i, j + 1) - U(i, j - 1)) / (2.0 * g.dy);
        vy = (V(i, j + 1) - V(i, j - 1)) / (2.0 * g.dy);
      }
      double txx, txy, tyy;
      visc_stress(muI, ux, uy, vx, vy, txx, txy, tyy);
      const double fx = txx * Sx + txy * Sy, fy = txy * Sx + tyy * Sy;
      const double e = U(i, j) * fx + V(i, j) * fy;
      double *X0 = side == 0 ? xn0 : xm0, *X1 = side == 0 ? xn1 : xm1, *X2 = side == 0 ? xn2 : xm2;
      X0[c] = X0[c] + fx;
      X1[c] = X1[c] + fy;
      X2[c] = X2[c] + e;
    }
  }
  block_max2(sN, sP, &sc->smax[0], &sc->smax[1]);
}

void launch_interface(const Grid &g, double *const wN[4], double *const wP[4], const double *phi,
                      const double *sx, const double *sy, const int *cut, int cut_cap,
                      double *const xn[3], double *const xm[3], double *ul0, double *ul1,
                      Scalars *sc, cudaStream_t st) {
  // one warp (16 cut cells) per block: the Newton solves are bound by the
  // FP64 lanes of the SMs they occupy, and a few hundred cut cells in
  // larger blocks would occupy a handful of SMs.  cut_cap bounds the cut
  // count (the kernel loops over the device count).
  int blocks = grid_for(2 * cut_cap, 32, 9728);
  launch_k(k_interface, blocks, 32, 0, st, g, wN[0], wN[1], wN[2], wN[3], wP[0], wP[1], wP[2], wP[3],
                                      phi, sx, sy, cut, &sc->n_cut, xn[0], xn[1], xn[2], xm[0],
                                      xm[1], xm[2], ul0, ul1, sc);
  sif_note_launches(1);
}

// the level set's new band values, each also written to the ghost cells
// whose image it is (the values the ghost fill would give them): phi
// changes only through these writes, so its ghost layers stay filled
__global__ void k_band_scatter_phi(Grid g, const int *__restrict__ band, const int *nband,
                                   const double *tmp, double *phi) {
  SIF_TICK();
  int n = *nband;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int a = (c % g.PX) - SIF_GH, b = (c / g.PX) - SIF_GH;
    double v = tmp[idx];
    phi[c] = v;
    if (a >= SIF_GH && a < g.nx - SIF_GH && b >= SIF_GH && b < g.ny - SIF_GH) continue;
    int xs[1 + 2 * SIF_GH], ys[1 + 2 * SIF_GH];
    int nx_ = ghost_preimages(a, g.nx, g.bc[0], g.bc[1], xs);
    int ny_ = ghost_preimages(b, g.ny, g.bc[2], g.bc[3], ys);
    for (int p = 0; p < nx_; p++)
      for (int q = 0; q < ny_; q++)
        if (p || q) phi[gidx(g, xs[p], ys[q])] = v;
  }
}

// ---------------------------------------------------------------------
// level-set advection (Eq. 6) with upwind HJ-WENO5, one RK stage

// WENO5-JS value of five differences with one division: the nonlinear
// weights d_r / t_r (t_r = (eps + b_r)^2) scaled by t0 t1 t2 and the
// candidates' common 1/6 moved into the final division.  Equal to
// weno5_plain up to rounding; weno5_plain where the scaled products leave
// the double range.
__device__ inline double weno5_hj(double v1, double v2, double v3, double v4, double v5,
                                  double eps) {
  double b0 = 13.0 / 12.0 * sqd(v1 - 2.0 * v2 + v3) + 0.25 * sqd(v1 - 4.0 * v2 + 3.0 * v3);
  double b1 = 13.0 / 12.0 * sqd(v2 - 2.0 * v3 + v4) + 0.25 * sqd(v2 - v4);
  double b2 = 13.0 / 12.0 * sqd(v3 - 2.0 * v4 + v5) + 0.25 * sqd(3.0 * v3 - 4.0 * v4 + v5);
  double q0 = 2.0 * v1 - 7.0 * v2 + 11.0 * v3;
  double q1 = -v2 + 5.0 * v3 + 2.0 * v4;
  double q2 = 2.0 * v3 + 5.0 * v4 - v5;
  double t0 = sqd(eps + b0), t1 = sqd(eps + b1), t2 = sqd(eps + b2);
  double u0 = 0.1 * (t1 * t2), u1 = 0.6 * (t0 * t2), u2 = 0.3 * (t0 * t1);
  double r = (u0 * q0 + u1 * q1 + u2 * q2) / (6.0 * (u0 + u1 + u2));
  if (!isfinite(r)) r = weno5_plain(v1, v2, v3, v4, v5, eps);
  return r;
}

// upwind HJ-WENO5 derivative along stride s; inv_h = 1 / h
__device__ inline double hj_deriv(const double *p, int c, int s, double inv_h, bool backward,
                                  double eps) {
  double v[5];
  if (backward) {
#pragma unroll
    for (int r = 0; r < 5; r++) {
      int m = c + (r - 2) * s;
      v[r] = (p[m] - p[m - s]) * inv_h;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 5; r++) {
      int m = c + (2 - r) * s;
      v[r] = (p[m + s] - p[m]) * inv_h;
    }
  }
  return weno5_hj(v[0], v[1], v[2], v[3], v[4], eps);
}

__global__ void k_ls_stage(Grid g, int s, double a, double b, const double *__restrict__ phi,
                           const double *__restrict__ phi0, const double *__restrict__ u0,
                           const double *__restrict__ u1, const int *__restrict__ band,
                           const int *nband, double *tmp, const double *dtp) {
  SIF_TICK();
  int n = *nband;
  double dt = *dtp;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    double u = u0[c], v = u1[c];
    double px = 0.0, py = 0.0;
    if (u != 0.0) px = hj_deriv(phi, c, 1, 1.0 / g.dx, u > 0.0, g.weno_eps);
    if (g.dim == 2 && v != 0.0) py = hj_deriv(phi, c, g.PX, 1.0 / g.dy, v > 0.0, g.weno_eps);
    double L = -(u * px + v * py);
    tmp[idx] = s == 1 ? phi[c] + dt * L : a * phi0[c] + b * (phi[c] + dt * L);
  }
}

void launch_ls_stage(const Grid &g, int s, int rk, double *phi, const double *phi0,
                     const double *ul0, const double *ul1, const int *band, const int *nband,
                     int band_cap, double *tmp, const double *dtp, cudaStream_t st) {
  static const double A2[3] = {0.0, 0.0, 0.5}, B2[3] = {0.0, 1.0, 0.5};
  static const double A3[4] = {0.0, 0.0, 0.75, 1.0 / 3.0}, B3[4] = {0.0, 1.0, 0.25, 2.0 / 3.0};
  double a = rk == 3 ? A3[s] : A2[s], b = rk == 3 ? B3[s] : B2[s];
  int blocks = grid_for(band_cap, 64, 2432);
  // phi's ghost layers are current: every change of phi fills them
  launch_k(k_ls_stage, blocks, 64, 0, st, g, s, a, b, phi, phi0, ul0, ul1, band, nband, tmp, dtp);
  launch_k(k_band_scatter_phi, blocks, 64, 0, st, g, band, nband, tmp, phi);
  sif_note_launches(2);
}

// ---------------------------------------------------------------------
// reinitialisation sweeps over the band and its face neighbours

__device__ inline double grad_est(const double *p, int c, int s, double h) {
  double dm = fabs(p[c] - p[c - s]), dp = fabs(p[c + s] - p[c]);
  double dc = 0.5 * fabs(p[c + s] - p[c - s]);
  return fmax(fmax(dc, dp), dm) / h;
}

__global__ void k_reinit(Grid g, const double *__restrict__ q, const double *__restrict__ z,
                         const int *__restrict__ rext, const int *nrext, double *tmp) {
  SIF_TICK();
  int n = *nrext;
  bool d2 = g.dim == 2;
  double h = g.h;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = rext[idx];
    double s0 = z[c];
    bool pos = s0 >= 0.0;
    bool cut = (z[c - 1] >= 0.0) != pos || (z[c + 1] >= 0.0) != pos;
    if (d2) cut = cut || (z[c - g.PX] >= 0.0) != pos || (z[c + g.PX] >= 0.0) != pos;
    double out = q[c];
    if (cut) {
      double gx = (z[c + 1] - z[c - 1]) / (2.0 * g.dx);
      double gy = d2 ? (z[c + g.PX] - z[c - g.PX]) / (2.0 * g.dy) : 0.0;
      double gm = sqrt(gx * gx + gy * gy);
      if (!(gm > 1e-8)) {
        gx = grad_est(z, c, 1, g.dx);
        gy = d2 ? grad_est(z, c, g.PX, g.dy) : 0.0;
        gm = sqrt(gx * gx + gy * gy);
      }
      double dmin = INFINITY;
      const int nbs[4] = {-1, 1, -g.PX, g.PX};
      for (int e = 0; e < (d2 ? 4 : 2); e++) {
        double zn = z[c + nbs[e]];
        if ((zn >= 0.0) == pos) continue;
        double hh = e < 2 ? g.dx : g.dy;
        double dd = fabs(s0) / (fabs(s0) + fabs(zn)) * hh;
        if (dd < dmin) dmin = dd;
      }
      double D = fabs(s0) / gm;
      if (D > dmin) D = dmin;
      D = pos ? D : -D;
      double sg = pos ? 1.0 : -1.0;
      out = q[c] - 0.5 * (sg * fabs(q[c]) - D);
    } else {
      double S = s0 / sqrt(s0 * s0 + h * h);
      const double idx_ = 1.0 / g.dx, idy_ = 1.0 / g.dy;
      double a = hj_deriv(q, c, 1, idx_, true, g.weno_eps);
      double b = hj_deriv(q, c, 1, idx_, false, g.weno_eps);
      double cc = 0.0, d = 0.0;
      if (d2) {
        cc = hj_deriv(q, c, g.PX, idy_, true, g.weno_eps);
        d = hj_deriv(q, c, g.PX, idy_, false, g.weno_eps);
      }
      double G = -1.0;
      if (s0 > 0.0)
        G = fmax(sqd(fmax(a, 0.0)), sqd(fmin(b, 0.0))) + fmax(sqd(fmax(cc, 0.0)), sqd(fmin(d, 0.0)));
      else if (s0 < 0.0)
        G = fmax(sqd(fmin(a, 0.0)), sqd(fmax(b, 0.0))) + fmax(sqd(fmin(cc, 0.0)), sqd(fmax(d, 0.0)));
      if (G >= 0.0) {
        out = q[c] - 0.5 * h * S * (sqrt(G) - 1.0);
        // no new extremum: a positive value stays at or above its smallest
        // face neighbour, a negative one at or below its largest (the WENO
        // derivatives can overshoot at kinks where the moving band meets
        // the level set outside it)
        double lo = fmin(q[c - 1], q[c + 1]), hi = fmax(q[c - 1], q[c + 1]);
        if (d2) {
          lo = fmin(lo, fmin(q[c - g.PX], q[c + g.PX]));
          hi = fmax(hi, fmax(q[c - g.PX], q[c + g.PX]));
        }
        if (s0 > 0.0 && out < lo) out = lo;
        if (s0 < 0.0 && out > hi) out = hi;
      }
    }
    tmp[idx] = out;
  }
}

void launch_reinit(const Grid &g, double *phi, double *phi0, const int *rext, const int *nrext,
                   int rext_cap, double *tmp, cudaStream_t st) {
  // phi's ghost layers are current (every change of phi fills them), so
  // the copy carries them too
  cudaMemcpyAsync(phi0, phi, sizeof(double) * (size_t)g.PX * g.PY, cudaMemcpyDeviceToDevice, st);
  int blocks = grid_for(rext_cap, 64, 2432);
  for (int it = 0; it < g.reinit_iters; it++) {
    launch_k(k_reinit, blocks, 64, 0, st, g, phi, phi0, rext, nrext, tmp);
    launch_k(k_band_scatter_phi, blocks, 64, 0, st, g, rext, nrext, tmp, phi);
  }
  sif_note_launches(2 * g.reinit_iters);
}

// ---------------------------------------------------------------------
// Eq. 8 (shared) / Eq. 9 (fluid-2 only) correction quantities, in the
// frame of fluid 1, accumulated in the cut cells of this interaction

// X_1, the exchange flux as applied to fluid 1 (with fluid 1's own
// interface pressure): fluid N's planes, or fluid P's negated planes
// negated back, by the cycle's role
__global__ void k_record(int shared, double bw, int fluid2, const int *__restrict__ cut,
                         const int *ncut,
                         const double *__restrict__ n0, const double *__restrict__ n1,
                         const double *__restrict__ n2, const double *__restrict__ m0,
                         const double *__restrict__ m1, const double *__restrict__ m2,
                         double *c0, double *c1, double *c2, const Scalars *sc) {
  SIF_TICK();
  int n = *ncut;
  const bool fN = sc->f1 == 0;
  const double sgn = fN ? 1.0 : -1.0;
  const double *x0 = fN ? n0 : m0, *x1 = fN ? n1 : m1, *x2 = fN ? n2 : m2;
  double dt1 = sc->dt1, dt2 = sc->dt2;
  if (shared == -1) shared = sc->sub == 1;
  else if (shared == -2) shared = sc->last;
  else if (shared == -3) shared = sc->sub == 1 && sc->last;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = cut[idx];
    const double *xs[3] = {x0, x1, x2};
    double *cs[3] = {c0, c1, c2};
    // explicitly rounded products and sums (never contracted into FMAs):
    // with dt1 = dt2 the fluid-1 and fluid-2 records must cancel exactly
    for (int m = 0; m < 3; m++) {
      double xv = __dmul_rn(sgn, xs[m][c]);
      double acc = cs[m][c];
      if (shared) acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(-bw, xv), dt1));
      if (fluid2) acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(bw, xv), dt2));
      cs[m][c] = acc;
    }
  }
}

void launch_record(const Grid &, int shared, const int *cut, int cut_cap, double *const xn[3],
                   double *const xm[3], double *xc0, double *xc1, double *xc2, Scalars *sc,
                   cudaStream_t st, double bw, int fluid2) {
  int blocks = grid_for(cut_cap, 128, 1216);
  launch_k(k_record, blocks, 128, 0, st, shared, bw, fluid2, cut, &sc->n_cut, xn[0], xn[1], xn[2],
                                   xm[0], xm[1], xm[2], xc0, xc1, xc2, sc);
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// Eq. 7: fluid-1 state at the current fluid-2 time

// Eq. 7 over the cells of a band list: every use of the intermediate
// fluid-1 state (mixing, the interaction step's stencil states with fluid 1
// in the band only) reads it inside the band
__global__ void k_interp(Grid g, double *i0, double *i1, double *i2, double *i3,
                         const double *__restrict__ p0, const double *__restrict__ p1,
                         const double *__restrict__ p2, const double *__restrict__ p3,
                         const double *__restrict__ f0, const double *__restrict__ f1,
                         const double *__restrict__ f2, const double *__restrict__ f3,
                         const double *thp, const int *__restrict__ band, const int *nband) {
  SIF_TICK();
  double th = *thp;
  int n = *nband;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int c = band[t];
    i0[c] = (1.0 - th) * p0[c] + th * f0[c];
    i1[c] = (1.0 - th) * p1[c] + th * f1[c];
    i2[c] = (1.0 - th) * p2[c] + th * f2[c];
    i3[c] = (1.0 - th) * p3[c] + th * f3[c];
  }
}

void launch_interp(const Grid &g, double *const qi[4], double *const prev[4],
                   double *const fut[4], const double *thp, const int *band, const int *nband,
                   int band_cap, cudaStream_t st) {
  launch_k(k_interp, grid_for(band_cap, 64, 2432), 64, 0, st, g, qi[0], qi[1], qi[2], qi[3], prev[0],
                                                       prev[1], prev[2], prev[3], fut[0],
                                                       fut[1], fut[2], fut[3], thp, band, nband);
  sif_note_launches(1);
}

// final interfacial flux correction of fluid 1

__global__ void k_correction(Grid g, double *q1, double *q2, double *q3, const double *c0,
                             const double *c1, const double *c2) {
  SIF_TICK();
  int n = g.nx * g.ny;
  double dxdy = g.dx * g.dy;
  // cells without a recorded correction would add exactly zero
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int c = gidx(g, t % g.nx, t / g.nx);
    double a = c0[c], b = c1[c], d = c2[c];
    if (a != 0.0) q1[c] += a / dxdy;
    if (b != 0.0) q2[c] += b / dxdy;
    if (d != 0.0) q3[c] += d / dxdy;
  }
}

void launch_correction(const Grid &g, double *const q[4], const double *xc0, const double *xc1,
                       const double *xc2, cudaStream_t st) {
  int n = g.nx * g.ny;
  launch_k(k_correction, grid_for(n, 256, 152 * 16), 256, 0, st, g, q[1], q[2], q[3], xc0, xc1, xc2);
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// RK3 cycle: the level set at fluid 1's third-stage time

__global__ void k_copy_if(const int *flag, const double *__restrict__ src, double *dst,
                          size_t n) {
  SIF_TICK();
  if (!*flag) return;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

void launch_copy_if(const int *flag, const double *src, double *dst, size_t n, cudaStream_t st) {
  launch_k(k_copy_if, grid_for((int)((n + 3) / 4), 256, 152 * 8), 256, 0, st, flag, src, dst, n);
  sif_note_launches(1);
}

// linear interpolation in time between two kept level sets; a cell where
// they agree keeps its value as it is
__global__ void k_phi_interp(Grid g, double *phi, const double *__restrict__ a,
                             const double *__restrict__ b, const double *thp) {
  SIF_TICK();
  const double th = *thp;
  int n = g.nx * g.ny;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int c = gidx(g, t % g.nx, t / g.nx);
    double va = a[c], vb = b[c];
    phi[c] = va == vb ? va : (1.0 - th) * va + th * vb;
  }
}

void launch_phi_interp(const Grid &g, double *phi, const double *a, const double *b,
                       const double *thp, cudaStream_t st) {
  int n = g.nx * g.ny;
  launch_k(k_phi_interp, grid_for(n, 256, 152 * 8), 256, 0, st, g, phi, a, b, thp);
  sif_note_launches(1);
}

__global__ void k_zero_cut(const int *__restrict__ cut, const int *ncut, double *a0, double *a1,
                           double *a2, double *b0, double *b1, double *b2) {
  SIF_TICK();
  int n = *ncut;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int c = cut[t];
    a0[c] = a1[c] = a2[c] = 0.0;
    b0[c] = b1[c] = b2[c] = 0.0;
  }
}

void launch_zero_cut(const Grid &, double *const xn[3], double *const xm[3], const int *cut,
                     const int *ncut, int cut_cap, cudaStream_t st) {
  launch_k(k_zero_cut, grid_for(cut_cap, 128, 1216), 128, 0, st, cut, ncut, xn[0], xn[1], xn[2], xm[0],
                                                          xm[1], xm[2]);
  sif_note_launches(1);
}

// ---------------------------------------------------------------------
// conserved totals: fixed-order per-row partial sums, then a fixed-order
// sum of the partials (deterministic)

struct Planes8 {
  const double *p[8];
};

__global__ void k_integrals_rows(Grid g, Planes8 planes, double *partial) {
  SIF_TICK();
  // blockIdx.y: plane (8), blockIdx.x: group of rows; one warp per row
  int pl = blockIdx.y;
  const double *a = planes.p[pl];
  int rows_per_block = blockDim.x / 32;
  int j = blockIdx.x * rows_per_block + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  double s = 0.0;
  if (j < g.ny)
    for (int i = lane; i < g.nx; i += 32) s += a[gidx(g, i, j)];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0 && j < g.ny) partial[(size_t)pl * g.ny + j] = s;
}

__global__ void k_integrals_final(Grid g, const double *partial, double *out) {
  SIF_TICK();
  int pl = threadIdx.x;
  if (pl >= 8) return;
  double s = 0.0;
  for (int j = 0; j < g.ny; j++) s += partial[(size_t)pl * g.ny + j];
  out[pl] = s * (g.dx * g.dy);
}

void launch_integrals(const Grid &g, double *const qN[4], double *const qP[4], double *partial,
                      int, double *out, cudaStream_t st) {
  Planes8 tab = {{qN[0], qN[1], qN[2], qN[3], qP[0], qP[1], qP[2], qP[3]}};
  dim3 grid((g.ny + 7) / 8, 8);
  launch_k(k_integrals_rows, grid, 256, 0, st, g, tab, partial);
  launch_k(k_integrals_final, 1, 32, 0, st, g, partial, out);
  sif_note_launches(2);
}

// ---------------------------------------------------------------------
// device-side scheduler of the single- and multi-time-step methods

// after a sub-step's length is known: does it reach fluid 1's third-stage
// time (t^n + dt1/2) of an RK3 cycle?  Then its level set at the start is
// kept.  Also whether the cycle has a single sub-step.
__device__ void sched_snap_a(Scalars *sc) {
  sc->single = sc->sub == 1 && sc->last;
  sc->snap_a = !sc->have_a && (0.5 * sc->dt1 < sc->t2 + sc->dt2 || sc->last);
  if (sc->snap_a) {
    sc->have_a = 1;
    sc->ta = sc->t2;
  }
}

__global__ void k_sched(int op, Scalars *sc, double cfl, double thr, int force1) {
  SIF_TICK();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sm0 = ull_as_double(sc->smax[0]), sm1 = ull_as_double(sc->smax[1]);
  double dtk[2] = {sm0 > 0.0 ? cfl / sm0 : INFINITY, sm1 > 0.0 ? cfl / sm1 : INFINITY};
  switch (op) {
    case SCHED_RESET_MAX:
      sc->smax[0] = sc->smax[1] = 0ull;
      sc->lf[0][0] = sc->lf[0][1] = sc->lf[1][0] = sc->lf[1][1] = 0ull;
      break;
    case SCHED_SINGLE_DT: {
      double dt = fmin(dtk[0], dtk[1]);
      if (sc->t_end > 0.0 && sc->t + dt > sc->t_end) dt = sc->t_end - sc->t;
      sc->dt = dt;
      break;
    }
    case SCHED_CYCLE_BEGIN: {
      for (int k = 0; k < 2; k++)
        if (sc->t_end > 0.0 && sc->t + dtk[k] > sc->t_end) dtk[k] = sc->t_end - sc->t;
      int f1 = dtk[1] > dtk[0] ? 1 : 0;
      double dt1 = dtk[f1], dt2 = dtk[1 - f1];
      double nraw = dt1 / dt2;
      sc->f1 = f1;
      sc->n_raw = nraw;
      sc->dtk_raw[0] = dtk[0];
      sc->dtk_raw[1] = dtk[1];
      int mode = 1;
      if (force1) {
        dt1 = dt2;
      } else {
        if (isfinite(dt1)) {
          double fl = floor(nraw);
          if (nraw - fl < thr) dt1 = fl * dt2;
        }
        if (!isfinite(dt1) || dt1 <= dt2) mode = 0;
      }
      sc->mode = mode;
      if (mode == 0) {
        sc->dt = dt2;
        sc->dt1 = dt2;
        sc->dt2 = dt2;
        sc->n_used = 1.0;
      } else {
        sc->dt1 = dt1;
        sc->dt2 = dt2;
        sc->n_used = dt1 / dt2;
      }
      sc->t2 = 0.0;
      sc->sub = 0;
      sc->last = 0;
      sc->single = 0;
      sc->have_a = sc->have_b = sc->snap_a = sc->snap_b = 0;
      sc->ta = sc->tb = 0.0;
      sc->dt2_first = sc->dt2;
      break;
    }
    case SCHED_SUBSTEP:
      sc->dt2 = dtk[sc->f1 == 0 ? 1 : 0];
      // fall through to the last-substep test
    case SCHED_FIRST_SUB: {
      sc->sub += 1;
      double dt1 = sc->dt1, t2 = sc->t2, dt2 = sc->dt2;
      int last = (dt1 - t2) <= dt2 * (1.0 + 1e-12);
      if (last) dt2 = dt1 - t2;
      sc->dt2 = dt2;
      sc->last = last;
      sc->theta = last ? 1.0 : (t2 + dt2) / dt1;
      sched_snap_a(sc);
      break;
    }
    case SCHED_ADVANCE:
      sc->t2 = sc->t2 + sc->dt2;
      sc->theta = sc->t2 / sc->dt1;
      break;
    case SCHED_DT2:
      sc->dt2 = dtk[sc->f1 == 0 ? 1 : 0];
      break;
    case SCHED_LAST: {
      sc->sub += 1;
      double dt1 = sc->dt1, t2 = sc->t2, dt2 = sc->dt2;
      int last = (dt1 - t2) <= dt2 * (1.0 + 1e-12);
      if (last) dt2 = dt1 - t2;
      sc->dt2 = dt2;
      sc->last = last;
      sc->theta = last ? 1.0 : (t2 + dt2) / dt1;
      sched_snap_a(sc);
      break;
    }
    case SCHED_THETA3:
      sc->theta = (sc->t2 + 0.5 * sc->dt2) / sc->dt1;
      break;
    case SCHED_SNAPB:
      // the sub-step that reached fluid 1's third-stage time ends here
      sc->snap_b = sc->have_a && !sc->have_b;
      if (sc->snap_b) {
        sc->have_b = 1;
        sc->tb = sc->t2 + sc->dt2;
      }
      break;
    case SCHED_W3:
      sc->theta = (0.5 * sc->dt1 - sc->ta) / (sc->tb - sc->ta);
      break;
    case SCHED_T_SINGLE:
      sc->t = sc->t + sc->dt;
      break;
    case SCHED_T_CYCLE:
      sc->t = sc->t + sc->dt1;
      break;
  }
}

// graph conditions from the scheduler's decisions
__global__ void k_cond(int op, Scalars *sc, cudaGraphConditionalHandle h0,
                       cudaGraphConditionalHandle h1, cudaGraphConditionalHandle h2, int max_sub) {
  SIF_TICK();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  switch (op) {
    case COND_CYCLE:
      cudaGraphSetConditional(h0, sc->mode == 0 ? 1u : 0u);
      cudaGraphSetConditional(h1, (sc->mode == 1 && sc->f1 == 0) ? 1u : 0u);
      cudaGraphSetConditional(h2, (sc->mode == 1 && sc->f1 == 1) ? 1u : 0u);
      break;
    case COND_NOT_FIRST:
      cudaGraphSetConditional(h0, sc->sub > 0 ? 1u : 0u);
      break;
    case COND_LAST:
      cudaGraphSetConditional(h0, sc->last ? 1u : 0u);
      cudaGraphSetConditional(h1, sc->last ? 0u : 1u);
      break;
    case COND_SINGLE:
      cudaGraphSetConditional(h0, sc->single ? 1u : 0u);
      cudaGraphSetConditional(h1, sc->single ? 0u : 1u);
      break;
    case COND_LAST_ONLY:
      cudaGraphSetConditional(h0, sc->last ? 1u : 0u);
      break;
    case COND_SINGLE_ONLY:
      cudaGraphSetConditional(h0, sc->single ? 1u : 0u);
      break;
    case COND_MULTI_ONLY:
      cudaGraphSetConditional(h0, sc->single ? 0u : 1u);
      break;
    case COND_LOOP: {
      // stop after the last sub-step, on a device error, or when the
      // sub-step count or step size has gone wrong
      bool go = !sc->last && sc->err == 0 && sc->sub < max_sub && sc->dt2 > 0.0;
      // the sub-step limit stops an unfinished cycle: an error, not an end
      if (!sc->last && sc->err == 0 && sc->sub >= max_sub) sc->err |= DERR_TIMEOUT;
      cudaGraphSetConditional(h0, go ? 1u : 0u);
      break;
    }
  }
}

void launch_cond(int op, Scalars *sc, cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1,
                 cudaGraphConditionalHandle h2, int max_sub, cudaStream_t st) {
  launch_k(k_cond, 1, 32, 0, st, op, sc, h0, h1, h2, max_sub);
}

void launch_sched(int op, Scalars *sc, double cfl, double thr, int force1, cudaStream_t st) {
  launch_k(k_sched, 1, 32, 0, st, op, sc, cfl, thr, force1);
  sif_note_launches(1);
}

SIF_TU_LAUNCH_READER(band)
