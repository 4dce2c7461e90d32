// adjoint.cu -- transposed kernels of the cut-cell right-hand side for the
// discrete adjoint of the single-time-step RK2 step with its schedule
// frozen (dt, Lax-Friedrichs speeds and level sets of both stages given).
//
// With the geometry fixed, the right-hand side L(Q) of both fluids (Eq. 2)
// is a composition of differentiable maps: primitive recovery at real
// cells, linear extension into the band, ghost fill, LF-split fluxes
// reconstructed by WENO5 (nonlinear weights included), the aperture-
// weighted divergence, and the interface exchange X from the exact
// two-material Riemann problem.  Its transpose runs here in reverse order:
//   face coefficients  (divergence^T, WENO5^T per face and component)
//   gather             (split-flux Jacobian^T per cell, both directions)
//   ghost^T            (ghost adjoints back to the cells they copy)
//   interface^T        (implicit-function theorem on the Riemann equation)
//   extension^T        (the Jacobi sweeps transposed, band-indexed)
//   primitive^T        (at real cells: above the sliver threshold and, for
//                       cut cells, holding a physical state), combined
//                       with the RK coefficients.
// Nothing here takes a branch that depends on rounding: every decision
// (real cells, targets, Riemann wave types at the converged state) is the
// forward's, so FMA contraction is allowed.
#include "sif_internal.cuh"

static int blocks_for(long long n, int per = 256, int cap = 8192) {
  long long b = (n + per - 1) / per;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

__device__ inline double lf_value(const unsigned long long *lf, int k, int d) {
  return ull_as_double(lf[k * 2 + d]);
}

// ---------------------------------------------------------------------
// WENO5-JS and its derivative with respect to the five stencil values

// The divisions are reciprocals (Newton's iteration from the device's
// approximate reciprocal, within an ulp of IEEE division) times the
// numerators, and the constant 1/6 a product: the derivative is the same
// function, rounded differently.
__device__ inline void weno5_grad(const double v[5], double eps, double g[5]) {
  constexpr double s6 = 1.0 / 6.0;
  const double q0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) * s6;
  const double q1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) * s6;
  const double q2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) * s6;
  // smoothness indicators b_i = 13/12 s_i^2 + 1/4 t_i^2
  const double s0 = v[0] - 2.0 * v[1] + v[2], t0 = v[0] - 4.0 * v[1] + 3.0 * v[2];
  const double s1 = v[1] - 2.0 * v[2] + v[3], t1 = v[1] - v[3];
  const double s2 = v[2] - 2.0 * v[3] + v[4], t2 = 3.0 * v[2] - 4.0 * v[3] + v[4];
  const double b0 = 13.0 / 12.0 * s0 * s0 + 0.25 * t0 * t0;
  const double b1 = 13.0 / 12.0 * s1 * s1 + 0.25 * t1 * t1;
  const double b2 = 13.0 / 12.0 * s2 * s2 + 0.25 * t2 * t2;
  const double i0 = recip_newton3(eps + b0), i1 = recip_newton3(eps + b1),
               i2 = recip_newton3(eps + b2);
  const double a0 = 0.1 * i0 * i0, a1 = 0.6 * i1 * i1, a2 = 0.3 * i2 * i2;
  const double iS = recip_newton3(a0 + a1 + a2);
  // normalised weights w_i = a_i / S and the reconstruction r
  const double w0 = a0 * iS, w1 = a1 * iS, w2 = a2 * iS;
  const double r = w0 * q0 + w1 * q1 + w2 * q2;
  // d r = sum_i (w_i dq_i + (q_i - r) da_i / S) with da_i = -2 a_i / e_i db_i
  const double c0 = -2.0 * w0 * i0 * (q0 - r), c1 = -2.0 * w1 * i1 * (q1 - r),
               c2 = -2.0 * w2 * i2 * (q2 - r);
  // db_i / dv = 13/6 s_i ds_i + 1/2 t_i dt_i
  const double u0 = 13.0 / 6.0 * s0, z0 = 0.5 * t0;
  const double u1 = 13.0 / 6.0 * s1, z1 = 0.5 * t1;
  const double u2 = 13.0 / 6.0 * s2, z2 = 0.5 * t2;
  const double d0[5] = {u0 + z0, -2.0 * u0 - 4.0 * z0, u0 + 3.0 * z0, 0.0, 0.0};
  const double d1[5] = {0.0, u1 + z1, -2.0 * u1, u1 - z1, 0.0};
  const double d2[5] = {0.0, 0.0, u2 + 3.0 * z2, -2.0 * u2 - 4.0 * z2, u2 + z2};
  const double dq0[5] = {2.0 / 6.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0};
  const double dq1[5] = {0.0, -1.0 / 6.0, 5.0 / 6.0, 2.0 / 6.0, 0.0};
  const double dq2[5] = {0.0, 0.0, 2.0 / 6.0, 5.0 / 6.0, -1.0 / 6.0};
#pragma unroll
  for (int k = 0; k < 5; k++)
    g[k] = w0 * dq0[k] + w1 * dq1[k] + w2 * dq2[k] + c0 * d0[k] + c1 * d1[k] + c2 * d2[k];
}

// LF split fluxes fp = (F + a U)/2, fm = (F - a U)/2 of one primitive state
// (ig1 = 1 / (gamma - 1))
__device__ inline void split_state(double rho, double u, double v, double p, double g, double pi,
                                   double ig1, int d, double a, double fp[4], double fm[4]) {
  double E = (p + g * pi) * ig1 + 0.5 * rho * (u * u + v * v);
  double U[4] = {rho, rho * u, rho * v, E};
  double vn = d == 0 ? u : v;
  double F[4] = {rho * vn, rho * u * vn, rho * v * vn, vn * (E + p)};
  F[1 + d] += p;
#pragma unroll
  for (int m = 0; m < 4; m++) {
    fp[m] = 0.5 * (F[m] + a * U[m]);
    fm[m] = 0.5 * (F[m] - a * U[m]);
  }
}

// ---------------------------------------------------------------------
// 1. face coefficients: for every face of direction d with fluid-k
// aperture A, lamF = A * scale * (mu_right - mu_left) / h, and the WENO5
// derivative of both reconstructions weighted by lamF:
//   G[r*4+m]      -> split flux fp of cell c + (r-3)s, r = 0..4
//   G[20 + r*4+m] -> split flux fm of cell c + (2-r)s, r = 0..4
// The split fluxes of every cell the faces read (ghost layers included)
// are computed once per (fluid, direction) into SP (fp then fm, four
// planes each); the face kernel then takes one (face, component) per
// thread.

struct Planes4 {
  double *p[4];
};
struct Planes8 {
  double *p[8];
};
struct Planes40 {
  double *p[40];
};

// plane base + m of a parameter array, m in 0..3 chosen without indexing
// the parameter array dynamically (which would copy it to local memory)
template <class P>
__device__ __forceinline__ double *plane_m(const P &pl, int base, int m) {
  return m == 0 ? pl.p[base] : m == 1 ? pl.p[base + 1] : m == 2 ? pl.p[base + 2] : pl.p[base + 3];
}

__global__ void k_adj_split(Grid g, int k, int d, Planes4 W, const unsigned long long *lf,
                            Planes8 SP) {
  SIF_TICK();
  // cells -3 .. n+2 along d, 0 .. n-1 across
  const int ncx = d == 0 ? g.nx + 2 * SIF_GH : g.nx;
  const int ncy = d == 0 ? g.ny : g.ny + 2 * SIF_GH;
  const int ox = d == 0 ? -SIF_GH : 0, oy = d == 0 ? 0 : -SIF_GH;
  const long long n = (long long)ncx * ncy;
  const double a = lf_value(lf, k, d);
  const double gm = g.gamma[k], pi = g.pinf[k], ig1 = 1.0 / (gm - 1.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = gidx(g, (int)(t % ncx) + ox, (int)(t / ncx) + oy);
    double fp[4], fm[4];
    split_state(W.p[0][c], W.p[1][c], W.p[2][c], W.p[3][c], gm, pi, ig1, d, a, fp, fm);
#pragma unroll
    for (int m = 0; m < 4; m++) {
      SP.p[m][c] = fp[m];
      SP.p[4 + m][c] = fm[m];
    }
  }
}

__global__ void k_adj_face(Grid g, int k, int d, Planes8 SP, const double *__restrict__ aperture,
                           Planes4 mu, const double *dtp, double fac, Planes40 G) {
  SIF_TICK();
  const int nfx = d == 0 ? g.nx + 1 : g.nx;
  const int nfy = d == 0 ? g.ny : g.ny + 1;
  const long long nf = (long long)nfx * nfy;
  const int s = d == 0 ? 1 : g.PX;
  const double ih = 1.0 / (d == 0 ? g.dx : g.dy);
  const double scale = fac * *dtp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 4 * nf;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / nf);
    const long long f = t % nf;
    const int i = (int)(f % nfx), j = (int)(f / nfx);
    const int c = gidx(g, i, j);
    const double ap = aperture[c];
    const double A = k == 1 ? ap : 1.0 - ap;
    // a face closed to fluid k contributes nothing: its coefficients are
    // neither written here nor read by the gather
    if (A == 0.0) continue;
    const bool has_r = d == 0 ? i < g.nx : j < g.ny;
    const bool has_l = d == 0 ? i > 0 : j > 0;
    const double *mum = plane_m(mu, 0, m);
    const double r_ = has_r ? mum[c] : 0.0, l_ = has_l ? mum[c - s] : 0.0;
    const double lF = A * scale * (r_ - l_) * ih;
    const double *fp = plane_m(SP, 0, m), *fm = plane_m(SP, 4, m);
    const double vp[5] = {fp[c - 3 * s], fp[c - 2 * s], fp[c - s], fp[c], fp[c + s]};
    const double vm[5] = {fm[c + 2 * s], fm[c + s], fm[c], fm[c - s], fm[c - 2 * s]};
    double gp[5], gq[5];
    weno5_grad(vp, g.weno_eps, gp);
    weno5_grad(vm, g.weno_eps, gq);
#pragma unroll
    for (int r = 0; r < 5; r++) {
      plane_m(G, r * 4, m)[c] = lF * gp[r];
      plane_m(G, 20 + r * 4, m)[c] = lF * gq[r];
    }
  }
}

// transpose of the split flux at one cell: lam_fp, lam_fm -> primitive adjoint
__device__ inline void split_T(double rho, double u, double v, double p, double g, double pi,
                               int d, double a, const double sp[4], const double sm[4],
                               double out[4]) {
  double E = (p + g * pi) / (g - 1.0) + 0.5 * rho * (u * u + v * v);
  double ke = 0.5 * (u * u + v * v);
  double lF[4], lU[4];
#pragma unroll
  for (int m = 0; m < 4; m++) {
    lF[m] = 0.5 * (sp[m] + sm[m]);
    lU[m] = 0.5 * a * (sp[m] - sm[m]);
  }
  // U = (rho, rho u, rho v, E)
  double gr = lU[0] + lU[1] * u + lU[2] * v + lU[3] * ke;
  double gu = lU[1] * rho + lU[3] * rho * u;
  double gv = lU[2] * rho + lU[3] * rho * v;
  double gp = lU[3] / (g - 1.0);
  double h1 = 1.0 / (g - 1.0) + 1.0;
  if (d == 0) {
    gr += lF[0] * u + lF[1] * u * u + lF[2] * u * v + lF[3] * u * ke;
    gu += lF[0] * rho + lF[1] * 2.0 * rho * u + lF[2] * rho * v + lF[3] * (E + p + rho * u * u);
    gv += lF[2] * rho * u + lF[3] * rho * u * v;
    gp += lF[1] + lF[3] * u * h1;
  } else {
    gr += lF[0] * v + lF[1] * u * v + lF[2] * v * v + lF[3] * v * ke;
    gu += lF[1] * rho * v + lF[3] * rho * u * v;
    gv += lF[0] * rho + lF[1] * rho * u + lF[2] * 2.0 * rho * v + lF[3] * (E + p + rho * v * v);
    gp += lF[2] + lF[3] * v * h1;
  }
  out[0] = gr;
  out[1] = gu;
  out[2] = gv;
  out[3] = gp;
}

// whether the face at index f is open to fluid k (P-aperture stored)
__device__ inline bool open_face(const double *aperture, int k, int f) {
  double ap = aperture[f];
  return (k == 1 ? ap : 1.0 - ap) != 0.0;
}

// 2. gather: every cell whose split fluxes enter a face of direction d
// (ghost cells included) collects its coefficients and adds the
// transposed split-flux Jacobian to the stencil-state adjoint lw
__global__ void k_adj_gather(Grid g, int k, int d, Planes4 W, const double *__restrict__ aperture,
                             const unsigned long long *lf, Planes40 G, Planes4 lw) {
  SIF_TICK();
  const int ncx = d == 0 ? g.nx + 2 * SIF_GH : g.nx;
  const int ncy = d == 0 ? g.ny : g.ny + 2 * SIF_GH;
  const int ox = d == 0 ? -SIF_GH : 0, oy = d == 0 ? 0 : -SIF_GH;
  const long long n = (long long)ncx * ncy;
  const int s = d == 0 ? 1 : g.PX;
  const int nfaces = d == 0 ? g.nx : g.ny;  // faces 0 .. nfaces along d
  const double a = lf_value(lf, k, d);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % ncx) + ox, j = (int)(t / ncx) + oy;
    int c = gidx(g, i, j);
    int pos = d == 0 ? i : j;
    double sp[4] = {0.0, 0.0, 0.0, 0.0}, sm[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int r = 0; r < 5; r++) {
      int fpos = pos + 3 - r;  // face whose fp stencil holds this cell at r
      if (fpos >= 0 && fpos <= nfaces) {
        int f = c + (3 - r) * s;
        if (open_face(aperture, k, f)) {
#pragma unroll
          for (int m = 0; m < 4; m++) sp[m] += G.p[r * 4 + m][f];
        }
      }
      int fneg = pos + r - 2;  // face whose fm stencil holds this cell at r
      if (fneg >= 0 && fneg <= nfaces) {
        int f = c + (r - 2) * s;
        if (open_face(aperture, k, f)) {
#pragma unroll
          for (int m = 0; m < 4; m++) sm[m] += G.p[20 + r * 4 + m][f];
        }
      }
    }
    double out[4];
    split_T(W.p[0][c], W.p[1][c], W.p[2][c], W.p[3][c], g.gamma[k], g.pinf[k], d, a, sp, sm, out);
#pragma unroll
    for (int m = 0; m < 4; m++) lw.p[m][c] += out[m];
  }
}

// 3. ghost^T: each interior cell collects the adjoints of the ghost cells
// that were copied from it (with the sign flip of the wall-normal velocity
// at reflective walls)
__device__ inline int ghost_src(int bc, int m, int n, bool low) {
  if (bc == SIF_BC_REFLECT) return low ? m : n - 1 - m;
  if (bc == SIF_BC_PERIODIC) return low ? n - 1 - m : m;
  return low ? 0 : n - 1;
}

__global__ void k_adj_ghost(Grid g, Planes8 lw) {
  SIF_TICK();
  const int vel[4] = {0, 1, 2, 0};
  const long long n = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % g.nx), j = (int)(t / g.nx);
    bool nearx = i < SIF_GH || i >= g.nx - SIF_GH || g.bc[0] == SIF_BC_PERIODIC;
    bool neary = g.dim == 2 && (j < SIF_GH || j >= g.ny - SIF_GH || g.bc[2] == SIF_BC_PERIODIC);
    if (!nearx && !neary) continue;
    int c = gidx(g, i, j);
    for (int q = 0; q < 8; q++) {
      int m = q & 3;
      double acc = 0.0;
      for (int mm = 0; mm < SIF_GH; mm++) {
        double sl = (vel[m] == 1 && g.bc[0] == SIF_BC_REFLECT) ? -1.0 : 1.0;
        double sr = (vel[m] == 1 && g.bc[1] == SIF_BC_REFLECT) ? -1.0 : 1.0;
        if (ghost_src(g.bc[0], mm, g.nx, true) == i) acc += sl * lw.p[q][gidx(g, -1 - mm, j)];
        if (ghost_src(g.bc[1], mm, g.nx, false) == i) acc += sr * lw.p[q][gidx(g, g.nx + mm, j)];
        if (g.dim == 2) {
          double sb = (vel[m] == 2 && g.bc[2] == SIF_BC_REFLECT) ? -1.0 : 1.0;
          double st = (vel[m] == 2 && g.bc[3] == SIF_BC_REFLECT) ? -1.0 : 1.0;
          if (ghost_src(g.bc[2], mm, g.ny, true) == j) acc += sb * lw.p[q][gidx(g, i, -1 - mm)];
          if (ghost_src(g.bc[3], mm, g.ny, false) == j) acc += st * lw.p[q][gidx(g, i, g.ny + mm)];
        }
      }
      lw.p[q][c] += acc;
    }
  }
}

// ---------------------------------------------------------------------
// 4. interface^T: X_N = (-p* Sx, -p* Sy, -p* u* |S|) enters L_N with
// +1/(dx dy) and L_P with -1/(dx dy); p*, u* solve
// f_L(p) + f_R(p) + u_R - u_L = 0 and u* = (u_L + u_R)/2 + (f_R - f_L)/2

// side function and its partials with respect to p, rho and the side
// pressure, at the converged p
__device__ inline void side_partials(double p, double rho, double pk, double g, double pi,
                                     double &f, double &fp, double &fr, double &fk) {
  double P = pk + pi, Pp = p + pi;
  double ck = sqrt(g * P / rho);
  if (p > pk) {
    double A = 2.0 / ((g + 1.0) * rho);
    double B = (g - 1.0) / (g + 1.0) * P;
    double qr = sqrt(A / (Pp + B));
    f = (p - pk) * qr;
    fp = qr * (1.0 - 0.5 * (p - pk) / (Pp + B));
    fk = -qr - 0.5 * (p - pk) * qr / (Pp + B) * (g - 1.0) / (g + 1.0);
  } else {
    double r = Pp / P;
    double re = pos_pow(r, (g - 1.0) / (2.0 * g));
    f = 2.0 * ck / (g - 1.0) * (re - 1.0);
    fp = re / (r * rho * ck);
    fk = f / (2.0 * P) - ck * re / (g * P);
  }
  fr = -f / (2.0 * rho);
}

__global__ void k_adj_interface(Grid g, Planes8 W, const double *__restrict__ phi,
                                const double *__restrict__ sx, const double *__restrict__ sy,
                                const int *__restrict__ cut, const int *ncut, Planes8 mu,
                                const double *dtp, double fac, Planes8 lw) {
  SIF_TICK();
  const int n = *ncut;
  const double scale = fac * *dtp / (g.dx * g.dy);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = cut[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    double Sx = sx[c], Sy = sy[c];
    double Sm = sqrt(Sx * Sx + Sy * Sy);
    double nxv, nyv;
    unit_normal(g, phi, i, j, nxv, nyv);
    if (nxv == 0.0 && nyv == 0.0) {
      nxv = Sx / Sm;
      nyv = Sy / Sm;
    }
    double rl = W.p[0][c], ul = W.p[1][c] * nxv + W.p[2][c] * nyv, pl = W.p[3][c];
    double rr = W.p[4][c], ur = W.p[5][c] * nxv + W.p[6][c] * nyv, pr = W.p[7][c];
    double gl = g.gamma[0], pil = g.pinf[0], gr = g.gamma[1], pir = g.pinf[1];
    double ps, us, csl, csr;
    riemann_solve(rl, ul, pl, gl, pil, rr, ur, pr, gr, pir, ps, us, csl, csr);
    double lx0 = scale * (mu.p[1][c] - mu.p[5][c]);
    double lx1 = scale * (mu.p[2][c] - mu.p[6][c]);
    double lx2 = scale * (mu.p[3][c] - mu.p[7][c]);
    double lam_p = -Sx * lx0 - Sy * lx1 - us * Sm * lx2;
    double lam_u = -ps * Sm * lx2;
    double fL, fpL, frL, fkL, fR, fpR, frR, fkR;
    side_partials(ps, rl, pl, gl, pil, fL, fpL, frL, fkL);
    side_partials(ps, rr, pr, gr, pir, fR, fpR, frR, fkR);
    double lp = lam_p + lam_u * 0.5 * (fpR - fpL);
    double kappa = lp / (fpL + fpR);
    double gL0 = -0.5 * lam_u * frL - kappa * frL;
    double gL1 = 0.5 * lam_u + kappa;
    double gL2 = -0.5 * lam_u * fkL - kappa * fkL;
    double gR0 = 0.5 * lam_u * frR - kappa * frR;
    double gR1 = 0.5 * lam_u - kappa;
    double gR2 = 0.5 * lam_u * fkR - kappa * fkR;
    lw.p[0][c] += gL0;
    lw.p[1][c] += gL1 * nxv;
    lw.p[2][c] += gL1 * nyv;
    lw.p[3][c] += gL2;
    lw.p[4][c] += gR0;
    lw.p[5][c] += gR1 * nxv;
    lw.p[6][c] += gR1 * nyv;
    lw.p[7][c] += gR2;
  }
}

// ---------------------------------------------------------------------
// 5. extension^T on the band (blockIdx.y = fluid): a target's value was
// the weighted mean of its upwind neighbours, every other cell kept its
// own, so a transposed sweep keeps the adjoint of non-targets and hands
// each target's adjoint to its neighbours (gathered from the four face
// neighbours; neighbours outside the band accumulate in the planes)

__global__ void k_adj_ext_load(Planes8 lw, const int *__restrict__ band, const int *nband,
                               int cap, double *buf) {
  SIF_TICK();
  const int n = *nband;
  const int k = blockIdx.y;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
#pragma unroll
    for (int m = 0; m < 4; m++) buf[(size_t)(k * 4 + m) * cap + idx] = lw.p[k * 4 + m][c];
  }
}

__global__ void k_adj_ext_sweep(Grid g, const ExtPlan *__restrict__ plan, int cap,
                                const int *__restrict__ band, const int *nband,
                                const int *__restrict__ map, const double *src, double *dst,
                                Planes8 lw) {
  SIF_TICK();
  const int n = *nband;
  const int k = blockIdx.y;
  const ExtPlan *P = plan + (size_t)k * cap;
  const double *in = src + (size_t)k * 4 * cap;
  double *out = dst + (size_t)k * 4 * cap;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
    int i = (c % g.PX) - SIF_GH, j = (c / g.PX) - SIF_GH;
    ExtPlan pl = P[idx];
    bool keeps = pl.cx < 0 && pl.cy < 0;
    double v[4];
#pragma unroll
    for (int m = 0; m < 4; m++) v[m] = keeps ? in[(size_t)m * cap + idx] : 0.0;
    const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    for (int e = 0; e < 4; e++) {
      if (g.dim == 1 && e >= 2) break;
      if (!inside(g, i + di[e], j + dj[e])) continue;
      int t = gidx(g, i + di[e], j + dj[e]);
      int pt = map[t];
      if (pt < 0) continue;
      ExtPlan q = P[pt];
      double w = (q.cx == c ? q.wx : 0.0) + (q.cy == c ? q.wy : 0.0);
      if (w == 0.0) continue;
#pragma unroll
      for (int m = 0; m < 4; m++) v[m] += w * in[(size_t)m * cap + pt];
    }
#pragma unroll
    for (int m = 0; m < 4; m++) out[(size_t)m * cap + idx] = v[m];
    // upwind neighbours outside the band keep their values through every
    // sweep: their adjoint accumulates in the planes
    if (pl.cx >= 0 && pl.bx < 0)
      for (int m = 0; m < 4; m++)
        atomicAdd(&lw.p[k * 4 + m][pl.cx], pl.wx * in[(size_t)m * cap + idx]);
    if (pl.cy >= 0 && pl.by < 0)
      for (int m = 0; m < 4; m++)
        atomicAdd(&lw.p[k * 4 + m][pl.cy], pl.wy * in[(size_t)m * cap + idx]);
  }
}

__global__ void k_adj_ext_store(Planes8 lw, const int *__restrict__ band, const int *nband,
                                int cap, const double *buf) {
  SIF_TICK();
  const int n = *nband;
  const int k = blockIdx.y;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    int c = band[idx];
#pragma unroll
    for (int m = 0; m < 4; m++) lw.p[k * 4 + m][c] = buf[(size_t)(k * 4 + m) * cap + idx];
  }
}

// ---------------------------------------------------------------------
// 6. primitive^T at real cells, combined: out = ca A + cb B + lq
// (A, B may be null; out may alias either)

__global__ void k_adj_prim(Grid g, Planes8 W, const double *__restrict__ alpha,
                           const unsigned char *__restrict__ ns0,
                           const unsigned char *__restrict__ ns1, Planes8 lw, Planes8 out,
                           Planes8 A, double ca, Planes8 B, double cb) {
  SIF_TICK();
  const long long n = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % g.nx), j = (int)(t / g.nx);
    int c = gidx(g, i, j);
    for (int k = 0; k < 2; k++) {
      double a = vol_k(alpha, k, c);
      double lq[4] = {0.0, 0.0, 0.0, 0.0};
      if (a > SIF_ALPHA_REAL && !(k == 0 ? ns0 : ns1)[c]) {
        double gm1 = g.gamma[k] - 1.0;
        double rho = W.p[k * 4][c], u = W.p[k * 4 + 1][c], v = W.p[k * 4 + 2][c];
        double lr = lw.p[k * 4][c], lu = lw.p[k * 4 + 1][c], lv = lw.p[k * 4 + 2][c],
               lp = lw.p[k * 4 + 3][c];
        double m0 = a * rho;
        lq[0] = lr / a - (lu * u + lv * v) / m0 + lp * gm1 * 0.5 * (u * u + v * v) / a;
        lq[1] = lu / m0 - lp * gm1 * u / a;
        lq[2] = lv / m0 - lp * gm1 * v / a;
        lq[3] = lp * gm1 / a;
      }
#pragma unroll
      for (int m = 0; m < 4; m++) {
        int q = k * 4 + m;
        double r = lq[m];
        if (A.p[q]) r += ca * A.p[q][c];
        if (B.p[q]) r += cb * B.p[q][c];
        out.p[q][c] = r;
      }
    }
  }
}

// transpose of the initialisation's conversion alpha_k U(prim) (before
// its mixing): lam (adjoint of alpha U, mixing already transposed) ->
// adjoint of the primitive fields
__global__ void k_adj_init(Grid g, Planes8 prim, const double *__restrict__ alpha, Planes8 lam,
                           Planes8 out) {
  SIF_TICK();
  const long long n = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % g.nx), j = (int)(t / g.nx);
    int c = gidx(g, i, j);
    for (int k = 0; k < 2; k++) {
      double a = vol_k(alpha, k, c);
      double rho = prim.p[k * 4][c], u = prim.p[k * 4 + 1][c], v = prim.p[k * 4 + 2][c];
      double l0 = lam.p[k * 4][c], l1 = lam.p[k * 4 + 1][c], l2 = lam.p[k * 4 + 2][c],
             l3 = lam.p[k * 4 + 3][c];
      out.p[k * 4][c] = a * (l0 + l1 * u + l2 * v + l3 * 0.5 * (u * u + v * v));
      out.p[k * 4 + 1][c] = a * (l1 * rho + l3 * rho * u);
      out.p[k * 4 + 2][c] = a * (l2 * rho + l3 * rho * v);
      out.p[k * 4 + 3][c] = a * l3 / (g.gamma[k] - 1.0);
    }
  }
}

// ---------------------------------------------------------------------
// host wrappers

static Planes4 p4(double *const a[4]) {
  Planes4 r;
  for (int m = 0; m < 4; m++) r.p[m] = a[m];
  return r;
}
static Planes8 p8(double *const a[2][4]) {
  Planes8 r;
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++) r.p[k * 4 + m] = a ? a[k][m] : nullptr;
  return r;
}

void launch_adj_rhs(const Grid &g, double *const W[2][4], const unsigned long long *lf,
                    const double *dtp, double fac, double *const mu[2][4], const double *ax,
                    const double *ay, const double *phi, const double *sx, const double *sy,
                    const int *cut, const int *ncut, int cut_cap, double *const G[40],
                    double *const SPp[8], double *const lw[2][4], cudaStream_t st) {
  Planes40 GG;
  for (int q = 0; q < 40; q++) GG.p[q] = G[q];
  Planes8 SP;
  for (int q = 0; q < 8; q++) SP.p[q] = SPp[q];
  for (int k = 0; k < 2; k++)
    for (int m = 0; m < 4; m++)
      cudaMemsetAsync(lw[k][m], 0, sizeof(double) * (size_t)g.PX * g.PY, st);
  for (int k = 0; k < 2; k++) {
    for (int d = 0; d < g.dim; d++) {
      long long nf = (long long)(g.nx + (d == 0)) * (g.ny + (d == 1));
      long long nc = d == 0 ? (long long)(g.nx + 2 * SIF_GH) * g.ny
                            : (long long)g.nx * (g.ny + 2 * SIF_GH);
      launch_k(k_adj_split, blocks_for(nc, 256), 256, 0, st, g, k, d, p4(W[k]), lf, SP);
      launch_k(k_adj_face, blocks_for(4 * nf, 128), 128, 0, st, g, k, d, SP, d == 0 ? ax : ay,
                                                          p4(mu[k]), dtp, fac, GG);
      launch_k(k_adj_gather, blocks_for(nc, 256), 256, 0, st, g, k, d, p4(W[k]), d == 0 ? ax : ay, lf,
                                                        GG, p4(lw[k]));
    }
  }
  long long n = (long long)g.nx * g.ny;
  launch_k(k_adj_ghost, blocks_for(n), 256, 0, st, g, p8(lw));
  launch_k(k_adj_interface, blocks_for(cut_cap, 128, 2432), 128, 0, st, g, p8(W), phi, sx, sy, cut,
                                                                   ncut, p8(mu), dtp, fac, p8(lw));
  sif_note_launches(6 * g.dim + 2);
}

void launch_adj_extension(const Grid &g, double *const lw[2][4], const ExtPlan *plan, int cap,
                          int work, const int *band, const int *nband, const int *map,
                          double *tmp, cudaStream_t st) {
  dim3 grid(blocks_for(work, 128, 2432), 2);
  double *buf[2] = {tmp, tmp + (size_t)8 * cap};
  launch_k(k_adj_ext_load, grid, 128, 0, st, p8(lw), band, nband, cap, buf[0]);
  int cur = 0;
  for (int it = 0; it < g.ext_iters; it++) {
    launch_k(k_adj_ext_sweep, grid, 128, 0, st, g, plan, cap, band, nband, map, buf[cur], buf[cur ^ 1],
                                          p8(lw));
    cur ^= 1;
  }
  launch_k(k_adj_ext_store, grid, 128, 0, st, p8(lw), band, nband, cap, buf[cur]);
  sif_note_launches(g.ext_iters + 2);
}

void launch_adj_prim(const Grid &g, double *const W[2][4], const double *alpha,
                     const unsigned char *const nostate[2], double *const lw[2][4],
                     double *const out[2][4], double *const A[2][4], double ca,
                     double *const B[2][4], double cb, cudaStream_t st) {
  long long n = (long long)g.nx * g.ny;
  launch_k(k_adj_prim, blocks_for(n), 256, 0, st, g, p8(W), alpha, nostate[0], nostate[1], p8(lw),
                                            p8(out), p8(A), ca, p8(B), cb);
  sif_note_launches(1);
}

void launch_adj_init(const Grid &g, double *const prim[2][4], const double *alpha,
                     double *const lam[2][4], double *const out[2][4], cudaStream_t st) {
  long long n = (long long)g.nx * g.ny;
  launch_k(k_adj_init, blocks_for(n), 256, 0, st, g, p8(prim), alpha, p8(lam), p8(out));
  sif_note_launches(1);
}

SIF_TU_LAUNCH_READER(adj)
